// Cluster-cooperative exact projection onto F = {mu^T x >= R, 1^T x = 1, x >= 0}
// (Sec. 3.1, Eqs. simplex-tau, simplex-proj, projF-dualpath).
//
// Search (the same mathematics as the paper's scalar dual search):
//  * inner -- the simplex threshold at fixed nu: h(tau) = sum max(w - tau, 0) - 1
//    (w = v + nu mu) is convex, decreasing, piecewise linear.  A Newton step
//    from any tau lands at or left of the root, and from the left the
//    supports are nested, so the iteration ends exactly when |S| stops
//    changing: tau = (sum_S w - 1)/|S|.  It replaces the paper's sort.
//  * outer -- phi(nu) = mu^T x(nu) is continuous, nondecreasing, piecewise
//    linear.  On the support S at the current nu the budget and return rows
//        |S| tau - nu sum_S mu = sum_S v - 1
//        sum_S mu tau - nu sum_S mu^2 = sum_S mu v - R
//    give the exact (tau, nu) of that piece (a Newton step on phi).  A
//    bracket psi(lo) < 0 <= psi(hi), psi = phi - R, is kept; the paper's
//    geometric expansion nu = 1, 2, 4, ... and bisection take over when the
//    Newton point leaves it; the search stops when the support at nu
//    reproduces nu (exact finish).  psi(0) >= 0 means the return row is
//    inactive and the simplex projection is the answer.
//
// Arithmetic designed for GB300, whose FP64 rate is ~2 lane-ops/clk/SM:
//  * every step is one reduction of |S|, sum_S v, sum_S mu, sum_S mu v,
//    sum_S mu^2; the sums are EXACT integer additions of fixed-point images
//    of the FP64 values (62-bit magnitudes scaled by the largest element,
//    converted with integer bit operations, so each image carries the full
//    FP64 mantissa), so no FP64 add runs per element or in the reduction
//    tree and the sums are at least as accurate as FP64 ones.  A thread
//    keeps each image as four 16-bit limbs summed in 32-bit registers; a
//    warp adds each limb with one redux.sync, and the limbs are recombined
//    into 128 bits only for the few cross-warp and cross-block additions;
//  * membership w_i > tau is decided in FP32 with a proven error margin;
//    only elements inside the margin repeat the test in FP64 (same result as
//    an FP64 evaluation of fma(nu, mu_i, v_i) > tau);
//  * the n elements are split over a cluster of CL thread blocks (one SM
//    each); block sums are exchanged through distributed shared memory and
//    added in rank order by every block, so all blocks hold bit-identical
//    sums and take identical decisions; the O(1) scalar FP64 logic runs on
//    one thread per block.
// The warm start (nu, tau of the previous call) only changes where the
// search begins, never the point it returns: the projection is unique.
// Warm-start shortcut: the support S0 at the hint gives, from the same
// reduction, the exact solution (nu*, tau*) of the budget and return rows on
// S0 (tau* alone at nu = 0 when the hint says the return row is inactive).
// The next reduction, at (nu*, tau*), also counts the elements whose
// membership differs from S0; none means S0 is the support at (nu*, tau*),
// so (nu*, tau*) is exact and the search ends after two reductions (the
// general search needs four when the support does not move).  Otherwise the
// general search continues from (nu*, tau*).
#pragma once

#include <cooperative_groups.h>

#include "mv_internal.cuh"

namespace mv {

namespace cg = cooperative_groups;

constexpr int kProjNT = 256;          // threads per block
constexpr int kProjMaxCL = 16;        // largest cluster
constexpr int kProjMaxLocal = 2048;   // elements per block (n <= 16 * 2048)
constexpr int kProjMaxN = kProjMaxCL * kProjMaxLocal;
constexpr int kFixBits = 62;          // fixed-point magnitude bound 2^62 (sums kept in 128 bits)

// round(d * 2^s) with integer operations only; |d| 2^s must stay below 2^62.
__device__ __forceinline__ long long to_fixed(double d, int s) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e == 0) return 0;                                    // zero or subnormal
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = e - 1075 + s;
    long long r;
    if (sh >= 0) {
        r = (long long)(m << (sh > 9 ? 9 : sh));
    } else if (sh > -64) {
        r = (long long)((m + (1ull << (-sh - 1))) >> (-sh));
    } else {
        r = 0;
    }
    return (b >> 63) ? -r : r;
}

// Biased exponent field of |d| (0 for zero).
__device__ __forceinline__ int exp_field(double d) {
    return (int)(((unsigned long long)__double_as_longlong(d) >> 52) & 0x7ff);
}

// 2^-s as an exact double (0 below the normal range).
__device__ __forceinline__ double pow2_neg(int s) {
    const int e = 1023 - s;
    if (e <= 0) return 0.0;
    if (e >= 2047) return INFINITY;
    return __longlong_as_double((long long)e << 52);
}

// Scale s such that every |q| whose exponent field is <= e satisfies |q| 2^s < 2^kFixBits.
__host__ __device__ __forceinline__ int fixed_scale(int e) { return e == 0 ? 0 : kFixBits + 1022 - e; }

// Signed 128-bit accumulator (two's complement, lo word unsigned).
struct I128 {
    unsigned long long lo;
    long long hi;
};
__device__ __forceinline__ void add128(I128 &a, long long x) {
    const unsigned long long nlo = a.lo + (unsigned long long)x;
    a.hi += (x >> 63) + (nlo < a.lo ? 1 : 0);
    a.lo = nlo;
}
__device__ __forceinline__ void add128(I128 &a, const I128 &b) {
    const unsigned long long nlo = a.lo + b.lo;
    a.hi += b.hi + (nlo < a.lo ? 1 : 0);
    a.lo = nlo;
}
__device__ __forceinline__ double i128_to_double(const I128 &a) {
    return (double)a.hi * 18446744073709551616.0 + (double)a.lo;
}
__device__ __forceinline__ I128 warp_sum_128(I128 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        I128 w;
        w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        add128(v, w);
    }
    return v;
}
// Warp-wide sum of a 32-bit integer (one instruction).
__device__ __forceinline__ int redux_add(int v) {
    int r;
    asm volatile("redux.sync.add.s32 %0, %1, 0xffffffff;" : "=r"(r) : "r"(v));
    return r;
}
// v * 2^s as a 128-bit value, s in {0, 16, 32, 48}.
__device__ __forceinline__ I128 shl128(long long v, int s) {
    I128 r;
    r.lo = (unsigned long long)v << s;
    r.hi = s == 0 ? (v >> 63) : (v >> (64 - s));
    return r;
}
// Adds the four 16-bit limbs of a fixed-point image (|x| < 2^62: the top
// limb, arithmetic, lies in [-2^14, 2^14]) to per-thread 32-bit sums.
__device__ __forceinline__ void add_limbs(int (&l)[4], long long x) {
    l[0] += (int)(x & 0xffff);
    l[1] += (int)((x >> 16) & 0xffff);
    l[2] += (int)((x >> 32) & 0xffff);
    l[3] += (int)(x >> 48);
}
// Recombines warp totals of the four limbs.
__device__ __forceinline__ I128 from_limbs(const int (&t)[4]) {
    I128 r = shl128(t[0], 0);
    add128(r, shl128(t[1], 16));
    add128(r, shl128(t[2], 32));
    add128(r, shl128(t[3], 48));
    return r;
}

// Cluster totals of one support step, as thread 0 of every block holds them.
struct SupportSums {
    double cnt, sv, sm, smv, smm;
    long long nan, diff;
};

struct ProjOut {
    double nu, tau;
    int status;
    int steps;
    int dykstra;      // 1 if the Dykstra safeguard ran
};

// Shared-memory workspace of one block of the projector.
struct ProjSmem {
    I128 part[2][kProjMaxCL][6];        // DSMEM slots: [parity][source rank][sum]
    double dpart[2][kProjMaxCL];
    int emax[kProjMaxCL][4];
    I128 wred[kProjNT / kWarp][6];
    double wredd[kProjNT / kWarp];
    int wmax[kProjNT / kWarp][4];
    // broadcast of the scalar state (written by thread 0)
    double nu, tau, dbcast, dmin, dmax;
    double mpart[2][kProjMaxCL][2];
    float nu32, tau32;
    double nu0, tau0;                   // hint whose support a verifying step compares against
    float nu032, tau032;
    int verify;
    int done, status, steps;
    int s_v, s_m, s_mv, s_mm;
    double p_v, p_m, p_mv, p_mm;        // 2^-s of the four scales
    int parity;
};

// Must run once per block before the first reduction (all threads).
__device__ inline void proj_smem_init(ProjSmem *sh) {
    if (threadIdx.x == 0) {
        sh->parity = 0;
        sh->verify = 0;
    }
    __syncthreads();
}

// Per-element arrays of the block's slice, in shared memory.
struct ProjElems {
    double *v, *mu;               // FP64 values
    float *v32, *mu32;            // FP32 images for screening
    long long *V, *M, *MV, *MM;   // fixed-point images
    int n;                        // elements in this block's slice
};

__host__ __device__ inline size_t proj_elem_bytes(int n_local) {
    return (size_t)n_local * (8 + 8 + 4 + 4 + 8 * 4) + 64;
}

__device__ inline ProjElems carve_elems(void *base, int n_local) {
    ProjElems e;
    char *p = reinterpret_cast<char *>(base);
    e.v = reinterpret_cast<double *>(p);
    p += 8 * (size_t)n_local;
    e.mu = reinterpret_cast<double *>(p);
    p += 8 * (size_t)n_local;
    e.V = reinterpret_cast<long long *>(p);
    p += 8 * (size_t)n_local;
    e.M = reinterpret_cast<long long *>(p);
    p += 8 * (size_t)n_local;
    e.MV = reinterpret_cast<long long *>(p);
    p += 8 * (size_t)n_local;
    e.MM = reinterpret_cast<long long *>(p);
    p += 8 * (size_t)n_local;
    e.v32 = reinterpret_cast<float *>(p);
    p += 4 * (size_t)n_local;
    e.mu32 = reinterpret_cast<float *>(p);
    e.n = n_local;
    return e;
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ int warp_max_i(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <int CL>
__device__ __forceinline__ void cluster_barrier() {
    if constexpr (CL > 1) {
        cg::this_cluster().sync();
    } else {
        __syncthreads();
    }
}

template <int CL>
__device__ __forceinline__ int cluster_rank() {
    if constexpr (CL > 1) {
        return (int)cg::this_cluster().block_rank();
    } else {
        return 0;
    }
}

template <int CL>
struct ClusterProj {
    ProjSmem *sh;
    ProjElems el;
    // Dykstra safeguard: 4 el.n doubles of global scratch for this block
    // (v, x, p, q) and the sweep budget; without scratch the safeguard is off.
    double *dyk = nullptr;
    int dyk_iters = 0;

    // Block-then-cluster sum of the 6 per-warp 128-bit partials in
    // sh->wred (after a __syncthreads); lane k < 6 of warp 0 of every block
    // ends with total k (integer sums: exact, so the order of addition does
    // not matter).  Lane k < 6 adds value k over the warps, lane r < CL
    // stores the block totals into block r, then lane k adds value k over
    // the CL blocks.
    __device__ I128 reduce_partials() {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int par = sh->parity;
        I128 t{0ull, 0ll};
        if (warp == 0) {
            if (lane < 6)
                for (int w = 0; w < kProjNT / kWarp; ++w) add128(t, sh->wred[w][lane]);
            const int me = cluster_rank<CL>();
            I128 tk[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                tk[k].lo = __shfl_sync(0xffffffffu, t.lo, k);
                tk[k].hi = __shfl_sync(0xffffffffu, t.hi, k);
            }
            if (lane < CL) {
                I128 *dst;
                if constexpr (CL > 1) {
                    dst = cg::this_cluster().map_shared_rank(&sh->part[par][me][0], lane);
                } else {
                    dst = &sh->part[par][0][0];
                }
#pragma unroll
                for (int k = 0; k < 6; ++k) dst[k] = tk[k];
            }
        }
        cluster_barrier<CL>();
        t = I128{0ull, 0ll};
        if (warp == 0) {
            if (lane < 6)
                for (int r = 0; r < CL; ++r) add128(t, sh->part[par][r][lane]);
            if (lane == 0) sh->parity = par ^ 1;
        }
        // The next exchange writes the other parity; the one after reuses this
        // one only after another cluster barrier, so no reader is overtaken.
        return t;
    }

    // Cluster sum of one double per thread, added in a fixed order (every
    // block gets the same value); result returned to all threads.
    __device__ double reduce_double(double x) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        x = warp_sum(x);
        if (lane == 0) sh->wredd[warp] = x;
        __syncthreads();
        const int par = sh->parity;
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < kProjNT / kWarp; ++w) t += sh->wredd[w];
            const int me = cluster_rank<CL>();
            if constexpr (CL > 1) {
                cg::cluster_group cl = cg::this_cluster();
                for (int r = 0; r < CL; ++r) *cl.map_shared_rank(&sh->dpart[par][me], r) = t;
            } else {
                sh->dpart[par][0] = t;
            }
        }
        cluster_barrier<CL>();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int r = 0; r < CL; ++r) t += sh->dpart[par][r];
            sh->dbcast = t;
            sh->parity = par ^ 1;
        }
        __syncthreads();
        const double r = sh->dbcast;
        __syncthreads();
        return r;
    }

    // Cluster-wide min and max of one double per thread; result to all threads.
    __device__ void reduce_minmax(double &mn, double &mx) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        mn = warp_min(mn);
        mx = warp_max(mx);
        if (lane == 0) {
            sh->wredd[warp] = mn;
            sh->wred[warp][0].hi = __double_as_longlong(mx);
        }
        __syncthreads();
        const int par = sh->parity;
        if (threadIdx.x == 0) {
            double a = INFINITY, b = -INFINITY;
            for (int w = 0; w < kProjNT / kWarp; ++w) {
                a = fmin(a, sh->wredd[w]);
                b = fmax(b, __longlong_as_double(sh->wred[w][0].hi));
            }
            const int me = cluster_rank<CL>();
            if constexpr (CL > 1) {
                cg::cluster_group cl = cg::this_cluster();
                for (int r = 0; r < CL; ++r) {
                    double *dst = cl.map_shared_rank(&sh->mpart[par][me][0], r);
                    dst[0] = a;
                    dst[1] = b;
                }
            } else {
                sh->mpart[par][0][0] = a;
                sh->mpart[par][0][1] = b;
            }
        }
        cluster_barrier<CL>();
        if (threadIdx.x == 0) {
            double a = INFINITY, b = -INFINITY;
            for (int r = 0; r < CL; ++r) {
                a = fmin(a, sh->mpart[par][r][0]);
                b = fmax(b, sh->mpart[par][r][1]);
            }
            sh->dmin = a;
            sh->dmax = b;
            sh->parity = par ^ 1;
        }
        __syncthreads();
        mn = sh->dmin;
        mx = sh->dmax;
        __syncthreads();
    }

    // Cluster-wide maxima of the exponent fields of |v|, |mu|, |mu v|, mu^2,
    // then the fixed-point images of the slice.  Expects el.v and el.mu set.
    __device__ void prepare() {
        int e[4] = {0, 0, 0, 0};
        for (int i = threadIdx.x; i < el.n; i += kProjNT) {
            const double v = el.v[i], m = el.mu[i];
            const double mv = m * v, mm = m * m;
            e[0] = max(e[0], exp_field(v));
            e[1] = max(e[1], exp_field(m));
            e[2] = max(e[2], exp_field(mv));
            e[3] = max(e[3], exp_field(mm));
            el.MV[i] = __double_as_longlong(mv);   // converted in place below
            el.MM[i] = __double_as_longlong(mm);
            el.v32[i] = (float)v;
            el.mu32[i] = (float)m;
        }
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int k = 0; k < 4; ++k) e[k] = warp_max_i(e[k]);
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < 4; ++k) sh->wmax[warp][k] = e[k];
        __syncthreads();
        if (threadIdx.x == 0) {
            int t[4] = {0, 0, 0, 0};
            for (int w = 0; w < kProjNT / kWarp; ++w)
#pragma unroll
                for (int k = 0; k < 4; ++k) t[k] = max(t[k], sh->wmax[w][k]);
            const int me = cluster_rank<CL>();
            if constexpr (CL > 1) {
                cg::cluster_group cl = cg::this_cluster();
                for (int r = 0; r < CL; ++r) {
                    int *dst = cl.map_shared_rank(&sh->emax[me][0], r);
#pragma unroll
                    for (int k = 0; k < 4; ++k) dst[k] = t[k];
                }
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) sh->emax[0][k] = t[k];
            }
        }
        cluster_barrier<CL>();
        if (threadIdx.x == 0) {
            int t[4] = {0, 0, 0, 0};
            for (int r = 0; r < CL; ++r)
#pragma unroll
                for (int k = 0; k < 4; ++k) t[k] = max(t[k], sh->emax[r][k]);
            sh->s_v = fixed_scale(t[0]);
            sh->s_m = fixed_scale(t[1]);
            sh->s_mv = fixed_scale(t[2]);
            sh->s_mm = fixed_scale(t[3]);
            // 2^-s as exact doubles (s in [-10, 2100]: build the bits, clamp to 0)
            sh->p_v = pow2_neg(sh->s_v);
            sh->p_m = pow2_neg(sh->s_m);
            sh->p_mv = pow2_neg(sh->s_mv);
            sh->p_mm = pow2_neg(sh->s_mm);
        }
        __syncthreads();
        const int sv = sh->s_v, sm = sh->s_m, smv = sh->s_mv, smm = sh->s_mm;
        for (int i = threadIdx.x; i < el.n; i += kProjNT) {
            el.V[i] = to_fixed(el.v[i], sv);
            el.M[i] = to_fixed(el.mu[i], sm);
            el.MV[i] = to_fixed(__longlong_as_double(el.MV[i]), smv);
            el.MM[i] = to_fixed(__longlong_as_double(el.MM[i]), smm);
        }
        // emax slots are rewritten only by the next prepare(), after at least
        // one more cluster barrier.
        __syncthreads();
    }

    // i in S(nu, tau), i.e. fma(nu, mu_i, v_i) > tau in FP64, screened in FP32
    // with a proven margin (the FP64 test runs only inside it).
    __device__ __forceinline__ bool member(int i, double nu, double tau, float nu32, float tau32, float anu,
                                           float atau, bool &nan) const {
        const float c = 2.384185791015625e-07f;   // 2^-22
        const float v32 = el.v32[i], m32 = el.mu32[i];
        const float d = fmaf(nu32, m32, v32) - tau32;
        const float margin = c * (fmaf(anu, fabsf(m32), fabsf(v32)) + atau);
        if (d > margin) return true;
        if (d < -margin) return false;
        const double w = fma(nu, el.mu[i], el.v[i]);
        if (!(w == w)) nan = true;
        return w > tau;
    }

    // Sums over S = {i : fma(nu, mu_i, v_i) > tau}; totals valid in thread 0.
    // Also counts NaNs met and (when sh->verify) the elements whose
    // membership differs from S(sh->nu0, sh->tau0).
    __device__ SupportSums support_sums(double nu, double tau, float nu32, float tau32) {
        int lb[4][4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int q = 0; q < 4; ++q) lb[k][q] = 0;
        int cnt = 0, diff = 0;
        const float anu = fabsf(nu32), atau = isinf(tau32) ? 0.f : fabsf(tau32);
        const bool verify = sh->verify != 0;
        const double nu0 = sh->nu0, tau0 = sh->tau0;
        const float nu032 = sh->nu032, tau032 = sh->tau032;
        const float anu0 = fabsf(nu032), atau0 = isinf(tau032) ? 0.f : fabsf(tau032);
        bool nan = false;
        for (int i = threadIdx.x; i < el.n; i += kProjNT) {
            const bool in = member(i, nu, tau, nu32, tau32, anu, atau, nan);
            if (verify && in != member(i, nu0, tau0, nu032, tau032, anu0, atau0, nan)) ++diff;
            if (in) {
                ++cnt;
                add_limbs(lb[0], el.V[i]);
                add_limbs(lb[1], el.M[i]);
                add_limbs(lb[2], el.MV[i]);
                add_limbs(lb[3], el.MM[i]);
            }
        }
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        int tl[4][4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int q = 0; q < 4; ++q) tl[k][q] = redux_add(lb[k][q]);
        const int tcnt = redux_add(cnt), tdiff = redux_add(diff), tnan = redux_add(nan ? 1 : 0);
        if (lane < 6) {
            I128 w;
            if (lane == 0) {
                w = I128{(unsigned long long)tcnt, 0ll};
            } else if (lane == 5) {
                w = I128{(unsigned long long)tnan, (long long)tdiff};
            } else {
                // lane k (1..4) recombines image k-1; the branch-free select keeps tl in registers
                int t4[4];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    t4[q] = lane == 1 ? tl[0][q] : (lane == 2 ? tl[1][q] : (lane == 3 ? tl[2][q] : tl[3][q]));
                w = from_limbs(t4);
            }
            sh->wred[warp][lane] = w;
        }
        __syncthreads();
        const I128 t = reduce_partials();
        // lane k converts total k to FP64 (the four images with their scales)
        double d = 0.0;
        if (warp == 0 && lane < 5) {
            const double p = lane == 1 ? sh->p_v : (lane == 2 ? sh->p_m : (lane == 3 ? sh->p_mv : sh->p_mm));
            d = lane == 0 ? (double)t.lo : i128_to_double(t) * p;
        }
        SupportSums out;
        out.cnt = __shfl_sync(0xffffffffu, d, 0);
        out.sv = __shfl_sync(0xffffffffu, d, 1);
        out.sm = __shfl_sync(0xffffffffu, d, 2);
        out.smv = __shfl_sync(0xffffffffu, d, 3);
        out.smm = __shfl_sync(0xffffffffu, d, 4);
        out.nan = (long long)__shfl_sync(0xffffffffu, t.lo, 5);
        out.diff = __shfl_sync(0xffffffffu, t.hi, 5);
        return out;
    }

    // Full search.  Returns (nu, tau, status) identically in all threads.
    __device__ ProjOut search(double R, int mode, double mu_min, double mu_max, double nu_hint, double tau_hint,
                             int budget) {
        // Thread-0-owned search state.
        double lo = -INFINITY, hi = INFINITY, nu = 0.0, tau = -INFINITY, prev_cnt = -1.0;
        bool have_lo = false, have_hi = false, zero_done = false, first = true;
        bool try_fast = true, verifying = false;
        int outer = 0, inner = 0, status = MV_OK;
        const bool ge = (mode == MV_RETURN_GE);
        if (threadIdx.x == 0) {
            sh->steps = 0;
            sh->done = 0;
            sh->verify = 0;
            if (!(R <= mu_max) || (!ge && !(R >= mu_min))) {
                sh->done = 1;
                sh->status = MV_ERR_INFEASIBLE;
                sh->nu = NAN;
                sh->tau = NAN;
            } else {
                nu = (nu_hint == nu_hint) ? nu_hint : 0.0;
                if (ge && !(nu > 0.0)) nu = 0.0;
                tau = (tau_hint == tau_hint) ? tau_hint : -INFINITY;
                sh->nu = nu;
                sh->tau = tau;
                sh->nu32 = (float)nu;
                sh->tau32 = (float)tau;
                sh->status = MV_OK;
            }
        }
        __syncthreads();
        double scaleR = 0.0;
        if (threadIdx.x == 0) scaleR = fmax(fabs(R), fmax(fabs(mu_max), fabs(mu_min)));
        while (true) {
            if (sh->done) break;                       // uniform: read after a barrier
            const double enu = sh->nu, etau = sh->tau;
            const float enu32 = sh->nu32, etau32 = sh->tau32;
            const SupportSums S = support_sums(enu, etau, enu32, etau32);
            if (threadIdx.x == 0) {
                sh->steps += 1;
                const double cnt = S.cnt, sv = S.sv, sm = S.sm, smv = S.smv, smm = S.smm;
                bool finish = false, handled = false;
                double next_nu = enu, next_tau = etau;
                if (S.nan != 0) {
                    status = MV_ERR_NUMERIC;
                    finish = true;
                    handled = true;
                } else if (verifying) {
                    // the candidate was built on S(nu0, tau0); it is exact iff the support is unchanged
                    verifying = false;
                    sh->verify = 0;
                    if (S.diff == 0) {
                        nu = enu;
                        tau = etau;
                        finish = true;
                        handled = true;
                    }
                } else if (try_fast && cnt > 0.0) {
                    try_fast = false;
                    const double a = cnt, b = sm, c = smm;
                    double nc = NAN, tc = NAN;
                    bool ok = false;
                    if (ge && enu == 0.0) {            // hint: return row inactive; simplex threshold on S0
                        tc = (sv - 1.0) / a;
                        nc = 0.0;
                        ok = (smv - tc * b) - R >= 0.0;
                    } else {
                        const double det = a * c - b * b;
                        if (det > 1e-13 * a * c) {
                            nc = (b * (sv - 1.0) - a * (smv - R)) / det;
                            tc = (fma(nc, b, sv) - 1.0) / a;
                            ok = !ge || nc >= 0.0;
                        }
                    }
                    if (ok && nc == nc && tc == tc && isfinite(nc) && isfinite(tc)) {
                        sh->nu0 = enu;
                        sh->tau0 = etau;
                        sh->nu032 = enu32;
                        sh->tau032 = etau32;
                        sh->verify = 1;
                        verifying = true;
                        next_nu = nc;
                        next_tau = tc;
                        handled = true;
                    }
                }
                if (handled) {
                    // decided above
                } else if (cnt == 0.0) {               // tau >= max w: restart from the left
                    next_tau = -INFINITY;
                    first = true;
                    if (++inner > 96) {
                        status = MV_ERR_NOT_CONVERGED;
                        finish = true;
                    }
                } else if (first || cnt != prev_cnt) {  // inner Newton step
                    first = false;
                    prev_cnt = cnt;
                    next_tau = (fma(enu, sm, sv) - 1.0) / cnt;
                    if (++inner > 96) {
                        status = MV_ERR_NOT_CONVERGED;
                        finish = true;
                    }
                } else {
                    // inner converged: etau is the threshold at enu, S its support
                    inner = 0;
                    nu = enu;
                    tau = etau;
                    if (nu == 0.0) zero_done = true;
                    const double a = cnt, b = sm, c = smm;
                    const double det = a * c - b * b;
                    const bool flat = !(det > 1e-13 * a * c);
                    const double psi = flat ? (b / a - R) : ((fma(nu, c, smv) - tau * b) - R);
                    double nu_c = NAN;
                    if (ge && nu == 0.0 && psi >= 0.0) {
                        finish = true;                 // return row inactive
                    } else if (psi == 0.0) {
                        finish = true;
                    } else if (flat && fabs(psi) <= 1e-12 * scaleR) {
                        finish = true;                 // target met on a flat piece
                    } else {
                        if (!flat) {
                            nu_c = (b * (sv - 1.0) - a * (smv - R)) / det;
                            if (fabs(nu_c - nu) <= 1e-13 * fmax(1.0, fabs(nu))) finish = true;   // exact finish
                        }
                        if (!finish) {
                            if (psi < 0.0) {
                                lo = nu;
                                have_lo = true;
                            } else {
                                hi = nu;
                                have_hi = true;
                            }
                            double nxt = nu_c;
                            if (ge && nxt == nxt && nxt <= 0.0 && !zero_done) nxt = 0.0;
                            const bool inside = (nxt == nxt) && (!have_lo || nxt > lo) && (!have_hi || nxt < hi) &&
                                                (!ge || nxt >= 0.0);
                            if (!inside) {
                                if (have_lo && have_hi) {
                                    nxt = 0.5 * (lo + hi);
                                } else if (have_lo) {          // expand right: 1, 2, 4, ...
                                    nxt = (lo < 0.0) ? 0.0 : (lo == 0.0 ? 1.0 : 2.0 * lo);
                                    if (nxt == 0.0 && zero_done) nxt = 1.0;
                                } else if (ge) {
                                    nxt = 0.0;
                                } else {                       // expand left (equality mode)
                                    nxt = (hi > 0.0) ? 0.0 : (hi == 0.0 ? -1.0 : 2.0 * hi);
                                    if (nxt == 0.0 && zero_done) nxt = -1.0;
                                }
                            }
                            if (nxt == nu || ++outer >= budget) {
                                status = MV_ERR_NOT_CONVERGED;
                                finish = true;
                            } else {
                                next_nu = nxt;
                                next_tau = (fma(nxt, b, sv) - 1.0) / a;   // threshold this support predicts
                                first = true;
                            }
                        }
                    }
                }
                if (finish) {
                    sh->done = 1;
                    sh->status = status;
                    sh->nu = nu;
                    sh->tau = tau;
                    if (status == MV_ERR_NUMERIC || (status == MV_ERR_NOT_CONVERGED && !(tau == tau))) {
                        sh->nu = enu;
                        sh->tau = etau;
                    }
                } else {
                    sh->nu = next_nu;
                    sh->tau = next_tau;
                    sh->nu32 = (float)next_nu;
                    sh->tau32 = (float)next_tau;
                }
            }
            __syncthreads();
        }
        ProjOut o;
        o.nu = sh->nu;
        o.tau = sh->tau;
        o.status = sh->status;
        o.steps = sh->steps;
        o.dykstra = 0;
        __syncthreads();   // all threads read the result before the slots are reused
        return o;
    }

    // Dykstra's alternating projections between Delta and H (the safeguard
    // of Sec. 3.1), started at the v held in el.v: x = v, p = q = 0, then
    //   y = Pi_Delta(x + p), p <- x + p - y;  w = y + q,
    //   x = w + theta mu (theta = max(0, (R - mu^T w) / ||mu||^2), any sign
    //   in equality mode), q <- w - x = -theta mu,
    // until x and y agree and stop moving (1e-10 max(1, |v|_inf)) or the
    // sweep budget is spent.  Pi_Delta is the scalar search at nu = 0 with
    // the return row dropped (R = -inf).  Returns theta, the return-row
    // multiplier of the limit, and in tau_out the threshold it implies
    // (tau = v_i + theta mu_i - x_i on the support, averaged); el.v and its
    // fixed-point images are restored.
    __device__ double dykstra(double R, int mode, double mu_min, double mu_max, int budget, int &sweeps,
                              double &tau_out) {
        const int n = el.n;
        double *v0 = dyk, *x = dyk + n, *p = dyk + 2 * n, *q = dyk + 3 * n;
        double vmax = 0.0, mm = 0.0;
        for (int i = threadIdx.x; i < n; i += kProjNT) {
            const double v = el.v[i];
            v0[i] = v;
            x[i] = v;
            p[i] = 0.0;
            q[i] = 0.0;
            vmax = fmax(vmax, fabs(v));
            mm = fma(el.mu[i], el.mu[i], mm);
        }
        mm = reduce_double(mm);
        double lo = 0.0, hi = vmax;
        reduce_minmax(lo, hi);
        const double tol = 1e-10 * fmax(1.0, hi);
        double theta = 0.0;
        sweeps = 0;
        for (int it = 0; it < dyk_iters; ++it) {
            for (int i = threadIdx.x; i < n; i += kProjNT) el.v[i] = x[i] + p[i];
            __syncthreads();
            prepare();
            const ProjOut s = search(-INFINITY, MV_RETURN_GE, mu_min, mu_max, 0.0, -INFINITY, budget);
            // el.v holds x + p: y = Pi_Delta(x + p), p <- x + p - y, w = y + q (parked in q)
            double c = 0.0;
            for (int i = threadIdx.x; i < n; i += kProjNT) {
                const double y = fmax(el.v[i] - s.tau, 0.0);
                p[i] = el.v[i] - y;
                const double w = y + q[i];
                q[i] = w;
                c = fma(el.mu[i], w, c);
            }
            c = reduce_double(c);
            double th = mm > 0.0 ? (R - c) / mm : 0.0;
            if (mode == MV_RETURN_GE) th = fmax(th, 0.0);
            // x <- w + theta mu, q <- w - x; measure |x_new - x_old| and |x_new - y|
            double dev = 0.0;
            for (int i = threadIdx.x; i < n; i += kProjNT) {
                const double w = q[i];
                const double y = fmax(el.v[i] - s.tau, 0.0);
                const double xn = fma(th, el.mu[i], w);
                dev = fmax(dev, fmax(fabs(xn - x[i]), fabs(xn - y)));
                x[i] = xn;
                q[i] = w - xn;
            }
            double a = -dev, b = fabs(th - theta) * sqrt(mm);
            reduce_minmax(a, b);
            theta = th;
            sweeps = it + 1;
            if (s.status != MV_OK) break;
            if (-a <= tol && b <= tol) break;
        }
        double st = 0.0, sc = 0.0;
        for (int i = threadIdx.x; i < n; i += kProjNT) {
            el.v[i] = v0[i];
            if (x[i] > 0.0) {
                st += fma(theta, el.mu[i], v0[i]) - x[i];
                sc += 1.0;
            }
        }
        st = reduce_double(st);
        sc = reduce_double(sc);
        tau_out = sc > 0.0 ? st / sc : -INFINITY;
        prepare();
        return theta;
    }

    // The projection: the scalar search, and the Dykstra safeguard when the
    // search does not finish within its budget (scratch permitting), whose
    // (theta, tau) restarts the exact search, with at least 100 outer steps.
    __device__ ProjOut solve(double R, int mode, double mu_min, double mu_max, double nu_hint, double tau_hint,
                             int budget) {
        ProjOut o = search(R, mode, mu_min, mu_max, nu_hint, tau_hint, budget);
        if (o.status != MV_ERR_NOT_CONVERGED || dyk == nullptr || dyk_iters <= 0) return o;
        int sweeps = 0;
        double tau_d = -INFINITY;
        const double theta = dykstra(R, mode, mu_min, mu_max, budget, sweeps, tau_d);
        const int steps = o.steps;
        o = search(R, mode, mu_min, mu_max, theta, tau_d, budget > 100 ? budget : 100);
        o.steps += steps;
        o.dykstra = 1;
        return o;
    }
};

// Cluster size used for a problem of n assets: about 512 elements per block
// (two per thread), at most 16 blocks.
inline int proj_cluster_size(int64_t n) {
    if (n <= 512) return 1;
    if (n <= 1024) return 2;
    if (n <= 2048) return 4;
    if (n <= 4096) return 8;
    return 16;
}

}  // namespace mv
