// CountSketch stage of STR (Sec. 2.3, construction (2)): tilde L = L Phi with
// Phi(t, h(t)) = s_t and every other entry 0, i.e. column j of tilde L is
// the signed sum of the columns t of L whose period hashes to bucket j.
//
// Deterministic by construction: the periods of each bucket are listed in
// ascending order (a histogram, a scan, an atomic fill and a per-bucket
// sort), and every output is summed over its list in that order.
//
//  * MV_LAYOUT_TN (L^T stored T x n): a CTA takes 8 buckets and a chunk of
//    256 x VEC assets; each thread adds, for each bucket, the signed 16-byte
//    slices of the rows t of L^T in the bucket (a warp reads 512 contiguous
//    bytes of a row), parks the 8 results in shared memory and writes them
//    out as 8 consecutive floats of tilde L's row (n x m, row-major).
//    Every row of L^T is read once in total: HBM-bound.
//  * MV_LAYOUT_NT (L stored n x T): a CTA stages one asset row of L in
//    shared memory (T e bytes, at most 200 KB) and its threads gather the
//    buckets from it.
// FP8 rows are multiplied by their scale at the write.
#include <algorithm>

#include "mv_internal.cuh"

namespace mv {

constexpr int kCsThreads = 256;
constexpr int kCsGroup = 8;                   // buckets per CTA (TN)
constexpr int kCsLoads = 4;                   // row slices in flight per thread (TN)
constexpr int kCsNtThreads = 512;
constexpr size_t kCsNtMaxRow = 200 * 1024;    // staged row bytes (NT)
constexpr int kCsMaxBucket = 4096;            // periods per bucket the in-place sort accepts

struct CsWs {
    int *cnt, *off, *fill, *err;
    unsigned *list;                           // period | sign bit 31 (negative)
};

static size_t cs_ws_bytes(int64_t T, int64_t m) {
    return align_up(4 * (size_t)m, 256) * 2 + align_up(4 * ((size_t)m + 1), 256) + align_up(4 * (size_t)T, 256) + 256;
}

static CsWs cs_carve(void *ws, int64_t T, int64_t m) {
    CsWs w;
    char *p = reinterpret_cast<char *>(ws);
    w.cnt = reinterpret_cast<int *>(p);
    p += align_up(4 * (size_t)m, 256);
    w.fill = reinterpret_cast<int *>(p);
    p += align_up(4 * (size_t)m, 256);
    w.off = reinterpret_cast<int *>(p);
    p += align_up(4 * ((size_t)m + 1), 256);
    w.list = reinterpret_cast<unsigned *>(p);
    p += align_up(4 * (size_t)T, 256);
    w.err = reinterpret_cast<int *>(p);
    return w;
}

__global__ void cs_count_kernel(const int *__restrict__ h, int T, int m, int *__restrict__ cnt, int *__restrict__ err) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        const int b = h[t];
        if (b < 0 || b >= m) {
            atomicExch(err, 1);
            continue;
        }
        atomicAdd(&cnt[b], 1);
    }
}

// Exclusive scan of m counts by one block of 1024 threads (chunked).
__global__ void __launch_bounds__(1024) cs_scan_kernel(const int *__restrict__ cnt, int m, int *__restrict__ off) {
    __shared__ int part[1024];
    const int per = (m + 1023) / 1024;
    const int b0 = threadIdx.x * per, b1 = min(m, b0 + per);
    int s = 0;
    for (int b = b0; b < b1; ++b) s += cnt[b];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {      // inclusive Hillis-Steele scan of the chunk sums
        const int v = threadIdx.x >= d ? part[threadIdx.x - d] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int run = threadIdx.x == 0 ? 0 : part[threadIdx.x - 1];
    for (int b = b0; b < b1; ++b) {
        off[b] = run;
        run += cnt[b];
    }
    if (threadIdx.x == 1023) off[m] = part[1023];
}

__global__ void cs_fill_kernel(const int *__restrict__ h, const int8_t *__restrict__ sign, int T, int m,
                               const int *__restrict__ off, int *__restrict__ fill, unsigned *__restrict__ list) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        const int b = h[t];
        if (b < 0 || b >= m) continue;
        const int pos = off[b] + atomicAdd(&fill[b], 1);
        list[pos] = (unsigned)t | (sign[t] < 0 ? 0x80000000u : 0u);
    }
}

__device__ __forceinline__ unsigned cs_key(unsigned e) { return e & 0x7fffffffu; }

// Ascending periods within one bucket of nb entries at list[p0..): up to 16
// in registers through a fixed 16-input odd-even transposition network (a
// uniform hash leaves a few periods per bucket), more by insertion in place.
__device__ __forceinline__ void cs_sort_bucket(unsigned *__restrict__ list, int p0, int nb) {
    if (nb <= 16) {
        unsigned v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = i < nb ? list[p0 + i] : 0xffffffffu;   // padding sorts last
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int i = r & 1; i + 1 < 16; i += 2) {
                const unsigned x = v[i], y = v[i + 1];
                const bool sw = cs_key(x) > cs_key(y);
                v[i] = sw ? y : x;
                v[i + 1] = sw ? x : y;
            }
        }
#pragma unroll
        for (int i = 0; i < 16; ++i)
            if (i < nb) list[p0 + i] = v[i];
        return;
    }
    for (int p = p0 + 1; p < p0 + nb; ++p) {
        const unsigned x = list[p];
        int q = p - 1;
        while (q >= p0 && cs_key(list[q]) > cs_key(x)) {
            list[q + 1] = list[q];
            --q;
        }
        list[q + 1] = x;
    }
}

// Sort every bucket (a bucket above kCsMaxBucket periods is refused).
__global__ void cs_sort_kernel(const int *__restrict__ off, int m, unsigned *__restrict__ list, int *__restrict__ err) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < m; b += gridDim.x * blockDim.x) {
        const int p0 = off[b], nb = off[b + 1] - p0;
        if (nb > kCsMaxBucket) {
            atomicExch(err, 2);
            continue;
        }
        cs_sort_bucket(list, p0, nb);
    }
}

template <int DT>
__global__ void __launch_bounds__(kCsThreads)
cs_tn_kernel(const void *__restrict__ Lt, int64_t ld, int n, int m, const int *__restrict__ off,
             const unsigned *__restrict__ list, const float *__restrict__ rs, float *__restrict__ out, int64_t ldS) {
    using St = Store<DT>;
    constexpr int VEC = St::VEC;
    constexpr int CHUNK = kCsThreads * VEC;
    extern __shared__ __align__(16) float tile[];                 // [kCsGroup][CHUNK]
    const int j0 = blockIdx.x * kCsGroup;
    const int a0 = blockIdx.y * CHUNK;
    const int my = a0 + threadIdx.x * VEC;
    const char *base = reinterpret_cast<const char *>(Lt);
    // the 9 bucket boundaries of the group, loaded together up front
    int bnd[kCsGroup + 1];
#pragma unroll
    for (int g = 0; g <= kCsGroup; ++g) bnd[g] = __ldg(off + min(j0 + g, m));
#pragma unroll
    for (int g = 0; g < kCsGroup; ++g) {
        float acc[VEC];
#pragma unroll
        for (int q = 0; q < VEC; ++q) acc[q] = 0.f;
        if (my < n) {
            const int p1 = bnd[g + 1];
            // kCsLoads list entries, then kCsLoads row slices in flight; the
            // additions keep the ascending period order
            for (int p = bnd[g]; p < p1; p += kCsLoads) {
                unsigned e[kCsLoads];
                uint4 u[kCsLoads];
#pragma unroll
                for (int k = 0; k < kCsLoads; ++k) e[k] = p + k < p1 ? __ldg(list + p + k) : 0u;
#pragma unroll
                for (int k = 0; k < kCsLoads; ++k)
                    u[k] = p + k < p1 ? ld_stream16(base + ((int64_t)(e[k] & 0x7fffffffu) * ld + my) *
                                                              (int64_t)sizeof(typename St::elem))
                                      : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                for (int k = 0; k < kCsLoads; ++k) {
                    if (p + k >= p1) break;
                    float f[VEC];
                    St::unpack(u[k], f);
                    if (e[k] & 0x80000000u) {
#pragma unroll
                        for (int q = 0; q < VEC; ++q) acc[q] -= f[q];
                    } else {
#pragma unroll
                        for (int q = 0; q < VEC; ++q) acc[q] += f[q];
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < VEC; ++q) tile[g * CHUNK + threadIdx.x * VEC + q] = acc[q];
    }
    __syncthreads();
    // row a of tilde L gets the kCsGroup consecutive buckets j0 ..
    const bool full = j0 + kCsGroup <= m && (ldS & 3) == 0;
    for (int k = threadIdx.x; k < CHUNK; k += kCsThreads) {
        const int a = a0 + k;
        if (a >= n) break;
        const float s = rs ? rs[a] : 1.f;
        float v[kCsGroup];
#pragma unroll
        for (int g = 0; g < kCsGroup; ++g) v[g] = tile[g * CHUNK + k] * s;
        float *dst = out + (int64_t)a * ldS + j0;
        if (full) {
            *reinterpret_cast<float4 *>(dst) = make_float4(v[0], v[1], v[2], v[3]);
            *reinterpret_cast<float4 *>(dst + 4) = make_float4(v[4], v[5], v[6], v[7]);
        } else {
#pragma unroll
            for (int g = 0; g < kCsGroup; ++g)
                if (j0 + g < m) dst[g] = v[g];
        }
    }
}

template <int DT>
__global__ void __launch_bounds__(kCsNtThreads)
cs_nt_kernel(const void *__restrict__ L, int64_t ld, int T, int m, const int *__restrict__ off,
             const unsigned *__restrict__ list, const float *__restrict__ rs, float *__restrict__ out, int64_t ldS) {
    using St = Store<DT>;
    using E = typename St::elem;
    extern __shared__ __align__(16) unsigned char row[];
    const int i = blockIdx.x;
    const int es = (int)sizeof(E);
    const int64_t bytes = ((int64_t)T * es + 15) / 16 * 16;       // within the row: ld e is a multiple of 16
    const char *src = reinterpret_cast<const char *>(L) + (int64_t)i * ld * es;
    for (int64_t o = (int64_t)threadIdx.x * 16; o < bytes; o += (int64_t)kCsNtThreads * 16)
        *reinterpret_cast<uint4 *>(row + o) = ld_stream16(src + o);
    __syncthreads();
    const E *r = reinterpret_cast<const E *>(row);
    const float s = rs ? rs[i] : 1.f;
    for (int j = threadIdx.x; j < m; j += kCsNtThreads) {
        float acc = 0.f;
        const int p1 = off[j + 1];
        for (int p = off[j]; p < p1; ++p) {
            const unsigned e = __ldg(list + p);
            const int t = (int)(e & 0x7fffffffu);
            float x;
            if constexpr (DT == MV_F32) {
                x = r[t];
            } else if constexpr (DT == MV_BF16) {
                x = __bfloat162float(r[t]);
            } else {
                __half_raw hh = __nv_cvt_fp8_to_halfraw(reinterpret_cast<const __nv_fp8_storage_t *>(r)[t], __NV_E4M3);
                x = __half2float(*reinterpret_cast<__half *>(&hh));
            }
            acc = (e & 0x80000000u) ? acc - x : acc + x;
        }
        out[(int64_t)i * ldS + j] = acc * s;
    }
}

template <typename K>
static int cs_smem_attr(K k, size_t bytes) {
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess
               ? MV_OK
               : record_message(MV_ERR_CUDA, "countsketch: shared-memory attribute refused");
}

template <int DT>
static int cs_launch(int layout, const void *L, int64_t ld, int n, int T, int m, const CsWs &w, const float *rs,
                     float *out, int64_t ldS, cudaStream_t s) {
    if (layout == MV_LAYOUT_TN) {
        constexpr int CHUNK = kCsThreads * Store<DT>::VEC;
        const size_t smem = (size_t)kCsGroup * CHUNK * 4;
        MV_TRY(cs_smem_attr(cs_tn_kernel<DT>, smem));
        dim3 grid((unsigned)((m + kCsGroup - 1) / kCsGroup), (unsigned)((n + CHUNK - 1) / CHUNK));
        cs_tn_kernel<DT><<<grid, kCsThreads, smem, s>>>(L, ld, n, m, w.off, w.list, rs, out, ldS);
    } else {
        const size_t smem = ((size_t)T * dtype_size(DT) + 15) / 16 * 16;
        MV_TRY(cs_smem_attr(cs_nt_kernel<DT>, smem));
        cs_nt_kernel<DT><<<(unsigned)n, kCsNtThreads, smem, s>>>(L, ld, T, m, w.off, w.list, rs, out, ldS);
    }
    return MV_OK;
}

}  // namespace mv

using namespace mv;

extern "C" {

size_t mv_countsketch_workspace_size(int64_t T, int64_t m) {
    if (T < 1 || m < 1 || T >= (1LL << 31) || m >= (1LL << 30)) return 0;
    return cs_ws_bytes(T, m);
}

int mv_countsketch(const void *d_L, int32_t dtype, int32_t layout, const float *d_row_scale, int64_t n, int64_t T,
                   int64_t ldL, const int32_t *d_hash, const int8_t *d_sign, int64_t m, float *d_L_sketch,
                   int64_t ldS, void *d_ws, size_t ws_bytes, mv_stream_t stream) {
    if (d_L == nullptr || d_hash == nullptr || d_sign == nullptr || d_L_sketch == nullptr) return MV_ERR_INVALID_ARG;
    if (dtype != MV_F32 && dtype != MV_BF16 && dtype != MV_FP8_E4M3) return MV_ERR_INVALID_ARG;
    if (layout != MV_LAYOUT_NT && layout != MV_LAYOUT_TN) return MV_ERR_INVALID_ARG;
    if (n < 1 || T < 1 || m < 1 || ldS < m) return MV_ERR_INVALID_ARG;
    if (ldL < (layout == MV_LAYOUT_TN ? n : T)) return MV_ERR_INVALID_ARG;
    if (n >= (1LL << 31) || T >= (1LL << 31) || m >= (1LL << 30))
        return record_message(MV_ERR_UNSUPPORTED, "mv_countsketch: n and T must be below 2^31 and m below 2^30");
    const int es = dtype_size(dtype);
    if (((uintptr_t)d_L) % 16 != 0 || (ldL * es) % 16 != 0 || ((uintptr_t)d_L_sketch) % 16 != 0) return MV_ERR_INVALID_ARG;
    if (dtype == MV_FP8_E4M3 && d_row_scale == nullptr) return MV_ERR_INVALID_ARG;
    if (layout == MV_LAYOUT_NT && (size_t)T * es > kCsNtMaxRow)
        return record_message(MV_ERR_UNSUPPORTED, "countsketch: an n x T row above 200 KB does not fit shared memory; "
                                                  "store L transposed (MV_LAYOUT_TN)");
    const size_t need = cs_ws_bytes(T, m);
    if (d_ws == nullptr || ws_bytes < need || ((uintptr_t)d_ws) % 256 != 0) return MV_ERR_WORKSPACE;
    (void)cudaGetLastError();
    cudaStream_t s = (cudaStream_t)stream;
    CsWs w = cs_carve(d_ws, T, m);
    MV_CUDA_TRY(cudaMemsetAsync(w.cnt, 0, 4 * (size_t)m, s));
    MV_CUDA_TRY(cudaMemsetAsync(w.fill, 0, 4 * (size_t)m, s));
    MV_CUDA_TRY(cudaMemsetAsync(w.err, 0, sizeof(int), s));
    const int tb = (int)std::min<int64_t>((T + 255) / 256, 4096);
    cs_count_kernel<<<tb, 256, 0, s>>>(d_hash, (int)T, (int)m, w.cnt, w.err);
    cs_scan_kernel<<<1, 1024, 0, s>>>(w.cnt, (int)m, w.off);
    cs_fill_kernel<<<tb, 256, 0, s>>>(d_hash, d_sign, (int)T, (int)m, w.off, w.fill, w.list);
    cs_sort_kernel<<<(unsigned)std::min<int64_t>((m + 255) / 256, 4096), 256, 0, s>>>(w.off, (int)m, w.list, w.err);
    const float *rs = dtype == MV_FP8_E4M3 ? d_row_scale : nullptr;
    switch (dtype) {
        case MV_F32: MV_TRY(cs_launch<MV_F32>(layout, d_L, ldL, (int)n, (int)T, (int)m, w, rs, d_L_sketch, ldS, s)); break;
        case MV_BF16: MV_TRY(cs_launch<MV_BF16>(layout, d_L, ldL, (int)n, (int)T, (int)m, w, rs, d_L_sketch, ldS, s)); break;
        default: MV_TRY(cs_launch<MV_FP8_E4M3>(layout, d_L, ldL, (int)n, (int)T, (int)m, w, rs, d_L_sketch, ldS, s)); break;
    }
    MV_CUDA_TRY(cudaGetLastError());
    int err = 0;
    MV_CUDA_TRY(cudaMemcpyAsync(&err, w.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    MV_CUDA_TRY(cudaStreamSynchronize(s));
    if (err == 1) return record_message(MV_ERR_INVALID_ARG, "countsketch: a bucket index lies outside [0, m)");
    if (err == 2) return record_message(MV_ERR_UNSUPPORTED, "countsketch: a bucket holds more than 4096 periods");
    return MV_OK;
}

}  // extern "C"
