// Truncation stage of STR (trunc.cu): the k largest eigenpairs of
// K = tilde L tilde L^T.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime.h>

namespace mv {

// Workspace bytes of topk_eigen (0 if the shape is not supported).
size_t topk_workspace_size(int64_t n, int64_t m, int64_t k);

// The k largest eigenpairs of K = Ls Ls^T (Ls n x m FP32, row pitch ldS):
// L_eff (n x k FP32, row pitch ldE) column c = u_c sigma_c, sigma (k FP64),
// both in descending order; lam (device, may be NULL) receives the
// *n_lam computed eigenvalues of K in descending order (all n on the direct
// route, the b Ritz values otherwise; the first k + 1 are the accurate ones).
// lam needs room for max(n, b) doubles.  Blocking.
int topk_eigen(const float *Ls, int64_t n, int64_t m, int64_t ldS, int64_t k, float *L_eff, int64_t ldE,
               double *sigma, double *lam, int64_t *n_lam, void *ws, size_t ws_bytes, cudaStream_t s);

}  // namespace mv
