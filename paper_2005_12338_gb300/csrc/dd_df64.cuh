// Double-float (fp32 pair) kernels of the deterministic block; see dd_df64.cu.
#pragma once

#include "common.cuh"

namespace rssri {

// y[e] = (hi, lo) with hi = fl32(x[e]), lo = fl32(x[e] - hi).
cudaError_t to_df64(const double *x, long long len, float2 *y, cudaStream_t s);
// T[m][q][j] = sum_{a in row m} sum_{b in row j} D[a*P+b] * At[(col[a]*n+col[b])*naux+q],
// D and At in double-float, T in fp64.
cudaError_t dd_exchange_spmm_df64(const int *rowptr, const int *pcol, const float2 *D, int P,
                                  const float2 *At, int n, int naux, double *T, cudaStream_t s);

}  // namespace rssri
