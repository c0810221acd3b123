// Double-float (fp32 pair) kernels of the deterministic block; see dd_df64.cu.
#pragma once

#include "common.cuh"

namespace rssri {

// y[e] = (hi, lo) with hi = fl32(x[e]), lo = fl32(x[e] - hi).  A pair keeps
// ~48 bits only inside fp32's exponent range (normal numbers from 2^-126, and
// products whose error terms stay normal), so when range is given (3 ints,
// range[1..2] zero before the first call) range[0] |= 1 if the largest
// magnitude of x lies outside [2^-40, 2^40].
cudaError_t to_df64(const double *x, long long len, float2 *y, cudaStream_t s,
                    int *range = nullptr);
// Per segment c of len values: e[c] such that the largest magnitude lies in
// [2^e, 2^(e+1)), and y = pairs of x 2^-e (exact scaling, so that the pairs
// sit in the middle of fp32's exponent range whatever x's magnitude).
cudaError_t to_df64_scaled(const double *x, int segments, long long len, float2 *y, int *e,
                           cudaStream_t s);
// x *= 2^(mult e[0]), e read on the device.
cudaError_t scale_pow2(double *x, long long len, const int *e, int mult, cudaStream_t s);
// T[m][q][j] = sum_{a in row m} sum_{b in row j} D[a*P+b] * At[(col[a]*n+col[b])*naux+q],
// D and At in double-float, T in fp64.
cudaError_t dd_exchange_spmm_df64(const int *rowptr, const int *pcol, const float2 *D, int P,
                                  const float2 *At, int n, int naux, double *T, cudaStream_t s);

// Double-float product C = alpha op(A) op(B) on (hi, lo) float pairs; exactly
// one of C64 (fp64) and C2 (pairs) is set.  Split K (fp64 output, batch 1)
// uses `work` of df_gemm_work() doubles.
struct DfGemm {
  int M = 0, N = 0, K = 0, batch = 1;
  const float2 *A = nullptr, *B = nullptr;
  long long lda = 0, ldb = 0, sA = 0, sB = 0;
  int transA = 0, transB = 0;
  double *C64 = nullptr;
  float2 *C2 = nullptr;
  long long ldc = 0, sC = 0;
  double alpha = 1.0;
  // the product is known to be symmetric (M == N, fp64 output, batch 1):
  // only tiles on and above the diagonal are computed, the rest mirrored
  int sym = 0;
};
cudaError_t df_gemm(const DfGemm &g, double *work, size_t work_elems, cudaStream_t s);
size_t df_gemm_work(const DfGemm &g);
// Flops of the tiles df_gemm computes (2 M N K batch; with sym, only the
// tiles on and above the diagonal).
double df_gemm_flops(const DfGemm &g);
// C[b][m][q] = sum_{a in [seg[b], seg[b+1])} A[col[a]*lda + m] * B[a*ldb + q], pairs out.
cudaError_t df_gemm_segmented(int batch, int M, int N, const int *seg, const int *col,
                              const float2 *A, long long lda, const float2 *B, long long ldb,
                              float2 *C, long long ldc, long long sC, cudaStream_t s);
cudaError_t gather_rows_f2(const float2 *src, const int *idx, int P, int ncols, float2 *dst,
                           cudaStream_t s);

}  // namespace rssri
