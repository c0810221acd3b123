// Internal helpers shared by the CUDA translation units of librssri.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "rssri.h"

namespace rssri {

// Error propagation: every launcher returns cudaError_t; the API layer maps
// it to an rssri_status.
// Records the first source location of a failing call since the last error
// was reported (diagnostics: rssri_last_cuda_error).
void note_error_site(const char *file, int line);

#define RS_TRY(expr)                                  \
  do {                                                \
    cudaError_t _e = (expr);                          \
    if (_e != cudaSuccess) {                          \
      ::rssri::note_error_site(__FILE__, __LINE__);   \
      return _e;                                      \
    }                                                 \
  } while (0)

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// Kernels launched so far by the calling host thread (every launch site of
// the library increments it; the API reports per-call differences).
long long &launch_counter();

// ---------------------------------------------------------------- GEMM ----
// C[b] = alpha * op(A[b]) * op(B[b]) + beta * C[b], all fp64, row-major.
//   op(A) is M x K: element (i,k) at A[i*lda+k] (transA=0) or A[k*lda+i] (1)
//   op(B) is K x N: element (k,j) at B[k*ldb+j] (transB=0) or B[j*ldb+k] (1)
//   C is M x N at C[i*ldc+j]; batch strides sA, sB, sC (elements, may be 0).
// When M*N is small and K large, the launcher splits K into chunks written to
// `work` (ksplit * batch * M * N doubles, caller-provided) and reduces them
// in a fixed order, so results stay bitwise reproducible.
struct GemmArgs {
  int M = 0, N = 0, K = 0, batch = 1;
  const double *A = nullptr, *B = nullptr;
  double *C = nullptr;
  long long lda = 0, ldb = 0, ldc = 0;
  long long sA = 0, sB = 0, sC = 0;
  int transA = 0, transB = 0;
  double alpha = 1.0, beta = 0.0;
};
// Number of K chunks the launcher will use for `g` (1 = no split).
int dgemm_ksplit(const GemmArgs &g);
// Scratch doubles needed by dgemm() for `g`.
size_t dgemm_work_elems(const GemmArgs &g);
cudaError_t dgemm(const GemmArgs &g, double *work, size_t work_elems, cudaStream_t s);
// Edge of the tile the autotuner chose for this shape (-1 before first use).
int dgemm_tile_edge(const GemmArgs &g);

// Segmented product used by the deterministic block (Sec. III):
//   C[b][m][q] = sum_{a in [seg[b], seg[b+1])} A[col[a]*lda + m] * B[a*ldb + q]
// for b < batch, m < M, q < N; C has row stride ldc and batch stride sC.
cudaError_t dgemm_segmented(int batch, int M, int N, const int *seg, const int *col,
                            const double *A, long long lda, const double *B, long long ldb,
                            double *C, long long ldc, long long sC, cudaStream_t s);

}  // namespace rssri
