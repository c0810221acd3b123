// BF16 tensor-core products (tcgen05, TMA, TMEM) for the reduced-precision
// chain of the stochastic part (Sec. III, Eq. 25 split by Eqs. 14-15).
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace rssri {

// One K segment of a product: A[b] is M x K and B[b] is N x K, both bf16
// with K contiguous (row stride ld, batch stride sb, in elements; strides must
// be multiples of 8 elements so that every TMA row starts on 16 bytes).
struct TcOperand {
  const __nv_bfloat16 *ptr = nullptr;
  long long ld = 0, sb = 0;
  int rows = 0;
};

// out[z] = sum_{b in group z} sum_{s < nseg} A_s[b] B_s[b]^T, where the batch
// entries are taken bpc at a time (one group per z, reduced in the tensor
// memory accumulator in a fixed order).  Outputs (any may be null):
//   c32 [z][M][N] fp32 (ld = N, stride M*N), c16 [z][M][ldc16] bf16
//   (ldc16 = 0 means N), c16t [z][N][M] bf16 (the transpose).
struct TcGemm {
  int M = 0, N = 0, batch = 1, bpc = 1, nseg = 1;
  TcOperand A[2], B[2];
  int K[2] = {0, 0};
  float *c32 = nullptr;
  __nv_bfloat16 *c16 = nullptr, *c16t = nullptr;
  long long ldc16 = 0;
  int *err = nullptr;  // device flag, set non-zero if a bounded wait gives up
};

cudaError_t tc_gemm(const TcGemm &g, cudaStream_t s);
// True when the tcgen05 path can run here (driver entry point found).
bool tc_available();
// One-time per-device launch attributes; call before capturing launches.
cudaError_t tc_prepare();

}  // namespace rssri
