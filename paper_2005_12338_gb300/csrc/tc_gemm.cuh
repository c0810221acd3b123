// BF16 and TF32 tensor-core products (tcgen05, TMA, TMEM) for the
// reduced-precision chain of the stochastic part (Sec. III, Eq. 25 split by
// Eqs. 14-15).
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace rssri {

// Operand kinds: bf16 (kind::f16) or fp32 storage read as tf32 (kind::tf32;
// values should already be rounded to tf32, the tensor core drops the low
// mantissa bits).
enum TcKind { TC_BF16 = 0, TC_TF32 = 1 };

// One K segment of a product: A[b] is M x K and B[b] is N x K, both of the
// product's kind with K contiguous (row stride ld, batch stride sb, in
// elements; strides must be multiples of 16 bytes so that every TMA row starts
// on a 16-byte boundary).
struct TcOperand {
  const void *ptr = nullptr;
  long long ld = 0, sb = 0;
  int rows = 0;
};

// out[z] = sum_{b in group z} sum_{s < nseg} A_s[b] B_s[b]^T, where the batch
// entries are taken bpc at a time (one group per z, reduced in the tensor
// memory accumulator in a fixed order).  Outputs (either may be null):
//   c32 [z][M][N] fp32 (ld = N, stride M*N); cop [z][M][ldcop] in the operand
//   type (bf16, or fp32 rounded to tf32), ldcop = 0 meaning N.
struct TcGemm {
  int kind = TC_BF16;
  int M = 0, N = 0, batch = 1, bpc = 1, nseg = 1;
  TcOperand A[2], B[2];
  int K[2] = {0, 0};
  float *c32 = nullptr;
  void *cop = nullptr;
  long long ldcop = 0;
  int *err = nullptr;  // device flag, set non-zero if a bounded wait gives up
  // testing only: > 0 issues no copy or product and gives up every wait after
  // this many polls (the error path with nothing in flight); 0 = normal
  int wait_polls = 0;
};

cudaError_t tc_gemm(const TcGemm &g, cudaStream_t s);
// True when the tcgen05 path can run here (driver entry point found).
bool tc_available();
// One-time per-device launch attributes; call before capturing launches.
cudaError_t tc_prepare();

}  // namespace rssri
