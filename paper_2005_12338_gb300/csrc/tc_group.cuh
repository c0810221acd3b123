// Many bf16 / tf32 tensor-core products in one persistent launch (the
// batched chains of the reduced-precision stochastic part, Sec. III, Eq. 25
// split by Eqs. 14-15): a device work queue of 128 x BN output tiles taken
// from up to TC_GROUP_MAX products of different shapes, walked by one CTA per
// SM; two tensor-memory accumulators let the epilogue of one tile overlap the
// products of the next.
#pragma once

#include "tc_gemm.cuh"

namespace rssri {

constexpr int TC_GROUP_MAX = 24;  // products per launch (kernel parameter space)

// One product: out[z] = sum_{b in group z} sum_{s < nseg} A_s[b] B_s[b]^T, as
// in TcGemm (same operand layout and outputs); an operand with batch stride 0
// is shared by every batch entry.  bn: N tile (a multiple of 16,
// <= 256); 0 lets the launcher choose (the autotuned value for this shape, or
// the width with the least padding).
struct TcProb {
  int M = 0, N = 0, batch = 1, bpc = 1, nseg = 1;
  TcOperand A[2], B[2];
  int K[2] = {0, 0};
  float *c32 = nullptr;
  void *cop = nullptr;
  long long ldcop = 0;
  int bn = 0;
};

// Enqueue the products (any number; launched TC_GROUP_MAX at a time) on s.
// All products are of the same kind.  err: device flag of bounded waits;
// wait_polls: testing only (see TcGemm).
cudaError_t tc_group(int kind, const TcProb *probs, int np, int *err, cudaStream_t s,
                     int wait_polls = 0);

// Autotuning of the N tile: for the shape of `prob` (kind, M, N, K, segments,
// batch, bpc), time each candidate width once on the product's own buffers
// (its outputs are overwritten; call outside any stream capture) and remember
// the fastest; later launches of that shape with bn = 0 use it.  Returns the
// chosen width (at once when the shape is already tuned).
int tc_group_tune(int kind, TcProb &prob, int *err, cudaStream_t s);
// Number of shapes tuned so far (diagnostics).
int tc_group_tuned_shapes();

}  // namespace rssri
