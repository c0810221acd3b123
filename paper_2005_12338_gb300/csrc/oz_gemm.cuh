// fp64-accurate products on the bf16 tensor cores by error-free digit slicing
// (the splitting idea of Ozaki, Ogita and Oishi, "Error-free transformations
// of matrix multiplication by using fast routines of matrix multiplication
// and its applications", Numer. Algorithms 59 (2012)), used for the dense
// contractions of the deterministic block (Sec. III, Eq. 20 on v^L).
//
// Each row of an fp64 operand is scaled by a power of two 2^e with every
// |x| < 2^e, rounded to a 47-bit fixed-point integer F, and written as six
// balanced base-256 digits, F = sum_p d_p 256^(5-p) with |d_p| <= 128.  The
// digits are stored in bf16 pre-scaled by 2^(-8p), so that
//     x ~= 2^(e-7) sum_p D_p,   D_p = d_p 2^(-8p),   |x - that| <= 2^(e-48).
// A product sum_k a_k b_k is then 2^(eA+eB-14) sum_{p,q} sum_k D^A_p D^B_q.
// Every bf16 x bf16 product of digits is exact in fp32, and a level
// p + q = L sums terms on the common grid 2^(-8L) with at most
// (L+1) 2^14 grid units each; over 256 terms of K the levels L = 0, 1, 2
// stay below 2^24 grid units, so the tensor core's fp32 accumulation of them
// is exact.  Levels 3 to 5 (p + q <= 5 are kept: 21 digit products; the
// dropped ones are below 2^-46 of the row maxima's product) share a fourth
// accumulator, which is ~2^-24 of the result and rounds at ~2^-48 of it.
// After every 256 terms of K the four accumulators are added into
// double-float (fp32 pair) running totals; the fp64 result is assembled once
// per output.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace rssri {

constexpr int OZ_S = 6;  // digits per fp64 value
constexpr int OZ_PRODUCTS = OZ_S * (OZ_S + 1) / 2;  // digit products kept (p + q < OZ_S)

// Digits of an fp64 matrix, K-major, interleaved by blocks of 16 columns so
// that every TMA row the products load is 128 or 64 bytes wide: with
// KB = ld / 16 blocks per row and column k = 16 kb + u,
//   digits 0-3:  d[((b rows + r) KB + kb) 64 + 16 p + u]            (p < 4)
//   digits 4-5:  d[G1 + ((b rows + r) KB + kb) 32 + 16 (p - 4) + u]  (p >= 4)
// with G1 = batch rows KB 64 (bf16, 6 batch rows ld values in all); and the
// biased fp64 exponent field of each row's largest magnitude, ef[b][r] (the
// row scale is e = max(ef, 1) - 1022).  ld >= K is a multiple of 16.
struct OzDigits {
  __nv_bfloat16 *d = nullptr;
  int *ef = nullptr;
  int batch = 1, rows = 0;
  long long K = 0, ld = 0;
};
inline size_t oz_digit_elems(const OzDigits &o) {
  return (size_t)OZ_S * o.batch * o.rows * o.ld;
}

// An fp64 source for the slicer: digit column kk of row r in batch b reads
//   k1 = kk / k2pad, k2 = kk % k2pad - k2off,
//   x[b*bs + r*rs + k1*cs1 + k2*cs2]   if 0 <= k2 < k2n, else 0.
// (A plain row-major matrix: cs2 = 1, k2pad = k2n = K, cs1 unused.)
// A double-float source (x2, pairs (hi, lo) with value hi + lo) may replace x.
struct OzView {
  const double *x = nullptr;
  const float2 *x2 = nullptr;
  long long bs = 0, rs = 0, cs1 = 0, cs2 = 1;
  long long k2pad = 0, k2n = 0;
  long long k2off = 0;  // k2 in [k2off, k2off + k2n) reads index k2 - k2off
  long long xlen = 0;  // elements of the source (bounds checks of RSSRI_CHECKS builds)
};

// Write the digits and row exponents of view v into out (rows x K per batch).
cudaError_t oz_slice(const OzView &v, const OzDigits &out, cudaStream_t s);

// C[b][i][j] = alpha * sum_k A[b][i][k] B[b'][j][k] in fp64, b' = b or 0 when
// B.batch == 1.  A: M x K, B: N x K digits.  C[b*sC + i*ldc + j].  alpha is
// +1 or -1 (anything else: cudaErrorInvalidValue).
// K is split over CTAs when the output has few tiles; the split partials go
// to `work` (oz_gemm_work() doubles) and are reduced in a fixed order.
struct OzGemm {
  OzDigits A, B;
  int M = 0, N = 0, batch = 1;
  double *C = nullptr;
  long long ldc = 0, sC = 0;
  long long ccap = 0;  // elements of C (bounds checks of RSSRI_CHECKS builds)
  double alpha = 1.0;
  int *err = nullptr;  // device flag, set non-zero if a bounded wait gives up
  // testing only: > 0 issues no copy or product and gives up every wait after
  // this many polls (the error path with nothing in flight); 0 = normal
  int wait_polls = 0;
};
size_t oz_gemm_work(const OzGemm &g);
cudaError_t oz_gemm(const OzGemm &g, double *work, size_t work_elems, cudaStream_t s);
double oz_gemm_flops(const OzGemm &g);  // tensor flops issued (digit products, padded tiles)

// The exchange contraction of the deterministic block in pair space:
//   T[j][m][q] = sum_{k, l} D[(m,k), (l,j)] At[k][l][q],
// D the pair-space v^L on the kept pairs (pidx[i*n+j] = pair index or -1).
// Output rows are tiles of 8 m x 16 j; a tile's K runs over the band of k
// around its m and of l around its j (half-width bk).  The left operand
// (built once from D by oz_exch_build) holds, per tile, the 128 rows x
// (8 + 2 bk) (16 nl16) values of D; the right operand is At sliced with
// digit rows q and columns (k, l'), l' = l + lsh (lsh in {0, 8}, so that every
// tile's window of l starts on a 16-column block) and l' padded to ldl, a
// multiple of 16: the slicer view of At takes k2pad = ldl, k2off = lsh.
struct OzExch {
  int n = 0, na = 0, bk = 0, nl16 = 0, mtiles = 0, jtiles = 0;
  long long kx = 0;  // K of a tile: (8 + 2 bk) * nl16 * 16
  long long ldl = 0;
  int lsh = 0;  // column shift of l in the right operand's digits
  int lb0 = 0;  // first 16-column block of j tile jt's window is jt + lb0
};
OzExch oz_exch_geometry(int n, int na, int bk);
// fp64 left operand [tiles][128][kx] of the exchange contraction (tiles =
// mtiles * jtiles), from D [P][P] and pidx; then sliced with oz_slice.
cudaError_t oz_exch_gather(const OzExch &x, const double *D, int P, const int *pidx,
                           double *xs, long long xs_cap, cudaStream_t s);
// T[(j*n + m)*na + q] = alpha * the contraction, fp64, alpha = +1 or -1.  X: digits [tiles][128][kx];
// At: digits [1][na][n*ldl] (k major, l' minor).
cudaError_t oz_exch(const OzExch &x, const OzDigits &X, const OzDigits &At, double *T,
                    long long tcap, double alpha, int *err, cudaStream_t s, int wait_polls = 0);
double oz_exch_flops(const OzExch &x);

// Row-batched operands of K^Q G, the block's first product (PG[i][m][Q] =
// sum over the kept pairs a = (i, k) of row i of K_P[a][Q] G[k][m]), padded to
// W columns per row i of the pair list (CSR rowptr, pair columns pcol):
//   oz_rows_kp:  out[i][Q][c] = K_P[rowptr[i] + c][Q]   ([n][na][W])
//   oz_rows_g:   out[i][m][c] = G[pcol[rowptr[i] + c]][m] ([n][n][W])
// with zeros for c >= the row's length.
cudaError_t oz_rows_kp(const double *KP, const int *rowptr, int n, int na, int W, double *out,
                       cudaStream_t s);
cudaError_t oz_rows_g(const double *G, const int *rowptr, const int *pcol, int n, int W,
                      double *out, cudaStream_t s);

// pidx[i*n + j] = index of pair (i, j) among the P kept pairs (linear
// indices pij, ascending), -1 for pairs not kept.
cudaError_t oz_pair_index(const int *pij, int P, int n, int *pidx, cudaStream_t s);
// U[(j*n + m)*na + q] += 2 L[a*na + q] for every kept pair a = (m, j):
// the direct term of the deterministic block added to the exchange term.
cudaError_t oz_fold_direct(const int *prow, const int *pcol, const double *L, int P, int n,
                           int na, double *U, cudaStream_t s);

bool oz_available();
// RSSRI_CHECKS builds: the first bounds violation any kernel of this file
// recorded since the last call, as {code, line, index low, index high}
// (code 0: none); the record is cleared.  Other builds return all zeros.
cudaError_t oz_check_fetch(int out[4]);
// Registers per thread of the product kernel and the most threads a launch of
// it may have (diagnostics).
int oz_kernel_regs(int *max_threads);

}  // namespace rssri
