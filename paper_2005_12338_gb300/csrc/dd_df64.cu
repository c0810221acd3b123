// The exchange contraction of the deterministic block (S7) in double-float
// arithmetic on the FP32 pipes.
//
// GB300 issues fp32 FMAs about 60 times faster than fp64 ones, so an fp64
// value x is carried as two floats x = hi + lo (hi = fl32(x),
// lo = fl32(x - hi): a 48-bit significand) and each multiply-add is done
// with error-free transformations: the product's rounding error comes from
// one fma (TwoProduct), the sum's from Knuth's TwoSum, and the two error
// streams are collected in a second float.  About a dozen fp32 operations
// replace one DFMA; after each row of the sparse operand (~40 terms) the pair
// is renormalised exactly (Fast2Sum) and every four rows it is added into an
// fp64 total.  The result agrees with the fp64 contraction to ~1e-12 relative.
#include "dd_df64.cuh"

namespace rssri {
namespace {

int grid_cap(long long work, int threads) {
  long long b = (work + threads - 1) / threads;
  return (int)(b < 1 ? 1 : (b > 152 * 32 ? 152 * 32 : b));
}

__global__ void to_df64_kernel(const double *__restrict__ x, long long len, float2 *__restrict__ y) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len;
       e += (long long)gridDim.x * blockDim.x) {
    const double v = x[e];
    const float hi = __double2float_rn(v);
    y[e] = make_float2(hi, __double2float_rn(v - (double)hi));
  }
}

// T[m][q][j] = sum_{a in row m} sum_{b in row j} D[a][b] At[(col a, col b)][q]
template <int QC>
__global__ void __launch_bounds__(128) dd_spmm_df64_kernel(
    const int *__restrict__ rowptr, const int *__restrict__ pcol, const float2 *__restrict__ D,
    int P, const float2 *__restrict__ At, int n, int naux, double *__restrict__ T) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * 4 + warp;
  const int m = blockIdx.y;
  if (j >= n) return;
  const int a0 = rowptr[m], a1 = rowptr[m + 1];
  const int b0 = rowptr[j], b1 = rowptr[j + 1];
  for (int q0 = 0; q0 < naux; q0 += 32 * QC) {
    double tot[QC];
#pragma unroll
    for (int c = 0; c < QC; ++c) tot[c] = 0.0;
    const int qv = naux - q0 - lane;
    float S[QC], E[QC];
#pragma unroll
    for (int c = 0; c < QC; ++c) S[c] = E[c] = 0.0f;
    for (int a = a0; a < a1; ++a) {
      const float2 *Drow = D + (long long)a * P;
      const float2 *Ak = At + (long long)pcol[a] * n * naux + q0 + lane;
      for (int b = b0; b < b1; ++b) {
        const float2 d = Drow[b];
        const float2 *ap = Ak + (long long)pcol[b] * naux;
#pragma unroll
        for (int c = 0; c < QC; ++c) {
          if (32 * c < qv) {
            const float2 x = ap[32 * c];
            // TwoProduct of the high parts plus the cross terms
            const float p = __fmul_rn(d.x, x.x);
            float e = __fmaf_rn(d.x, x.x, -p);
            e = __fmaf_rn(d.x, x.y, e);
            e = __fmaf_rn(d.y, x.x, e);
            // TwoSum S + p
            const float s = __fadd_rn(S[c], p);
            const float bp = __fsub_rn(s, S[c]);
            const float err = __fadd_rn(__fsub_rn(S[c], __fsub_rn(s, bp)), __fsub_rn(p, bp));
            S[c] = s;
            E[c] = __fadd_rn(E[c], __fadd_rn(err, e));
          }
        }
      }
      // exact renormalisation per row (Fast2Sum); fp64 fold every 4 rows
      const bool fold = ((a - a0) & 3) == 3 || a + 1 == a1;
#pragma unroll
      for (int c = 0; c < QC; ++c) {
        const float s = __fadd_rn(S[c], E[c]);
        E[c] = __fsub_rn(E[c], __fsub_rn(s, S[c]));
        S[c] = s;
        if (fold) {
          tot[c] += (double)S[c] + (double)E[c];
          S[c] = E[c] = 0.0f;
        }
      }
    }
#pragma unroll
    for (int c = 0; c < QC; ++c)
      if (32 * c < qv) T[((long long)m * naux + q0 + lane + 32 * c) * n + j] = tot[c];
  }
}

}  // namespace

cudaError_t to_df64(const double *x, long long len, float2 *y, cudaStream_t s) {
  if (len <= 0) return cudaSuccess;
  to_df64_kernel<<<grid_cap(len, 256), 256, 0, s>>>(x, len, y);
  ++launch_counter();
  return cudaGetLastError();
}

cudaError_t dd_exchange_spmm_df64(const int *rowptr, const int *pcol, const float2 *D, int P,
                                  const float2 *At, int n, int naux, double *T, cudaStream_t s) {
  // at most 10 accumulator pairs per lane: more resident warps hide the
  // latency of the dependent TwoSum chains better than longer rows do
  static const int kQC[] = {1, 2, 3, 4, 5, 6, 8, 10};
  int best = 8;
  long long best_lanes = -1;
  for (int qc : kQC) {
    const long long passes = (naux + 32LL * qc - 1) / (32LL * qc);
    const long long lanes = passes * 32 * qc + passes * 64;
    if (best_lanes < 0 || lanes < best_lanes) {
      best_lanes = lanes;
      best = qc;
    }
  }
  dim3 grid(ceil_div(n, 4), n);
#define RS_SPMM(QC)                                                                           \
  case QC:                                                                                    \
    dd_spmm_df64_kernel<QC><<<grid, 128, 0, s>>>(rowptr, pcol, D, P, At, n, naux, T); \
    break;
  switch (best) {
    RS_SPMM(1) RS_SPMM(2) RS_SPMM(3) RS_SPMM(4) RS_SPMM(5) RS_SPMM(6) RS_SPMM(8) RS_SPMM(10)
    default: return cudaErrorInvalidValue;
  }
#undef RS_SPMM
  ++launch_counter();
  return cudaGetLastError();
}

}  // namespace rssri
