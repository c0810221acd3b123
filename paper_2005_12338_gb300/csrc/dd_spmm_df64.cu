// The exchange contraction of the deterministic block (S7) in double-float
// arithmetic on the fp32 pipes (dd_arith.cuh): per tau point
// T[m][Q][j] = sum_{a in row m, b in row j} v^L[a][b] At[(col a, col b)][Q]
// over the kept pairs, with the running sums renormalised exactly (Fast2Sum)
// after each pair of row m's list (~40 terms) and added into float-pair totals
// every four pairs.  The result agrees with the fp64 contraction to ~1e-12.
#include <climits>
#include <algorithm>

#include "dd_arith.cuh"
#include "dd_df64.cuh"

namespace rssri {
namespace {

// T[m][q][j] = sum_{a in row m} sum_{b in row j} D[a][b] At[(col a, col b)][q]
//
// One warp per (row m, group of 4 consecutive rows j, chunk of 128 aux
// indices q; lane t owns q0 + 4t .. q0 + 4t + 3).  For each pair a = (m, k)
// of row m and each window of SLR = 64 columns l covering the group's pairs,
// the warp writes its rows' v^L entries D[a][(j, l)] into a dense 4 x SLR table
// in shared memory (zero where (j, l) is not a kept pair) and then runs over
// the columns the group actually holds, two at a time: per column two 16-byte
// loads of At[k][l][4 aux] feed 16 multiply-adds (4 rows x 4 aux indices).
// The D entries of the next (pair, window) are loaded into registers before
// the current one is computed and the table is double-buffered, so a warp
// never waits on another warp and global latency hides behind the arithmetic.
constexpr int SLR = 64, SQW = 128, SWARPS = 4, SREG = 6;  // SREG x 8 entries per row in registers

__global__ void __launch_bounds__(32 * SWARPS) dd_spmm_warp_df64_kernel(
    const int *__restrict__ rowptr, const int *__restrict__ pcol, const float2 *__restrict__ D,
    int P, const float2 *__restrict__ At, int n, int naux, double *__restrict__ T) {
  __shared__ float2 Dt[SWARPS][2][4][SLR];
  // running pair totals (TH, TL) of the 16 outputs of each thread, touched
  // once every 4 pairs: kept in shared memory ([output][thread], conflict-free)
  __shared__ float2 Tot[16][32 * SWARPS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // aux chunks vary fastest in the launch order, so the blocks that read the
  // same rows of D run together and share them through L2
  const int q0 = blockIdx.x * SQW, j0 = (blockIdx.y * SWARPS + warp) * 4, m = blockIdx.z;
  if (j0 >= n) return;  // whole warp
  const int j1 = min(n, j0 + 4);
  const int a0 = rowptr[m], a1 = rowptr[m + 1];
  // column extent of the group's rows (columns are sorted within a row)
  int lo = INT_MAX, hi = -1;
  for (int j = j0; j < j1; ++j) {
    const int b0 = rowptr[j], b1 = rowptr[j + 1];
    if (b1 > b0) {
      lo = min(lo, pcol[b0]);
      hi = max(hi, pcol[b1 - 1]);
    }
  }
  const int nwin = hi >= lo ? (hi - lo) / SLR + 1 : 0;
  const int nstage = (a1 - a0) * nwin;
  // lane -> (row of the group, sub-lane) for the table fill
  const int r_fill = lane >> 3, sub = lane & 7;
  const int j_fill = j0 + r_fill;
  const int fb0 = j_fill < j1 ? rowptr[j_fill] : 0, fb1 = j_fill < j1 ? rowptr[j_fill + 1] : 0;
  float2 dv[SREG];
  int dc[SREG];
  auto prefetch = [&](int st) {
    const float2 *Drow = D + (long long)(a0 + st / nwin) * P;
#pragma unroll
    for (int t = 0; t < SREG; ++t) {
      const int b = fb0 + sub + 8 * t;
      dc[t] = b < fb1 ? pcol[b] : -1;
      dv[t] = b < fb1 ? Drow[b] : make_float2(0.f, 0.f);
    }
  };
  auto fill = [&](int st, int buf) {
    const int a = a0 + st / nwin, lc = lo + (st % nwin) * SLR;
    float2 *row = &Dt[warp][buf][r_fill][0];
    for (int c = sub; c < SLR; c += 8) row[c] = make_float2(0.f, 0.f);
    __syncwarp();
#pragma unroll
    for (int t = 0; t < SREG; ++t) {
      const int c = dc[t] - lc;
      if (dc[t] >= 0 && c >= 0 && c < SLR) row[c] = dv[t];
    }
    // rows longer than SREG x 8 entries: the rest straight from memory
    const float2 *Drow = D + (long long)a * P;
    for (int b = fb0 + sub + 8 * SREG; b < fb1; b += 8) {
      const int c = pcol[b] - lc;
      if (c >= 0 && c < SLR) row[c] = Drow[b];
    }
    __syncwarp();
  };

  float S[4][4], E[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      S[r][c] = E[r][c] = 0.0f;
      Tot[r * 4 + c][threadIdx.x] = make_float2(0.f, 0.f);
    }
  const int q = q0 + 4 * lane;
  const int nq = max(0, min(4, naux - q));  // valid aux indices of this lane
  const bool vec = (naux % 2) == 0 && nq == 4;  // two 16-byte aligned loads
  auto load4 = [&](const float2 *ap, float2 (&x)[4]) {
    if (vec) {
      const float4 u = __ldg(reinterpret_cast<const float4 *>(ap));
      const float4 v = __ldg(reinterpret_cast<const float4 *>(ap + 2));
      x[0] = make_float2(u.x, u.y);
      x[1] = make_float2(u.z, u.w);
      x[2] = make_float2(v.x, v.y);
      x[3] = make_float2(v.z, v.w);
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c) x[c] = c < nq ? __ldg(ap + c) : make_float2(0.f, 0.f);
    }
  };
  if (nstage > 0) {
    prefetch(0);
    fill(0, 0);
  }
  for (int st = 0; st < nstage; ++st) {
    const int buf = st & 1;
    if (st + 1 < nstage) prefetch(st + 1);
    const int a = a0 + st / nwin, lc = lo + (st % nwin) * SLR;
    const int lb = max(lo, lc), le = min(hi, lc + SLR - 1);
    // local column index li = l - lc in [0, SLR)
    const float2 *Ak = At + ((long long)pcol[a] * n + lc) * naux + q;
    const float2 *Dw = &Dt[warp][buf][0][0];
    const int le_i = le - lc;
    int li = lb - lc;
    // software pipeline over pairs of columns: two register sets alternate,
    // so the loads of columns li+2, li+3 fly while li, li+1 are multiplied
    float2 xa[4] = {}, xb[4] = {}, na[4] = {}, nb[4] = {};
    auto ld = [&](int c, float2 (&x)[4]) {
      if (c <= le_i) load4(Ak + (long long)c * naux, x);
    };
    auto mac = [&](int c, const float2 (&x)[4]) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float2 d = Dw[r * SLR + c];
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) df_mac2(S[r][cc], E[r][cc], d, x[cc].x, x[cc].y);
      }
    };
    ld(li, xa);
    ld(li + 1, xb);
    for (; li + 3 <= le_i; li += 4) {
      ld(li + 2, na);
      ld(li + 3, nb);
      mac(li, xa);
      mac(li + 1, xb);
      ld(li + 4, xa);
      ld(li + 5, xb);
      mac(li + 2, na);
      mac(li + 3, nb);
    }
    // 0 to 3 columns left; xa, xb hold li and li + 1 where those exist
    if (li + 2 <= le_i) ld(li + 2, na);
    if (li <= le_i) mac(li, xa);
    if (li + 1 <= le_i) mac(li + 1, xb);
    if (li + 2 <= le_i) mac(li + 2, na);
    // after the last window of a pair: exact renormalisation (Fast2Sum);
    // added into the pair totals every 4 pairs and at the end
    if (st % nwin == nwin - 1) {
      const int ia = st / nwin;
      const bool fold = (ia & 3) == 3 || ia + 1 == a1 - a0;
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float sn = __fadd_rn(S[r][c], E[r][c]);
          E[r][c] = __fsub_rn(E[r][c], __fsub_rn(sn, S[r][c]));
          S[r][c] = sn;
          if (fold) {
            float2 t = Tot[r * 4 + c][threadIdx.x];
            df_acc(t.x, t.y, S[r][c], E[r][c]);
            Tot[r * 4 + c][threadIdx.x] = t;
            S[r][c] = E[r][c] = 0.0f;
          }
        }
    }
    if (st + 1 < nstage) fill(st + 1, buf ^ 1);
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int qc = q + c;
    if (qc >= naux) continue;
    double *out = T + ((long long)m * naux + qc) * n;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int j = j0 + r;
      const float2 t = Tot[r * 4 + c][threadIdx.x];
      if (j < j1) out[j] = (double)t.x + (double)t.y;
    }
  }
}
}  // namespace

cudaError_t dd_exchange_spmm_df64(const int *rowptr, const int *pcol, const float2 *D, int P,
                                  const float2 *At, int n, int naux, double *T, cudaStream_t s) {
  if (n <= 0 || naux <= 0) return cudaSuccess;
  dim3 grid(ceil_div(naux, SQW), ceil_div(n, 4 * SWARPS), n);
  if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidValue;
  dd_spmm_warp_df64_kernel<<<grid, 32 * SWARPS, 0, s>>>(rowptr, pcol, D, P, At, n, naux, T);
  ++launch_counter();
  return cudaGetLastError();
}

}  // namespace rssri
