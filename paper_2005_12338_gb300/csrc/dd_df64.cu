// The exchange contraction of the deterministic block (S7) in double-float
// arithmetic on the FP32 pipes.
//
// GB300 issues fp32 FMAs about 60 times faster than fp64 ones, so an fp64
// value x is carried as two floats x = hi + lo (hi = fl32(x),
// lo = fl32(x - hi): a 48-bit significand) and each multiply-add is done
// with error-free transformations: the product's rounding error comes from
// one fma (TwoProduct), the sum's from Knuth's TwoSum, and the two error
// streams are collected in a second float.  About a dozen fp32 operations
// replace one DFMA; after each pair of the sparse operand's row (~40 terms)
// the pair is renormalised exactly (Fast2Sum) and every four pairs it is
// added into an fp64 total.  The result agrees with the fp64 contraction to
// ~1e-12 relative.
#include <climits>
#include <algorithm>

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

__device__ __forceinline__ void df_mac2(float &S, float &E, float2 d, float xh, float xl) {
  // TwoProduct of the high parts plus the cross terms, then TwoSum S + p
  const float p = __fmul_rn(d.x, xh);
  float e = __fmaf_rn(d.x, xh, -p);
  e = __fmaf_rn(d.x, xl, e);
  e = __fmaf_rn(d.y, xh, e);
  const float s = __fadd_rn(S, p);
  const float bp = __fsub_rn(s, S);
  const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(s, bp)), __fsub_rn(p, bp));
  S = s;
  E = __fadd_rn(E, __fadd_rn(err, e));
}

// (TH, TL) += (S, E): double-float addition of two normalised pairs (TwoSum of
// the high parts, low parts and error added, Fast2Sum).  All fp32: on this GPU
// a few fp64 operations per output would cost as much as the products.
__device__ __forceinline__ void df_acc(float &TH, float &TL, float S, float E) {
  const float s = __fadd_rn(TH, S);
  const float bp = __fsub_rn(s, TH);
  const float err = __fadd_rn(__fsub_rn(TH, __fsub_rn(s, bp)), __fsub_rn(S, bp));
  const float t = __fadd_rn(__fadd_rn(TL, E), err);
  TH = __fadd_rn(s, t);
  TL = __fsub_rn(t, __fsub_rn(TH, s));
}

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

// ------------------------------------------------- double-float products --
// C = alpha op(A) op(B) with A, B already split into (hi, lo) float pairs.
// MODE 0: strided operands; MODE 1: segmented (A(m,kk) = A[col[s0+kk]*lda + m],
// B(kk,q) = B[(s0+kk)*ldb + q], s0 = seg[b]).  OUT 0: fp64 C (or raw fp64
// partials of a K chunk); OUT 1: C written as (hi, lo) pairs.  Each thread
// owns 4 x 4 outputs of a 64 x 64 tile; K goes in 16-deep slabs through
// shared memory; the pairs are renormalised exactly after each slab and folded
// into fp64 totals every 256 terms.
// Tile geometries: TY x TX threads, each owning TI x TJ outputs at strides
// TY and TX; K in slabs of BK; MINB resident CTAs per SM asked of the
// compiler.  G64: 64 x 64 tiles (256 threads); G40: 40 x 40 tiles (64
// threads, 25 outputs each), for shapes such as N = 200 and N_aux = 600 that
// 64-wide tiles would pad by up to 64%.
template <int TY_, int TX_, int TI_, int TJ_, int BK_, int MINB_>
struct DfGeo {
  static constexpr int TY = TY_, TX = TX_, TI = TI_, TJ = TJ_, BK = BK_, MINB = MINB_;
  static constexpr int BM = TY * TI, BN = TX * TJ, NT = TY * TX;
};
using G64 = DfGeo<16, 16, 4, 4, 16, 2>;
using G40 = DfGeo<8, 8, 5, 5, 8, 6>;

__device__ __forceinline__ void df_mac(float &S, float &E, float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  const float s = __fadd_rn(S, p);
  const float bp = __fsub_rn(s, S);
  const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(s, bp)), __fsub_rn(p, bp));
  S = s;
  E = __fadd_rn(E, __fadd_rn(err, e));
}

template <class GEO, int MODE, int TA, int TB, int OUT>
__global__ void __launch_bounds__(GEO::NT, GEO::MINB) df_gemm_kernel(
    int M, int N, int K, int kchunk, int ksplit, const float2 *__restrict__ A, long long lda,
    long long sA, const float2 *__restrict__ B, long long ldb, long long sB, void *__restrict__ Cv,
    long long ldc, long long sC, double alpha, int partial, int sym, const int *__restrict__ seg,
    const int *__restrict__ col) {
  constexpr int DBM = GEO::BM, DBN = GEO::BN, DBK = GEO::BK, DNT = GEO::NT;
  constexpr int TY = GEO::TY, TX = GEO::TX, TI = GEO::TI, TJ = GEO::TJ;
  __shared__ float2 As[2][DBK][DBM + 1];
  __shared__ float2 Bs[2][DBK][DBN + 1];
  constexpr int LA = DBM * DBK / DNT, LB = DBN * DBK / DNT;
  static_assert(LA * DNT == DBM * DBK && LB * DNT == DBN * DBK, "tile loads");
  constexpr bool AK = (MODE == 0 && TA == 0), BKc = (MODE == 0 && TB == 1);
  // symmetric result: only the tiles on and above the diagonal are computed
  if (sym && blockIdx.y > blockIdx.x) return;
  const int z = blockIdx.z;
  const int b = z / ksplit, ks = z % ksplit;
  int kbeg, kend;
  long long s0 = 0;
  if (MODE == 1) {
    s0 = seg[b];
    kbeg = 0;
    kend = seg[b + 1] - seg[b];
  } else {
    kbeg = ks * kchunk;
    kend = min(K, kbeg + kchunk);
    A += (long long)b * sA;
    B += (long long)b * sB;
  }
  const int row0 = blockIdx.y * DBM, col0 = blockIdx.x * DBN;
  const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
  // thread (tx, ty) owns rows ty + TY i and columns tx + TX j of the tile, so
  // that a warp's shared-memory reads are a broadcast or two (A) and runs of
  // consecutive pairs (B)
  float TH[TI][TJ], TL[TI][TJ];
  float S[TI][TJ], E[TI][TJ];
#pragma unroll
  for (int i = 0; i < TI; ++i)
#pragma unroll
    for (int j = 0; j < TJ; ++j) TH[i][j] = TL[i][j] = S[i][j] = E[i][j] = 0.0f;
  float2 ra[LA], rb[LB];
  const float2 zero = make_float2(0.f, 0.f);
  auto load = [&](int kt) {
#pragma unroll
    for (int r = 0; r < LA; ++r) {
      const int e = tid + r * DNT;
      const int i = AK ? e / DBK : e % DBM, k = AK ? e % DBK : e / DBM;
      const int gi = row0 + i, gk = kt + k;
      float2 v = zero;
      if (gi < M && gk < kend) {
        if (MODE == 1) v = A[(long long)col[s0 + gk] * lda + gi];
        else if (TA == 0) v = A[(long long)gi * lda + gk];
        else v = A[(long long)gk * lda + gi];
      }
      ra[r] = v;
    }
#pragma unroll
    for (int r = 0; r < LB; ++r) {
      const int e = tid + r * DNT;
      const int j = BKc ? e / DBK : e % DBN, k = BKc ? e % DBK : e / DBN;
      const int gj = col0 + j, gk = kt + k;
      float2 v = zero;
      if (gj < N && gk < kend) {
        if (MODE == 1) v = B[(s0 + gk) * ldb + gj];
        else if (TB == 0) v = B[(long long)gk * ldb + gj];
        else v = B[(long long)gj * ldb + gk];
      }
      rb[r] = v;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int r = 0; r < LA; ++r) {
      const int e = tid + r * DNT;
      const int i = AK ? e / DBK : e % DBM, k = AK ? e % DBK : e / DBM;
      As[buf][k][i] = ra[r];
    }
#pragma unroll
    for (int r = 0; r < LB; ++r) {
      const int e = tid + r * DNT;
      const int j = BKc ? e / DBK : e % DBN, k = BKc ? e % DBK : e / DBN;
      Bs[buf][k][j] = rb[r];
    }
  };
  constexpr int FOLD = 256 / DBK;
  int slab = 0;
  if (kbeg < kend) {
    load(kbeg);
    store(0);
    __syncthreads();
    int buf = 0;
    for (int kt = kbeg; kt < kend; kt += DBK) {
      const bool more = kt + DBK < kend;
      if (more) load(kt + DBK);
#pragma unroll
      for (int kk = 0; kk < DBK; ++kk) {
        float2 a[TI], bb[TJ];
#pragma unroll
        for (int i = 0; i < TI; ++i) a[i] = As[buf][kk][ty + TY * i];
#pragma unroll
        for (int j = 0; j < TJ; ++j) bb[j] = Bs[buf][kk][tx + TX * j];
#pragma unroll
        for (int i = 0; i < TI; ++i)
#pragma unroll
          for (int j = 0; j < TJ; ++j) df_mac(S[i][j], E[i][j], a[i], bb[j]);
      }
      ++slab;
#pragma unroll
      for (int i = 0; i < TI; ++i)
#pragma unroll
        for (int j = 0; j < TJ; ++j) {
          const float sn = __fadd_rn(S[i][j], E[i][j]);
          E[i][j] = __fsub_rn(E[i][j], __fsub_rn(sn, S[i][j]));
          S[i][j] = sn;
          if (slab == FOLD || !more) {
            df_acc(TH[i][j], TL[i][j], S[i][j], E[i][j]);
            S[i][j] = E[i][j] = 0.0f;
          }
        }
      if (slab == FOLD) slab = 0;
      if (more) {
        store(buf ^ 1);
        __syncthreads();
        buf ^= 1;
      }
    }
  }
  const bool neg = alpha == -1.0, unit = alpha == 1.0 || neg;
  for (int i = 0; i < TI; ++i) {
    const int gi = row0 + ty + TY * i;
    if (gi >= M) continue;
    for (int j = 0; j < TJ; ++j) {
      const int gj = col0 + tx + TX * j;
      if (gj >= N) continue;
      const float h = TH[i][j], l = TL[i][j];
      if (partial) {
        static_cast<double *>(Cv)[(long long)z * M * N + (long long)gi * N + gj] =
            (double)h + (double)l;
      } else {
        const long long o = (long long)b * sC + (long long)gi * ldc + gj;
        if (OUT == 0) {
          const double v = (double)h + (double)l;
          static_cast<double *>(Cv)[o] = unit ? (neg ? -v : v) : alpha * v;
        } else if (unit) {
          static_cast<float2 *>(Cv)[o] = neg ? make_float2(-h, -l) : make_float2(h, l);
        } else {
          const double v = alpha * ((double)h + (double)l);
          const float hi = __double2float_rn(v);
          static_cast<float2 *>(Cv)[o] = make_float2(hi, __double2float_rn(v - (double)hi));
        }
      }
    }
  }
}

// C = alpha * (sum of the ks partial products); with sym (M == N, square tiles
// of edge tile), elements of tiles below the diagonal take the transposed
// position's partials (only tiles on and above the diagonal were computed).
__global__ void df_reduce_kernel(const double *__restrict__ part, int ks, int M, int N,
                                 double *__restrict__ C, long long ldc, double alpha, int sym,
                                 int tile) {
  const long long mn = (long long)M * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < mn;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / N, j = e - i * N;
    const long long src = (sym && i / tile > j / tile) ? j * N + i : e;
    double s = 0.0;
    for (int k = 0; k < ks; ++k) s += part[k * mn + src];
    C[i * ldc + j] = alpha * s;
  }
}

// C[i][j] = C[j][i] for the elements of tiles below the diagonal (sym, no split).
__global__ void df_mirror_kernel(double *__restrict__ C, long long ldc, int M, int tile) {
  const long long mm = (long long)M * M;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < mm;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / M, j = e - i * M;
    if (i / tile > j / tile) C[i * ldc + j] = C[j * ldc + i];
  }
}

__global__ void gather_rows_f2_kernel(const float2 *__restrict__ src, const int *__restrict__ idx,
                                      int ncols, float2 *__restrict__ dst) {
  const int r = blockIdx.x;
  const float2 *s = src + (long long)idx[r] * ncols;
  float2 *d = dst + (long long)r * ncols;
  for (int c = threadIdx.x; c < ncols; c += blockDim.x) d[c] = s[c];
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
  if (n <= 0 || naux <= 0) return cudaSuccess;
  dim3 grid(ceil_div(naux, SQW), ceil_div(n, 4 * SWARPS), n);
  if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidValue;
  dd_spmm_warp_df64_kernel<<<grid, 32 * SWARPS, 0, s>>>(rowptr, pcol, D, P, At, n, naux, T);
  ++launch_counter();
  return cudaGetLastError();
}

namespace {

// 40-wide tiles only where 64-wide ones would pad the output by more than 30%
// more: a 64-wide CTA issues better (16 warps per SM against 12, measured
// 73% against 51-55% of the FMA pipe), so it wins unless it wastes more.
bool use_g40(int M, int N) {
  const long long a64 = (long long)ceil_div(M, 64) * 64 * ceil_div(N, 64) * 64;
  const long long a40 = (long long)ceil_div(M, 40) * 40 * ceil_div(N, 40) * 40;
  return 10 * a64 > 13 * a40;
}

// Split of K (fp64 output, batch 1, few tiles, long K) into ks chunks of kc.
template <class GEO>
void df_plan(const DfGemm &g, int *ks_out, int *kc_out) {
  const long long tiles = (long long)ceil_div(g.M, GEO::BM) * ceil_div(g.N, GEO::BN) * g.batch;
  const long long target = 2LL * GEO::MINB * 152;  // resident CTAs x 2 waves
  int ks = 1;
  if (g.C64 && g.batch == 1 && tiles < target / 2 && g.K >= 1024) {
    ks = (int)std::min<long long>((target + tiles - 1) / tiles, g.K / 256);
    ks = std::max(1, std::min(ks, 256));
  }
  const int kc = ((ceil_div(g.K, ks) + GEO::BK - 1) / GEO::BK) * GEO::BK;
  *kc_out = kc;
  *ks_out = std::max(1, ceil_div(g.K, kc));
}

template <class GEO>
cudaError_t df_gemm_geo(const DfGemm &g, double *work, size_t work_elems, cudaStream_t s) {
  int ks, kc;
  df_plan<GEO>(g, &ks, &kc);
  if (ks > 1 && work_elems < (size_t)ks * g.M * g.N) return cudaErrorInvalidValue;
  if (g.batch * ks > 65535) return cudaErrorInvalidValue;
  dim3 grid(ceil_div(g.N, GEO::BN), ceil_div(g.M, GEO::BM), g.batch * ks);
  void *out = ks > 1 ? (void *)work : (g.C64 ? (void *)g.C64 : (void *)g.C2);
  const int part = ks > 1;
#define RS_DF(TA, TB, OUT)                                                                \
  df_gemm_kernel<GEO, 0, TA, TB, OUT><<<grid, GEO::NT, 0, s>>>(                           \
      g.M, g.N, g.K, kc, ks, g.A, g.lda, g.sA, g.B, g.ldb, g.sB, out, g.ldc, g.sC, g.alpha, \
      part, g.sym, nullptr, nullptr)
  const int o = g.C2 ? 1 : 0;
  if (!g.transA && !g.transB) { if (o) RS_DF(0, 0, 1); else RS_DF(0, 0, 0); }
  else if (!g.transA && g.transB) { if (o) RS_DF(0, 1, 1); else RS_DF(0, 1, 0); }
  else if (g.transA && !g.transB) { if (o) RS_DF(1, 0, 1); else RS_DF(1, 0, 0); }
  else { if (o) RS_DF(1, 1, 1); else RS_DF(1, 1, 0); }
#undef RS_DF
  ++launch_counter();
  RS_TRY(cudaGetLastError());
  if (part) {
    const long long mn = (long long)g.M * g.N;
    df_reduce_kernel<<<grid_cap(mn, 256), 256, 0, s>>>(work, ks, g.M, g.N, g.C64, g.ldc, g.alpha,
                                                      g.sym, GEO::BM);
    ++launch_counter();
    RS_TRY(cudaGetLastError());
  } else if (g.sym) {
    df_mirror_kernel<<<grid_cap((long long)g.M * g.M, 256), 256, 0, s>>>(g.C64, g.ldc, g.M,
                                                                         GEO::BM);
    ++launch_counter();
    RS_TRY(cudaGetLastError());
  }
  return cudaSuccess;
}

}  // namespace

cudaError_t df_gemm(const DfGemm &g, double *work, size_t work_elems, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
  if ((g.C64 == nullptr) == (g.C2 == nullptr)) return cudaErrorInvalidValue;
  if (g.sym && (g.M != g.N || !g.C64 || g.batch != 1)) return cudaErrorInvalidValue;
  return use_g40(g.M, g.N) ? df_gemm_geo<G40>(g, work, work_elems, s)
                           : df_gemm_geo<G64>(g, work, work_elems, s);
}

size_t df_gemm_work(const DfGemm &g) {
  int ks, kc;
  if (use_g40(g.M, g.N)) df_plan<G40>(g, &ks, &kc);
  else df_plan<G64>(g, &ks, &kc);
  return ks > 1 ? (size_t)ks * g.M * g.N : 0;
}

cudaError_t df_gemm_segmented(int batch, int M, int N, const int *seg, const int *col,
                              const float2 *A, long long lda, const float2 *B, long long ldb,
                              float2 *C, long long ldc, long long sC, cudaStream_t s) {
  if (batch <= 0 || M <= 0 || N <= 0) return cudaSuccess;
  const bool g40 = use_g40(M, N);
  for (int b0 = 0; b0 < batch; b0 += 65535) {
    const int nb = std::min(65535, batch - b0);
    if (g40) {
      dim3 grid(ceil_div(N, G40::BN), ceil_div(M, G40::BM), nb);
      df_gemm_kernel<G40, 1, 1, 0, 1><<<grid, G40::NT, 0, s>>>(
          M, N, 0, 0, 1, A, lda, 0, B, ldb, 0, C + (long long)b0 * sC, ldc, sC, 1.0, 0, 0,
          seg + b0, col);
    } else {
      dim3 grid(ceil_div(N, G64::BN), ceil_div(M, G64::BM), nb);
      df_gemm_kernel<G64, 1, 1, 0, 1><<<grid, G64::NT, 0, s>>>(
          M, N, 0, 0, 1, A, lda, 0, B, ldb, 0, C + (long long)b0 * sC, ldc, sC, 1.0, 0, 0,
          seg + b0, col);
    }
    ++launch_counter();
    RS_TRY(cudaGetLastError());
  }
  return cudaSuccess;
}

cudaError_t gather_rows_f2(const float2 *src, const int *idx, int P, int ncols, float2 *dst,
                           cudaStream_t s) {
  if (P <= 0) return cudaSuccess;
  gather_rows_f2_kernel<<<P, 128, 0, s>>>(src, idx, ncols, dst);
  ++launch_counter();
  return cudaGetLastError();
}

}  // namespace rssri
