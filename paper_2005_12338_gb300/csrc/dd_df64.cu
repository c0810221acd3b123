// The deterministic block's dense products (S7) in double-float arithmetic on
// the fp32 pipes: GB300 issues fp32 FMAs about 60 times faster than fp64 ones,
// so each fp64 operand is carried as a (hi, lo) pair of floats and every
// multiply-add is done with error-free transformations (dd_arith.cuh); about
// a dozen fp32 operations replace one DFMA, at ~1e-13 relative error.
#include <climits>
#include <algorithm>

#include "dd_arith.cuh"
#include "dd_df64.cuh"

namespace rssri {
namespace {

int grid_cap(long long work, int threads) {
  long long b = (work + threads - 1) / threads;
  return (int)(b < 1 ? 1 : (b > 152 * 32 ? 152 * 32 : b));
}

// range[0] |= 1 when the largest magnitude of x lies outside [2^-40, 2^40]
// (zero arrays pass): the block maxima of the exponent field go to range[1],
// and the last block to finish (range[2] counts them) checks and resets both.
__global__ void to_df64_kernel(const double *__restrict__ x, long long len, float2 *__restrict__ y,
                               int *__restrict__ range) {
  int mx = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len;
       e += (long long)gridDim.x * blockDim.x) {
    const double v = x[e];
    const float hi = __double2float_rn(v);
    y[e] = make_float2(hi, __double2float_rn(v - (double)hi));
    mx = max(mx, (int)((__double_as_longlong(v) >> 52) & 0x7FF));
  }
  if (!range) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __shared__ int smax;
  __shared__ bool last;
  if (threadIdx.x == 0) smax = 0;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) atomicMax(&smax, mx);
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicMax(&range[1], smax);
    __threadfence();
    last = atomicAdd(&range[2], 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    const int m = atomicExch(&range[1], 0);
    // the exponent field of 2^k is 1023 + k
    if (m != 0 && (m < 1023 - 40 || m > 1023 + 40)) atomicOr(&range[0], 1);
    atomicExch(&range[2], 0);
  }
}

// One block per segment c of len values: e[c] = the exponent of the segment's
// largest magnitude (2^e <= max < 2^(e+1); 0 for a zero segment) and
// y = pairs of x 2^-e (an exact power-of-two scaling).
__global__ void __launch_bounds__(1024) to_df64_scaled_kernel(const double *__restrict__ x,
                                                              long long len,
                                                              float2 *__restrict__ y,
                                                              int *__restrict__ e_out) {
  const long long base = (long long)blockIdx.x * len;
  int mx = 0;
  for (long long i = threadIdx.x; i < len; i += blockDim.x)
    mx = max(mx, (int)((__double_as_longlong(x[base + i]) >> 52) & 0x7FF));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __shared__ int smax;
  if (threadIdx.x == 0) smax = 0;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) atomicMax(&smax, mx);
  __syncthreads();
  const int e = smax ? smax - 1023 : 0;
  if (threadIdx.x == 0) e_out[blockIdx.x] = e;
  for (long long i = threadIdx.x; i < len; i += blockDim.x) {
    const double v = scalbn(x[base + i], -e);
    const float hi = __double2float_rn(v);
    y[base + i] = make_float2(hi, __double2float_rn(v - (double)hi));
  }
}

// x *= 2^(mult e[0])
__global__ void scale_pow2_kernel(double *__restrict__ x, long long len,
                                  const int *__restrict__ e, int mult) {
  const int k = mult * e[0];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x)
    x[i] = scalbn(x[i], k);
}

// ------------------------------------------------- double-float products --
// C = alpha op(A) op(B) with A, B already split into (hi, lo) float pairs.
// MODE 0: strided operands; MODE 1: segmented (A(m,kk) = A[col[s0+kk]*lda + m],
// B(kk,q) = B[(s0+kk)*ldb + q], s0 = seg[b]).  OUT 0: fp64 C (or raw fp64
// partials of a K chunk); OUT 1: C written as (hi, lo) pairs.  K goes through
// shared memory in slabs; after each slab the running pairs are renormalised
// exactly (Fast2Sum) and every 256 terms they are added into float-pair
// totals, so the only fp64 work is the conversion of the outputs.
//
// Tile geometries: TY x TX threads, each owning TI x TJ outputs at strides
// TY and TX; K in slabs of BK; MINB resident CTAs per SM asked of the
// compiler.  G64: 64 x 64 tiles (256 threads); G40: 40 x 40 tiles (64
// threads, 25 outputs each), for shapes such as N = 200 and N_aux = 600 that
// 64-wide tiles would pad by up to 64%.
// KU: how many k steps of a slab are unrolled; a fully unrolled slab (3-5 k
// steps x 16-25 multiply-adds x 12 instructions each) outgrew the instruction
// cache (ncu: "no instruction" the top stall).
template <int TY_, int TX_, int TI_, int TJ_, int BK_, int MINB_, int KU_>
struct DfGeo {
  static constexpr int TY = TY_, TX = TX_, TI = TI_, TJ = TJ_, BK = BK_, MINB = MINB_, KU = KU_;
  static constexpr int BM = TY * TI, BN = TX * TJ, NT = TY * TX;
};
using G64 = DfGeo<16, 16, 4, 4, 16, 2, 4>;
using G40 = DfGeo<8, 8, 5, 5, 8, 6, 1>;

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
#pragma unroll GEO::KU
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

cudaError_t to_df64_scaled(const double *x, int segments, long long len, float2 *y, int *e,
                           cudaStream_t s) {
  if (segments <= 0 || len <= 0) return cudaSuccess;
  to_df64_scaled_kernel<<<segments, 1024, 0, s>>>(x, len, y, e);
  ++launch_counter();
  return cudaGetLastError();
}

cudaError_t scale_pow2(double *x, long long len, const int *e, int mult, cudaStream_t s) {
  if (len <= 0) return cudaSuccess;
  scale_pow2_kernel<<<grid_cap(len, 256), 256, 0, s>>>(x, len, e, mult);
  ++launch_counter();
  return cudaGetLastError();
}

cudaError_t to_df64(const double *x, long long len, float2 *y, cudaStream_t s, int *range) {
  if (len <= 0) return cudaSuccess;
  to_df64_kernel<<<grid_cap(len, 256), 256, 0, s>>>(x, len, y, range);
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

double df_gemm_flops(const DfGemm &g) {
  if (!g.sym) return 2.0 * g.M * (double)g.N * g.K * g.batch;
  // symmetric: only the tiles on and above the diagonal are computed
  const int bm = use_g40(g.M, g.N) ? G40::BM : G64::BM;
  const int t = ceil_div(g.M, bm);
  double f = 0.0;
  for (int i = 0; i < t; ++i)
    for (int j = i; j < t; ++j)
      f += 2.0 * std::min(bm, g.M - i * bm) * (double)std::min(bm, g.N - j * bm) * g.K;
  return f * g.batch;
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
