// fp64 matrix products for the RS-SRI-GF2 path.
//
// On GB300 the fp64 ceiling is the scalar DFMA pipe (two fp64 FMAs per clock
// per SM, about 1.2 TFLOP/s for the GPU; the fp64 mma.sync path is slower),
// so these are register-tiled SIMT kernels: a 64x64 output tile per 256
// threads, 4x4 outputs per thread, 16-deep K slabs double-buffered through
// shared memory with coalesced global loads for either operand layout.
#include <algorithm>

#include "common.cuh"

namespace rssri {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;
constexpr int PAD = 2;  // keeps rows 16-byte aligned, spreads banks

// MODE 0: strided operands (transA/transB per TA/TB).
// MODE 1: segmented: A(m,kk) = A[col[s0+kk]*lda + m], B(kk,q) = B[(s0+kk)*ldb + q],
//         with s0 = seg[b] and K_b = seg[b+1] - seg[b].
template <int MODE, int TA, int TB>
__global__ void __launch_bounds__(NT) dgemm_kernel(
    int M, int N, int K, int kchunk, int ksplit, const double *__restrict__ A, long long lda,
    long long sA, const double *__restrict__ B, long long ldb, long long sB,
    double *__restrict__ C, long long ldc, long long sC, double alpha, double beta,
    int partial, const int *__restrict__ seg, const int *__restrict__ col) {
  __shared__ __align__(16) double As[2][BK][BM + PAD];
  __shared__ __align__(16) double Bs[2][BK][BN + PAD];

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
  double *Cb = partial ? C + (long long)z * M * N : C + (long long)b * sC;
  const long long ldcb = partial ? N : ldc;

  const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  double ra[4], rb[4];
  auto load = [&](int kt) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = tid + r * NT;
      int i, k;
      if (MODE == 0 && TA == 0) { i = e >> 4; k = e & 15; }
      else { k = e >> 6; i = e & 63; }
      const int gi = row0 + i, gk = kt + k;
      double v = 0.0;
      if (gi < M && gk < kend) {
        if (MODE == 1) v = A[(long long)col[s0 + gk] * lda + gi];
        else if (TA == 0) v = A[(long long)gi * lda + gk];
        else v = A[(long long)gk * lda + gi];
      }
      ra[r] = v;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = tid + r * NT;
      int j, k;
      if (MODE == 0 && TB == 1) { j = e >> 4; k = e & 15; }
      else { k = e >> 6; j = e & 63; }
      const int gj = col0 + j, gk = kt + k;
      double v = 0.0;
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
    for (int r = 0; r < 4; ++r) {
      const int e = tid + r * NT;
      int i, k;
      if (MODE == 0 && TA == 0) { i = e >> 4; k = e & 15; }
      else { k = e >> 6; i = e & 63; }
      As[buf][k][i] = ra[r];
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = tid + r * NT;
      int j, k;
      if (MODE == 0 && TB == 1) { j = e >> 4; k = e & 15; }
      else { k = e >> 6; j = e & 63; }
      Bs[buf][k][j] = rb[r];
    }
  };

  if (kbeg < kend) {
    load(kbeg);
    store(0);
    __syncthreads();
    int buf = 0;
    for (int kt = kbeg; kt < kend; kt += BK) {
      const bool more = kt + BK < kend;
      if (more) load(kt + BK);
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        const double2 a01 = *reinterpret_cast<const double2 *>(&As[buf][kk][ty * 4]);
        const double2 a23 = *reinterpret_cast<const double2 *>(&As[buf][kk][ty * 4 + 2]);
        const double2 b01 = *reinterpret_cast<const double2 *>(&Bs[buf][kk][tx * 4]);
        const double2 b23 = *reinterpret_cast<const double2 *>(&Bs[buf][kk][tx * 4 + 2]);
        const double a[4] = {a01.x, a01.y, a23.x, a23.y};
        const double bb[4] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
      }
      if (more) {
        store(buf ^ 1);
        __syncthreads();
        buf ^= 1;
      }
    }
  }

#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gi = row0 + ty * 4 + i;
    if (gi >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gj = col0 + tx * 4 + j;
      if (gj >= N) continue;
      double *p = Cb + (long long)gi * ldcb + gj;
      if (partial) *p = acc[i][j];
      else *p = (beta != 0.0) ? fma(alpha, acc[i][j], beta * *p) : alpha * acc[i][j];
    }
  }
}

// C[b] = alpha * sum_{ks} part[b][ks] + beta * C[b], fixed order over ks.
__global__ void splitk_reduce_kernel(int M, int N, int batch, int ksplit,
                                     const double *__restrict__ part, double *__restrict__ C,
                                     long long ldc, long long sC, double alpha, double beta) {
  const long long mn = (long long)M * N;
  const long long total = mn * batch;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e / mn);
    const long long r = e - (long long)b * mn;
    const int i = (int)(r / N), j = (int)(r - (long long)i * N);
    const double *p = part + (long long)b * ksplit * mn + r;
    double s = 0.0;
    for (int k = 0; k < ksplit; ++k) s += p[k * mn];
    double *c = C + (long long)b * sC + (long long)i * ldc + j;
    *c = (beta != 0.0) ? fma(alpha, s, beta * *c) : alpha * s;
  }
}

template <int TA, int TB>
cudaError_t launch_strided(const GemmArgs &g, int ksplit, int kchunk, int b0, int nb,
                           double *work, cudaStream_t s) {
  dim3 grid(ceil_div(g.N, BN), ceil_div(g.M, BM), nb * ksplit);
  const bool part = ksplit > 1;
  dgemm_kernel<0, TA, TB><<<grid, NT, 0, s>>>(
      g.M, g.N, g.K, kchunk, ksplit, g.A + (long long)b0 * g.sA, g.lda, g.sA,
      g.B + (long long)b0 * g.sB, g.ldb, g.sB, part ? work : g.C + (long long)b0 * g.sC,
      g.ldc, g.sC, g.alpha, g.beta, part ? 1 : 0, nullptr, nullptr);
  ++launch_counter();
  RS_TRY(cudaGetLastError());
  if (part) {
    const long long total = (long long)g.M * g.N * nb;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 16);
    splitk_reduce_kernel<<<blocks, 256, 0, s>>>(g.M, g.N, nb, ksplit, work,
                                                 g.C + (long long)b0 * g.sC, g.ldc, g.sC,
                                                 g.alpha, g.beta);
    ++launch_counter();
    RS_TRY(cudaGetLastError());
  }
  return cudaSuccess;
}

void split_plan(const GemmArgs &g, int *ksplit, int *kchunk) {
  const long long tiles = (long long)ceil_div(g.M, BM) * ceil_div(g.N, BN) * g.batch;
  int ks = 1;
  if (tiles < 2 * 152 && g.K >= 1024) {
    ks = (int)std::min<long long>((4 * 152 + tiles - 1) / tiles, g.K / 256);
    ks = std::max(1, std::min(ks, 256));
  }
  int kc = ceil_div(g.K, ks);
  kc = ceil_div(kc, BK) * BK;
  ks = std::max(1, ceil_div(g.K, kc));
  *ksplit = ks;
  *kchunk = std::max(kc, BK);
}

}  // namespace

int dgemm_ksplit(const GemmArgs &g) {
  int ks, kc;
  split_plan(g, &ks, &kc);
  return ks;
}

size_t dgemm_work_elems(const GemmArgs &g) {
  const int ks = dgemm_ksplit(g);
  if (ks <= 1) return 0;
  const int per = std::max(1, 65535 / ks);
  const int nb = std::min(g.batch, per);
  return (size_t)ks * nb * g.M * g.N;
}

cudaError_t dgemm(const GemmArgs &g, double *work, size_t work_elems, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
  int ks, kc;
  split_plan(g, &ks, &kc);
  if (ks > 1 && work_elems < dgemm_work_elems(g)) return cudaErrorInvalidValue;
  const int per = std::max(1, 65535 / ks);
  for (int b0 = 0; b0 < g.batch; b0 += per) {
    const int nb = std::min(per, g.batch - b0);
    cudaError_t e;
    if (!g.transA && !g.transB) e = launch_strided<0, 0>(g, ks, kc, b0, nb, work, s);
    else if (!g.transA && g.transB) e = launch_strided<0, 1>(g, ks, kc, b0, nb, work, s);
    else if (g.transA && !g.transB) e = launch_strided<1, 0>(g, ks, kc, b0, nb, work, s);
    else e = launch_strided<1, 1>(g, ks, kc, b0, nb, work, s);
    RS_TRY(e);
  }
  return cudaSuccess;
}

cudaError_t dgemm_segmented(int batch, int M, int N, const int *seg, const int *col,
                            const double *A, long long lda, const double *B, long long ldb,
                            double *C, long long ldc, long long sC, cudaStream_t s) {
  if (batch <= 0 || M <= 0 || N <= 0) return cudaSuccess;
  for (int b0 = 0; b0 < batch; b0 += 65535) {
    const int nb = std::min(65535, batch - b0);
    dim3 grid(ceil_div(N, BN), ceil_div(M, BM), nb);
    dgemm_kernel<1, 1, 0><<<grid, NT, 0, s>>>(M, N, 0, 0, 1, A, lda, 0, B, ldb, 0,
                                             C + (long long)b0 * sC, ldc, sC, 1.0, 0.0, 0,
                                             seg + b0, col);
    ++launch_counter();
    RS_TRY(cudaGetLastError());
  }
  return cudaSuccess;
}

}  // namespace rssri
