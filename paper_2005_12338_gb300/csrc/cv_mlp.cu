// Learned control variate: per-element statistics of the stochastic terms,
// orbital-pair features, and a small MLP (10 -> 256 -> 256 -> 256 -> 1, SiLU)
// trained and evaluated by the kernels in this file.
//
// With E[F(R^L, R'^L)] = Sigma_DD exactly, Sigma_c = mean F(R,R') -
// c o (mean F(R^L,R'^L) - Sigma_DD) is unbiased for any c fixed independently
// of the draws it is used with, and per element its variance is smallest at
// c* = Cov(F, F^L) / Var(F^L).  The network maps features of (i, j, tau) to
// c = 1 + y and is fitted on an independent training run by minimising
// sum w (c - c*)^2 / sum w with w = Var(F^L).  The products of the two hidden
// 256 x 256 layers, forward and backward, run on the tensor cores with bf16
// operands and fp32 accumulation (tcgen05); the 10-wide input layer, the
// 1-wide output layer, activations, loss and Adam are fp32.  Fixed-order
// reductions throughout.
#include <cuda_bf16.h>

#include "cv_mlp.cuh"
#include "tc_gemm.cuh"

namespace rssri {
namespace {

int grid_cap(long long work, int threads) {
  long long b = (work + threads - 1) / threads;
  return (int)(b < 1 ? 1 : (b > 152 * 32 ? 152 * 32 : b));
}

// ------------------------------------------------------------- sgemm -----
// C = alpha * op(A) op(B) + beta * C (row-major fp32); partial = 1 writes the
// raw sum of this block's K chunk to C + z * M * N.
template <int TA, int TB>
__global__ void __launch_bounds__(256) sgemm_kernel(int M, int N, int K, int kchunk,
                                                    const float *__restrict__ A, long long lda,
                                                    const float *__restrict__ B, long long ldb,
                                                    float *__restrict__ C, long long ldc,
                                                    float alpha, float beta, int partial) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ float As[BK][BM + 1];
  __shared__ float Bs[BK][BN + 1];
  const int z = blockIdx.z;
  const int kbeg = z * kchunk, kend = min(K, kbeg + kchunk);
  const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[4][4] = {};
  for (int kt = kbeg; kt < kend; kt += BK) {
    for (int e = tid; e < BM * BK; e += 256) {
      const int i = TA ? e % BM : e / BK, k = TA ? e / BM : e % BK;
      const int gi = row0 + i, gk = kt + k;
      float v = 0.f;
      if (gi < M && gk < kend) v = TA ? A[(long long)gk * lda + gi] : A[(long long)gi * lda + gk];
      As[k][i] = v;
    }
    for (int e = tid; e < BN * BK; e += 256) {
      const int j = TB ? e / BK : e % BN, k = TB ? e % BK : e / BN;
      const int gj = col0 + j, gk = kt + k;
      float v = 0.f;
      if (gj < N && gk < kend) v = TB ? B[(long long)gj * ldb + gk] : B[(long long)gk * ldb + gj];
      Bs[k][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  for (int i = 0; i < 4; ++i) {
    const int gi = row0 + ty * 4 + i;
    if (gi >= M) continue;
    for (int j = 0; j < 4; ++j) {
      const int gj = col0 + tx * 4 + j;
      if (gj >= N) continue;
      if (partial) {
        C[(long long)z * M * N + (long long)gi * N + gj] = acc[i][j];
      } else {
        float *p = C + (long long)gi * ldc + gj;
        *p = (beta != 0.f) ? alpha * acc[i][j] + beta * *p : alpha * acc[i][j];
      }
    }
  }
}

__global__ void sreduce_kernel(const float *__restrict__ part, int ks, int M, int N,
                               float *__restrict__ C, long long ldc, float alpha) {
  const long long mn = (long long)M * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < mn;
       e += (long long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int k = 0; k < ks; ++k) s += part[k * mn + e];
    const long long i = e / N, j = e - i * N;
    C[i * ldc + j] = alpha * s;
  }
}

// Z += b (per column), A = silu(Z) (A may be null)
__global__ void bias_silu_kernel(float *__restrict__ Z, const float *__restrict__ b, long long M,
                                 int N, float *__restrict__ A) {
  const long long total = M * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const float z = Z[e] + b[e % N];
    Z[e] = z;
    if (A) A[e] = z / (1.f + __expf(-z));
  }
}

// dZ = dA * silu'(Z)
__global__ void silu_back_kernel(const float *__restrict__ dA, const float *__restrict__ Z,
                                 long long total, float *__restrict__ dZ) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const float z = Z[e];
    const float s = 1.f / (1.f + __expf(-z));
    dZ[e] = dA[e] * s * (1.f + z * (1.f - s));
  }
}

// dst = bf16(src), elementwise
__global__ void to_bf16_kernel(const float *__restrict__ src, long long n,
                               __nv_bfloat16 *__restrict__ dst) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    dst[e] = __float2bfloat16_rn(src[e]);
}

// dst[c][r] = bf16(src[r][c]) for r < rows, c < cols (dst row stride ldd,
// columns rows..ldd-1 set to zero), through 32 x 32 shared-memory tiles
__global__ void transpose_bf16_kernel(const float *__restrict__ src, int rows, int cols,
                                      long long lds, __nv_bfloat16 *__restrict__ dst,
                                      long long ldd) {
  __shared__ float t[32][33];
  const long long r0 = (long long)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int k = ty; k < 32; k += blockDim.x >> 5) {
    const long long r = r0 + k;
    const int c = c0 + tx;
    t[k][tx] = (r < rows && c < cols) ? src[r * lds + c] : 0.f;
  }
  __syncthreads();
  for (int k = ty; k < 32; k += blockDim.x >> 5) {
    const int c = c0 + k;
    const long long r = r0 + tx;
    if (c < cols && r < ldd) dst[(long long)c * ldd + r] = __float2bfloat16_rn(t[tx][k]);
  }
}

// out[j] = sum_i X[i][j], i in order (one thread per column)
__global__ void colsum_kernel(const float *__restrict__ X, int M, int N, float *__restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  float s = 0.f;
  for (int i = 0; i < M; ++i) s += X[(long long)i * N + j];
  out[j] = s;
}

// dy = 2 w (1 + y - t) / sum w ; loss = sum w (1 + y - t)^2 / sum w
__global__ void loss_kernel(const float *__restrict__ y, const float *__restrict__ t,
                            const float *__restrict__ w, int M, float *__restrict__ dy,
                            float *__restrict__ loss) {
  __shared__ double sh[2][32];
  double sw = 0, sl = 0;
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    sw += w[i];
    const double r = 1.0 + y[i] - t[i];
    sl += w[i] * r * r;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sw += __shfl_down_sync(0xffffffffu, sw, o);
    sl += __shfl_down_sync(0xffffffffu, sl, o);
  }
  const int wi = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (l == 0) {
    sh[0][wi] = sw;
    sh[1][wi] = sl;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int k = 0; k < nw; ++k) {
      a += sh[0][k];
      b += sh[1][k];
    }
    sh[0][0] = a;
    sh[1][0] = b;
  }
  __syncthreads();
  const double swt = sh[0][0];
  if (threadIdx.x == 0 && loss) loss[0] = (float)(sh[1][0] / swt);
  for (int i = threadIdx.x; i < M; i += blockDim.x)
    dy[i] = (float)(2.0 * w[i] * (1.0 + y[i] - t[i]) / swt);
}

__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g,
                            float *__restrict__ m, float *__restrict__ v, int n, float lr, float b1,
                            float b2, float eps, float bc1, float bc2) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const float gi = g[e];
    const float mi = b1 * m[e] + (1.f - b1) * gi;
    const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    p[e] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  }
}

// stats[0..4][e] += F, F^L, F^2, (F^L)^2, F F^L with F = BC[x], F^L = -BC[nh + x]
__global__ void cv_stats_kernel(const double *__restrict__ BC, int nh, long long nn,
                                double *__restrict__ stats) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn;
       e += (long long)gridDim.x * blockDim.x) {
    double s0 = 0, s1 = 0, s2 = 0, s3 = 0, s4 = 0;
    for (int x = 0; x < nh; ++x) {
      const double f = BC[(long long)x * nn + e], fl = -BC[(long long)(nh + x) * nn + e];
      s0 += f;
      s1 += fl;
      s2 += f * f;
      s3 += fl * fl;
      s4 += f * fl;
    }
    stats[e] += s0;
    stats[nn + e] += s1;
    stats[2 * nn + e] += s2;
    stats[3 * nn + e] += s3;
    stats[4 * nn + e] += s4;
  }
}

// c* = Cov(F, F^L) / Var(F^L) (1 where Var = 0), weight Var(F^L)
__global__ void cv_targets_kernel(const double *__restrict__ stats, long long nn, int nt, int ns,
                                  float *__restrict__ target, float *__restrict__ weight) {
  const long long total = nn * nt;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long t = e / nn, r = e - t * nn;
    const double *s = stats + t * 5 * nn;
    const double sf = s[r], sl = s[nn + r], sll = s[3 * nn + r], sfl = s[4 * nn + r];
    const double var = (sll - sl * sl / ns) / (ns - 1);
    const double cov = (sfl - sf * sl / ns) / (ns - 1);
    const bool ok = var > 0.0;
    target[e] = ok ? (float)(cov / var) : 1.f;
    weight[e] = ok ? (float)var : 0.f;
  }
}

// per tau: mx[t] = {max |sdd(t)|, max_k |G_kk(t)|, max_k |Gb_kk(t)|}
__global__ void cv_maxima_kernel(const double *__restrict__ sdd, const double *__restrict__ G,
                                 const double *__restrict__ Gb, int n, double *__restrict__ mx) {
  __shared__ double sh[3][32];
  const int t = blockIdx.x;
  const long long nn = (long long)n * n;
  double a = 0, b = 0, c = 0;
  for (long long e = threadIdx.x; e < nn; e += blockDim.x) a = fmax(a, fabs(sdd[t * nn + e]));
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    b = fmax(b, fabs(G[t * nn + (long long)k * n + k]));
    c = fmax(c, fabs(Gb[t * nn + (long long)k * n + k]));
  }
  for (int o = 16; o > 0; o >>= 1) {
    a = fmax(a, __shfl_down_sync(0xffffffffu, a, o));
    b = fmax(b, __shfl_down_sync(0xffffffffu, b, o));
    c = fmax(c, __shfl_down_sync(0xffffffffu, c, o));
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (l == 0) {
    sh[0][w] = a;
    sh[1][w] = b;
    sh[2][w] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < nw; ++k) {
      sh[0][0] = fmax(sh[0][0], sh[0][k]);
      sh[1][0] = fmax(sh[1][0], sh[1][k]);
      sh[2][0] = fmax(sh[2][0], sh[2][k]);
    }
    mx[3 * t] = sh[0][0];
    mx[3 * t + 1] = sh[1][0];
    mx[3 * t + 2] = sh[2][0];
  }
}

// rn[i] = Frobenius norm of row i of [K]^L (sum over its kept pairs and Q)
__global__ void cv_rownorm_kernel(const double *__restrict__ KP, const int *__restrict__ rowptr,
                                  int naux, double *__restrict__ rn) {
  const int i = blockIdx.x;
  double s = 0;
  const long long beg = (long long)rowptr[i] * naux, end = (long long)rowptr[i + 1] * naux;
  for (long long e = beg + threadIdx.x; e < end; e += blockDim.x) s += KP[e] * KP[e];
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) v += sh[k];
    rn[i] = sqrt(v);
  }
}

// out[0] = max x[0..n)
__global__ void max_small_kernel(const double *__restrict__ x, int n, double *__restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double m = 0;
  for (int i = 0; i < n; ++i) m = fmax(m, x[i]);
  out[0] = m;
}

__global__ void cv_features_kernel(const double *__restrict__ sdd, const double *__restrict__ G,
                                   const double *__restrict__ Gb, const double *__restrict__ tau,
                                   double lnbeta, const double *__restrict__ rn,
                                   const double *__restrict__ rmaxp, const double *__restrict__ mx,
                                   int n, int nt, float *__restrict__ X) {
  const double rmax = rmaxp[0];
  const long long nn = (long long)n * n, total = nn * nt;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long t = e / nn, r = e - t * nn;
    const int i = (int)(r / n), j = (int)(r - (long long)i * n);
    const double *g = G + t * nn, *gb = Gb + t * nn;
    const double sm = mx[3 * t], gm = mx[3 * t + 1], gbm = mx[3 * t + 2];
    float *f = X + e * CV_NFEAT;
    f[0] = (float)((double)abs(i - j) / n);
    f[1] = (float)(log(tau[t]) / lnbeta);
    f[2] = sm > 0 ? (float)(sdd[t * nn + r] / sm) : 0.f;
    f[3] = (float)(g[(long long)i * n + i] / gm);
    f[4] = (float)(g[(long long)j * n + j] / gm);
    f[5] = (float)(gb[(long long)i * n + i] / gbm);
    f[6] = (float)(gb[(long long)j * n + j] / gbm);
    f[7] = rmax > 0 ? (float)(rn[i] / rmax) : 0.f;
    f[8] = rmax > 0 ? (float)(rn[j] / rmax) : 0.f;
    f[9] = (i == j) ? 1.f : 0.f;
  }
}

// rows of a [total][cols] array taken at (s * stride + k) mod total, k < m
__global__ void gather_stride_kernel(const float *__restrict__ src, int cols, long long total,
                                     long long start, long long stride, int m,
                                     float *__restrict__ dst) {
  const long long n = (long long)m * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long k = e / cols, c = e - k * cols;
    const long long row = (start + k * stride) % total;
    dst[e] = src[row * cols + c];
  }
}

__global__ void add_one_kernel(const float *__restrict__ y, long long m, double *__restrict__ c) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < m;
       e += (long long)gridDim.x * blockDim.x)
    c[e] = 1.0 + (double)y[e];
}

// sig = (init ? c o base : sig) + sum_x (BC[x] + c o BC[nh + x]) / ns   (BC[nh+x] = -F^L)
__global__ void cv_accumulate_kernel(const double *__restrict__ BC, int nh, long long nn,
                                     double ns, const double *__restrict__ base,
                                     const double *__restrict__ c, int init,
                                     double *__restrict__ sig) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn;
       e += (long long)gridDim.x * blockDim.x) {
    const double ce = c[e];
    double acc = 0.0;
    for (int x = 0; x < nh; ++x)
      acc += BC[(long long)x * nn + e] + ce * BC[(long long)(nh + x) * nn + e];
    sig[e] = (init ? ce * base[e] : sig[e]) + acc / ns;
  }
}

// e_st[x] += -w ((2 t^2 - s2) - Tr((c o F^L) Gb)) / ne, block per pair x
__global__ void cv_pair_energy_kernel(const double *__restrict__ BC, int nh, int n,
                                      const double *__restrict__ c, const double *__restrict__ gb,
                                      const double *__restrict__ t, const double *__restrict__ s2,
                                      double w, double ne, double *__restrict__ e_st) {
  __shared__ double sh[32];
  const int x = blockIdx.x;
  const long long nn = (long long)n * n;
  const double *FL = BC + (long long)(nh + x) * nn;  // -F^L
  double q = 0;
  for (long long e = threadIdx.x; e < nn; e += blockDim.x) {
    const long long i = e / n, j = e - i * n;
    q += c[e] * FL[e] * gb[j * n + i];
  }
  for (int o = 16; o > 0; o >>= 1) q += __shfl_down_sync(0xffffffffu, q, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = q;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) v += sh[k];
    const double de = (2.0 * t[x] * t[x] - s2[x]) + v;
    e_st[x] += -w * de / ne;
  }
}

// out[t] = sum_ij W[t][i][j] X[t][i][j] Y[t][j][i]
__global__ void trace_prod_w_kernel(const double *__restrict__ X, const double *__restrict__ Y,
                                    const double *__restrict__ W, int n, double *__restrict__ out) {
  __shared__ double sh[32];
  const int ti = blockIdx.x;
  const long long nn = (long long)n * n;
  const double *x = X + ti * nn, *y = Y + ti * nn, *w = W + ti * nn;
  double s = 0.0;
  for (long long e = threadIdx.x; e < nn; e += blockDim.x) {
    const long long i = e / n, j = e - i * n;
    s += w[e] * x[e] * y[j * n + i];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) v += sh[k];
    out[ti] = v;
  }
}

}  // namespace

// ------------------------------------------------------------ launchers --
#define RS_L()                  \
  do {                          \
    ++launch_counter();         \
    RS_TRY(cudaGetLastError()); \
  } while (0)

size_t sgemm_work_floats(int M, int N, int K) {
  const long long tiles = (long long)ceil_div(M, 64) * ceil_div(N, 64);
  if (tiles >= 152 || K < 2048) return 0;
  const int ks = (int)std::min<long long>(ceil_div(2 * 152, tiles), K / 512);
  return ks > 1 ? (size_t)ks * M * N : 0;
}

cudaError_t sgemm(int M, int N, int K, const float *A, long long lda, int ta, const float *B,
                  long long ldb, int tb, float *C, long long ldc, float alpha, float beta,
                  float *work, cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const size_t wn = sgemm_work_floats(M, N, K);
  int ks = 1, kc = K;
  if (wn && work && beta == 0.f) {
    ks = (int)(wn / ((size_t)M * N));
    kc = ((ceil_div(K, ks) + 15) / 16) * 16;
    ks = ceil_div(K, kc);
  }
  dim3 grid(ceil_div(N, 64), ceil_div(M, 64), ks);
  const int part = ks > 1;
  float *out = part ? work : C;
#define RS_SG(a, b) sgemm_kernel<a, b><<<grid, 256, 0, s>>>(M, N, K, kc, A, lda, B, ldb, out, ldc, alpha, beta, part)
  if (!ta && !tb) RS_SG(0, 0);
  else if (!ta && tb) RS_SG(0, 1);
  else if (ta && !tb) RS_SG(1, 0);
  else RS_SG(1, 1);
#undef RS_SG
  RS_L();
  if (part) {
    sreduce_kernel<<<grid_cap((long long)M * N, 256), 256, 0, s>>>(work, ks, M, N, C, ldc, alpha);
    RS_L();
  }
  return cudaSuccess;
}

// Parameter layout (floats): W0 [256][10], b0, W1 [256][256], b1, W2, b2, W3 [1][256], b3.
namespace {
constexpr long long O_W0 = 0, O_B0 = O_W0 + CV_HIDDEN * CV_NFEAT, O_W1 = O_B0 + CV_HIDDEN,
                    O_B1 = O_W1 + CV_HIDDEN * CV_HIDDEN, O_W2 = O_B1 + CV_HIDDEN,
                    O_B2 = O_W2 + CV_HIDDEN * CV_HIDDEN, O_W3 = O_B2 + CV_HIDDEN,
                    O_B3 = O_W3 + CV_HIDDEN;
static_assert(O_B3 + 1 == CV_NPARAM, "parameter layout");
}  // namespace

// Split of a contraction over the m rows into g chunks of kc (a multiple of
// 64): the tensor-core weight-gradient products take the chunks as batch
// entries of strided views of one transposed buffer of row stride g kc.
void tc_split(int m, int *g, int *kc) {
  int gg = std::max(1, std::min(8, m / 2048));
  int k = (ceil_div(m, gg) + 63) / 64 * 64;
  *g = gg;
  *kc = k;
}

long long tc_ldt(int m) {
  int g, kc;
  tc_split(m, &g, &kc);
  return (long long)g * kc;
}

// act layout (floats): Z0 A0 Z1 A1 Z2 A2 [m][256] fp32, y [m], dy [m], 2 spare,
// then bf16: H0, H1 [m][256] (bf16 activations / gradient rows), T0, T1
// [256][ldt] (transposes for the weight gradients)
size_t cv_act_floats(int m) {
  // tc_ldt(m) <= m + 8 * 63: sized with m + 512 so that the size grows with m
  return (size_t)m * (6 * CV_HIDDEN + 4) + (size_t)m * CV_HIDDEN +
         (size_t)CV_HIDDEN * ((size_t)m + 512);
}

// work layout (floats): bf16 W1, W2, W1^T, W2^T (4 x 256 x 256), the weight
// gradient partials [8][256][256] fp32, then the fp32 products' split-K scratch
size_t cv_tc_work_floats() {
  return 2LL * CV_HIDDEN * CV_HIDDEN + 8LL * CV_HIDDEN * CV_HIDDEN;
}

namespace {
struct Bf16Bufs {
  __nv_bfloat16 *h0, *h1, *t0, *t1, *w[2], *wt[2];
  float *part;
  float *work;  // fp32 split-K scratch
  long long ldt;
};

Bf16Bufs bf16_bufs(const float *params, float *act, float *work, int m) {
  const int H = CV_HIDDEN;
  Bf16Bufs b;
  float *base = act + (long long)m * (6 * H + 4);
  b.h0 = reinterpret_cast<__nv_bfloat16 *>(base);
  b.h1 = b.h0 + (long long)m * H;
  b.ldt = tc_ldt(m);
  b.t0 = b.h1 + (long long)m * H;
  b.t1 = b.t0 + (long long)H * b.ldt;
  __nv_bfloat16 *wb = reinterpret_cast<__nv_bfloat16 *>(work);
  b.w[0] = wb;
  b.w[1] = wb + H * H;
  b.wt[0] = wb + 2 * H * H;
  b.wt[1] = wb + 3 * H * H;
  b.part = work + 2 * H * H;
  b.work = b.part + 8 * H * H;
  (void)params;
  return b;
}

TcOperand tco(const void *p, long long ld, long long sb, int rows) {
  TcOperand t;
  t.ptr = p;
  t.ld = ld;
  t.sb = sb;
  t.rows = rows;
  return t;
}

// C [M][N] fp32 = A [M][K] B^T, A and B bf16 K-contiguous (tensor cores)
cudaError_t tc_mm(const __nv_bfloat16 *A, long long lda, const __nv_bfloat16 *B, long long ldb,
                  int M, int N, int K, float *C, cudaStream_t s) {
  TcGemm g;
  g.kind = TC_BF16;
  g.M = M;
  g.N = N;
  g.K[0] = K;
  g.A[0] = tco(A, lda, 0, M);
  g.B[0] = tco(B, ldb, 0, N);
  g.c32 = C;
  return tc_gemm(g, s);
}

// dW [N][M]... : out[o][i] = sum_r At[o][r] Bt[i][r] over r < m, split into g
// chunks (batch entries of strided views), partials reduced in order
cudaError_t tc_wgrad(const __nv_bfloat16 *At, const __nv_bfloat16 *Bt, long long ldt, int m,
                     float *part, float *out, cudaStream_t s) {
  const int H = CV_HIDDEN;
  int g, kc;
  tc_split(m, &g, &kc);
  TcGemm t;
  t.kind = TC_BF16;
  t.M = H;
  t.N = H;
  t.batch = g;
  t.bpc = 1;
  t.K[0] = kc;
  t.A[0] = tco(At, ldt, kc, H);
  t.B[0] = tco(Bt, ldt, kc, H);
  t.c32 = part;
  RS_TRY(tc_gemm(t, s));
  sreduce_kernel<<<grid_cap((long long)H * H, 256), 256, 0, s>>>(part, g, H, H, out, H, 1.f);
  ++launch_counter();
  return cudaGetLastError();
}

cudaError_t to_bf16(const float *src, long long n, __nv_bfloat16 *dst, cudaStream_t s) {
  to_bf16_kernel<<<grid_cap(n, 256), 256, 0, s>>>(src, n, dst);
  ++launch_counter();
  return cudaGetLastError();
}

// dst [cols][ldd] = bf16 src[rows][cols]^T (zero beyond rows)
cudaError_t transpose_bf16(const float *src, int rows, int cols, long long lds,
                           __nv_bfloat16 *dst, long long ldd, cudaStream_t s) {
  dim3 grid((unsigned)((ldd + 31) / 32), (unsigned)ceil_div(cols, 32));
  transpose_bf16_kernel<<<grid, 256, 0, s>>>(src, rows, cols, lds, dst, ldd);
  ++launch_counter();
  return cudaGetLastError();
}
}  // namespace

cudaError_t cv_forward(const float *params, const float *X, int m, float *act, float *work,
                       cudaStream_t s) {
  const int H = CV_HIDDEN;
  float *Z0 = act, *A0 = Z0 + (long long)m * H, *Z1 = A0 + (long long)m * H,
        *A1 = Z1 + (long long)m * H, *Z2 = A1 + (long long)m * H, *A2 = Z2 + (long long)m * H,
        *y = A2 + (long long)m * H;
  Bf16Bufs b = bf16_bufs(params, act, work, m);
  // bf16 copies of the hidden weights W1, W2 (the B operands: rows = outputs)
  RS_TRY(to_bf16(params + O_W1, (long long)H * H, b.w[0], s));
  RS_TRY(to_bf16(params + O_W2, (long long)H * H, b.w[1], s));
  // layer 0 (10 inputs): fp32
  RS_TRY(sgemm(m, H, CV_NFEAT, X, CV_NFEAT, 0, params + O_W0, CV_NFEAT, 1, Z0, H, 1.f, 0.f,
               b.work, s));
  bias_silu_kernel<<<grid_cap((long long)m * H, 256), 256, 0, s>>>(Z0, params + O_B0, m, H, A0);
  RS_L();
  // layers 1, 2: tensor cores on bf16 activations
  RS_TRY(to_bf16(A0, (long long)m * H, b.h0, s));
  RS_TRY(tc_mm(b.h0, H, b.w[0], H, m, H, H, Z1, s));
  bias_silu_kernel<<<grid_cap((long long)m * H, 256), 256, 0, s>>>(Z1, params + O_B1, m, H, A1);
  RS_L();
  RS_TRY(to_bf16(A1, (long long)m * H, b.h1, s));
  RS_TRY(tc_mm(b.h1, H, b.w[1], H, m, H, H, Z2, s));
  bias_silu_kernel<<<grid_cap((long long)m * H, 256), 256, 0, s>>>(Z2, params + O_B2, m, H, A2);
  RS_L();
  // output layer (1 output): fp32
  RS_TRY(sgemm(m, 1, H, A2, H, 0, params + O_W3, H, 1, y, 1, 1.f, 0.f, b.work, s));
  bias_silu_kernel<<<grid_cap(m, 256), 256, 0, s>>>(y, params + O_B3, m, 1, nullptr);
  RS_L();
  return cudaSuccess;
}

cudaError_t cv_backward(const float *params, const float *X, int m, const float *target,
                        const float *weight, float *act, float *grad, float *loss, float *work,
                        cudaStream_t s) {
  const int H = CV_HIDDEN;
  float *Z0 = act, *A0 = Z0 + (long long)m * H, *Z1 = A0 + (long long)m * H,
        *A1 = Z1 + (long long)m * H, *Z2 = A1 + (long long)m * H, *A2 = Z2 + (long long)m * H,
        *y = A2 + (long long)m * H, *dy = y + m;
  Bf16Bufs b = bf16_bufs(params, act, work, m);
  // bf16 W1^T, W2^T (the B operands of dA = dZ W: rows = inputs)
  RS_TRY(transpose_bf16(params + O_W1, H, H, H, b.wt[0], H, s));
  RS_TRY(transpose_bf16(params + O_W2, H, H, H, b.wt[1], H, s));
  loss_kernel<<<1, 1024, 0, s>>>(y, target, weight, m, dy, loss);
  RS_L();
  // layer 3: dW3 = dy^T A2, db3 = sum dy, dA2 = dy W3 (fp32)
  RS_TRY(sgemm(1, H, m, dy, 1, 1, A2, H, 0, grad + O_W3, H, 1.f, 0.f, b.work, s));
  colsum_kernel<<<1, 32, 0, s>>>(dy, m, 1, grad + O_B3);
  RS_L();
  RS_TRY(sgemm(m, H, 1, dy, 1, 0, params + O_W3, H, 0, A2, H, 1.f, 0.f, b.work, s));
  silu_back_kernel<<<grid_cap((long long)m * H, 256), 256, 0, s>>>(A2, Z2, (long long)m * H, Z2);
  RS_L();  // Z2 now holds dZ2
  // layer 2: dW2 = dZ2^T A1, db2; dA1 = dZ2 W2; dZ1 = dA1 silu'(Z1)
  RS_TRY(transpose_bf16(Z2, m, H, H, b.t0, b.ldt, s));
  RS_TRY(transpose_bf16(A1, m, H, H, b.t1, b.ldt, s));
  RS_TRY(tc_wgrad(b.t0, b.t1, b.ldt, m, b.part, grad + O_W2, s));
  colsum_kernel<<<ceil_div(H, 128), 128, 0, s>>>(Z2, m, H, grad + O_B2);
  RS_L();
  RS_TRY(to_bf16(Z2, (long long)m * H, b.h1, s));
  RS_TRY(tc_mm(b.h1, H, b.wt[1], H, m, H, H, A1, s));
  silu_back_kernel<<<grid_cap((long long)m * H, 256), 256, 0, s>>>(A1, Z1, (long long)m * H, Z1);
  RS_L();  // Z1 now holds dZ1
  // layer 1: dW1 = dZ1^T A0, db1; dA0 = dZ1 W1; dZ0 = dA0 silu'(Z0)
  RS_TRY(transpose_bf16(Z1, m, H, H, b.t0, b.ldt, s));
  RS_TRY(transpose_bf16(A0, m, H, H, b.t1, b.ldt, s));
  RS_TRY(tc_wgrad(b.t0, b.t1, b.ldt, m, b.part, grad + O_W1, s));
  colsum_kernel<<<ceil_div(H, 128), 128, 0, s>>>(Z1, m, H, grad + O_B1);
  RS_L();
  RS_TRY(to_bf16(Z1, (long long)m * H, b.h0, s));
  RS_TRY(tc_mm(b.h0, H, b.wt[0], H, m, H, H, A0, s));
  silu_back_kernel<<<grid_cap((long long)m * H, 256), 256, 0, s>>>(A0, Z0, (long long)m * H, Z0);
  RS_L();  // Z0 now holds dZ0
  // layer 0 (10 inputs): dW0 = dZ0^T X, db0 (fp32)
  RS_TRY(sgemm(H, CV_NFEAT, m, Z0, H, 1, X, CV_NFEAT, 0, grad + O_W0, CV_NFEAT, 1.f, 0.f, b.work,
               s));
  colsum_kernel<<<ceil_div(H, 128), 128, 0, s>>>(Z0, m, H, grad + O_B0);
  RS_L();
  return cudaSuccess;
}

cudaError_t cv_adam(float *p, const float *g, float *m, float *v, int n, float lr, int step,
                    cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float bc1 = 1.f - powf(b1, (float)step), bc2 = 1.f - powf(b2, (float)step);
  adam_kernel<<<grid_cap(n, 256), 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, 1e-8f, bc1, bc2);
  RS_L();
  return cudaSuccess;
}

cudaError_t cv_stats(const double *BC, int nh, int n, double *stats, cudaStream_t s) {
  const long long nn = (long long)n * n;
  cv_stats_kernel<<<grid_cap(nn, 256), 256, 0, s>>>(BC, nh, nn, stats);
  RS_L();
  return cudaSuccess;
}

cudaError_t cv_targets(const double *stats, int n, int nt, int ns, float *target, float *weight,
                       cudaStream_t s) {
  const long long nn = (long long)n * n;
  cv_targets_kernel<<<grid_cap(nn * nt, 256), 256, 0, s>>>(stats, nn, nt, ns, target, weight);
  RS_L();
  return cudaSuccess;
}

cudaError_t cv_features(const double *sdd, const double *G, const double *Gb, const double *tau,
                        double beta, const double *KP, const int *rowptr, int naux, int n, int nt,
                        double *scratch, float *X, cudaStream_t s) {
  double *mx = scratch, *rn = scratch + 3 * nt;
  cv_maxima_kernel<<<nt, 256, 0, s>>>(sdd, G, Gb, n, mx);
  RS_L();
  cv_rownorm_kernel<<<n, 256, 0, s>>>(KP, rowptr, naux, rn);
  RS_L();
  max_small_kernel<<<1, 32, 0, s>>>(rn, n, rn + n);
  RS_L();
  cv_features_kernel<<<grid_cap((long long)n * n * nt, 256), 256, 0, s>>>(
      sdd, G, Gb, tau, log(beta), rn, rn + n, mx, n, nt, X);
  RS_L();
  return cudaSuccess;
}

cudaError_t cv_gather(const float *src, int cols, long long total, long long start,
                      long long stride, int m, float *dst, cudaStream_t s) {
  gather_stride_kernel<<<grid_cap((long long)m * cols, 256), 256, 0, s>>>(src, cols, total, start,
                                                                          stride, m, dst);
  RS_L();
  return cudaSuccess;
}

cudaError_t cv_accumulate(const double *BC, int nh, int n, double ns, const double *base,
                          const double *c, int init, double *sig, cudaStream_t s) {
  const long long nn = (long long)n * n;
  cv_accumulate_kernel<<<grid_cap(nn, 256), 256, 0, s>>>(BC, nh, nn, ns, base, c, init, sig);
  RS_L();
  return cudaSuccess;
}

cudaError_t cv_pair_energy(const double *BC, int nh, int n, const double *c, const double *gb,
                           const double *t, const double *s2, double w, double ne, double *e_st,
                           cudaStream_t s) {
  cv_pair_energy_kernel<<<nh, 256, 0, s>>>(BC, nh, n, c, gb, t, s2, w, ne, e_st);
  RS_L();
  return cudaSuccess;
}

cudaError_t trace_prod_w(const double *X, const double *Y, const double *W, int n, int nt,
                         double *out, cudaStream_t s) {
  trace_prod_w_kernel<<<nt, 256, 0, s>>>(X, Y, W, n, out);
  RS_L();
  return cudaSuccess;
}

cudaError_t cv_coefficients(const float *y, long long m, double *c, cudaStream_t s) {
  add_one_kernel<<<grid_cap(m, 256), 256, 0, s>>>(y, m, c);
  RS_L();
  return cudaSuccess;
}

}  // namespace rssri
