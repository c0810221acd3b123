// Element-wise kernels of the reduced-precision chain (S8 on the tensor cores
// with bf16 or tf32 operands), in the range-separated split of Eqs. 14-15:
// with R = R^L + R^S,
//   C^L = R^L G R'^L,  dC = R^S G R' + R^L G R'^S,  C = C^L + dC,
//   X = dC Gb,  Y = C^L Gb,  dt = Tr X,  t^L = Tr Y,
//   F(R,R') - F(R^L,R'^L) = (2 dt I - X) C + (2 t^L I - Y) dC,
//   Tr[(F - F^L) Gb] = 2 dt (2 t^L + dt) - Tr(X X) - 2 Tr(X Y).
// Only the small R^S terms ever appear on their own, so the rounding of every
// operand (2^-8 relative for bf16, 2^-11 for tf32) costs an error of that
// order of the stochastic remainder, not of the full self-energy.  Traces and
// energies are summed in fp64.
#include <cuda_bf16.h>

#include "chain_tc.cuh"
#include "tc_gemm.cuh"

namespace rssri {
namespace {

// Operand storage: bf16, or fp32 holding a value rounded to tf32.
__device__ __forceinline__ void put(__nv_bfloat16 *p, double v) { *p = __double2bfloat16(v); }
__device__ __forceinline__ void put(float *p, double v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(__double2float_rn(v)));
  *p = __uint_as_float(r);
}
// From fp32 (the fold's operands: fp32 products rounded once more to the
// operand type; no fp64 instruction on the way)
__device__ __forceinline__ void putf(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void putf(float *p, float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  *p = __uint_as_float(r);
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ double block_sum_d(double v) {
  __shared__ double sh[32];
  __syncthreads();
  v = warp_sum_d(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    double x = (l < nw) ? sh[l] : 0.0;
    x = warp_sum_d(x);
    if (l == 0) sh[0] = x;
  }
  __syncthreads();
  return sh[0];
}

int grid_cap(long long work, int threads) {
  long long b = (work + threads - 1) / threads;
  return (int)(b < 1 ? 1 : (b > 152 * 32 ? 152 * 32 : b));
}

// fac = [set][kind][x][n][n] fp64 (kind 0: R, kind 1: R^L)
template <class T>
__global__ void factors_kernel(const double *__restrict__ fac, int ns, int n, int ldp,
                               T *__restrict__ xsl, T *__restrict__ y3) {
  const long long nn = (long long)n * n, mat = (long long)n * ldp;
  const long long total = (long long)ns * n * ldp;
  const double *r0 = fac, *rl0 = fac + ns * nn, *r1 = fac + 2 * ns * nn, *rl1 = fac + 3 * ns * nn;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long x = e / mat, r = e - x * mat;
    const int i = (int)(r / ldp), j = (int)(r - (long long)i * ldp);
    double a = 0, al = 0, b = 0, bl = 0;
    if (j < n) {
      const long long src = x * nn + (long long)i * n + j;
      a = r0[src];
      al = rl0[src];
      b = r1[src];
      bl = rl1[src];
    }
    put(&xsl[e], a - al);            // R^S
    put(&xsl[ns * mat + e], al);     // R^L
    put(&y3[e], b);                  // R'
    put(&y3[ns * mat + e], b - bl);  // R'^S
    put(&y3[2 * ns * mat + e], bl);  // R'^L
  }
}

template <class T>
__global__ void matrices_kernel(const double *__restrict__ src, int cnt, int n, int ldp,
                                T *__restrict__ dst) {
  const long long mat = (long long)n * ldp, total = (long long)cnt * mat;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long x = e / mat, r = e - x * mat;
    const int i = (int)(r / ldp), j = (int)(r - (long long)i * ldp);
    put(&dst[e], j < n ? src[x * n * n + (long long)i * n + j] : 0.0);
  }
}

// The fold works on 32 x 32 tiles staged in shared memory, so that every
// global read and write is coalesced (including the transposes), in two
// passes over a grid of (tile row, sample pair) blocks of 256 threads:
//  1. partial sums of Tr X, Tr Y, Tr(X X) = sum X_ij X_ji, Tr(X Y) = sum Y_ij X_ji
//     per tile row;
//  2. the operands 2 dt I - X, 2 t^L I - Y, (C^L + dC)^T and dC^T of that tile
//     row, after summing the partials of pass 1 in a fixed order; the block of
//     tile row 0 adds the pair energy.
__global__ void __launch_bounds__(256) fold_traces_kernel(const float *__restrict__ xy, int ns,
                                                          int n, double *__restrict__ part) {
  __shared__ float ta[32][33], tb[32][33], tc[32][33];
  const int bi = blockIdx.x, x = blockIdx.y, nt = gridDim.x;
  const long long nn = (long long)n * n;
  const float *X = xy + x * nn, *Y = xy + (ns + x) * nn;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  double dx = 0, dy = 0;
  float sxx = 0.f, sxy = 0.f;  // per thread: 4 rows x the tile columns (fp32)
  if (ty == 0) {
    const int i = bi * 32 + tx;
    if (i < n) {
      dx = X[(long long)i * n + i];
      dy = Y[(long long)i * n + i];
    }
  }
  for (int bj = 0; bj < nt; ++bj) {
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
      const int i = bi * 32 + r, j = bj * 32 + tx;
      const int i2 = bj * 32 + r, j2 = bi * 32 + tx;
      const bool in1 = i < n && j < n, in2 = i2 < n && j2 < n;
      ta[r][tx] = in1 ? X[(long long)i * n + j] : 0.f;
      tc[r][tx] = in1 ? Y[(long long)i * n + j] : 0.f;
      tb[r][tx] = in2 ? X[(long long)i2 * n + j2] : 0.f;  // block (bj, bi) of X
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
      const float xt = tb[tx][r];  // X_ji, i = bi*32 + r, j = bj*32 + tx
      sxx = fmaf(ta[r][tx], xt, sxx);
      sxy = fmaf(tc[r][tx], xt, sxy);
    }
  }
  const double v0 = block_sum_d(dx), v1 = block_sum_d(dy), v2 = block_sum_d((double)sxx),
               v3 = block_sum_d((double)sxy);
  if (threadIdx.x == 0) {
    double *o = part + ((long long)x * nt + bi) * 4;
    o[0] = v0;
    o[1] = v1;
    o[2] = v2;
    o[3] = v3;
  }
}

// One 32 x 32 tile (bi, bj) of pair x per block: every load of the tile is
// issued before the first store; the transposes go through shared memory.
template <class T>
__global__ void __launch_bounds__(256) fold_operands_kernel(
    const float *__restrict__ xy, const float *__restrict__ dc, const float *__restrict__ cl, int ns,
    int n, int ldp, int nt, const double *__restrict__ part, double w, double ne,
    T *__restrict__ a6, T *__restrict__ ct, T *__restrict__ dct, T *__restrict__ clt,
    double *__restrict__ e_st) {
  __shared__ float ta[32][33], tb[32][33], tl32[32][33];
  __shared__ double sums[4];
  const int bj = blockIdx.x, bi = blockIdx.y, x = blockIdx.z;
  const long long nn = (long long)n * n, mat = (long long)n * ldp;
  if (threadIdx.x < 4) {
    double v = 0;
    for (int t = 0; t < nt; ++t) v += part[((long long)x * nt + t) * 4 + threadIdx.x];
    sums[threadIdx.x] = v;
  }
  const float *X = xy + x * nn, *Y = xy + (ns + x) * nn;
  const float *DC = dc + x * nn, *CL = cl + x * nn;
  T *A = a6 + x * mat, *Ab = a6 + (ns + x) * mat;
  T *Ct = ct + x * mat, *Dt = dct + x * mat;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  // loads: rows ty, ty + 8, ... of the tile of X and Y, and of the
  // transposed-source tile (bj, bi) of C^L and dC
  float xv[4], yv[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int r = ty + 8 * u;
    const int i = bi * 32 + r, j = bj * 32 + tx;
    const bool in = i < n && j < n;
    xv[u] = in ? X[(long long)i * n + j] : 0.f;
    yv[u] = in ? Y[(long long)i * n + j] : 0.f;
    const int i2 = bj * 32 + r, j2 = bi * 32 + tx;  // source (i2, j2) of C and dC
    const bool in2 = i2 < n && j2 < n;
    const float c = in2 ? CL[(long long)i2 * n + j2] : 0.f;
    const float d = in2 ? DC[(long long)i2 * n + j2] : 0.f;
    ta[r][tx] = c + d;
    tb[r][tx] = d;
    tl32[r][tx] = c;
  }
  __syncthreads();
  const double dt = sums[0], tl = sums[1];
  const float dt2 = (float)(2.0 * dt), tl2 = (float)(2.0 * tl);
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int r = ty + 8 * u;
    const int i = bi * 32 + r, j = bj * 32 + tx;  // destination (i, j) = source (j, i)
    if (i < n && j < ldp) {
      const long long o = (long long)i * ldp + j;
      const bool in = j < n;
      putf(&A[o], in ? (i == j ? dt2 : 0.f) - xv[u] : 0.f);
      putf(&Ab[o], in ? (i == j ? tl2 : 0.f) - yv[u] : 0.f);
      putf(&Ct[o], in ? ta[tx][r] : 0.f);
      putf(&Dt[o], in ? tb[tx][r] : 0.f);
      if (clt) putf(&clt[x * mat + o], in ? tl32[tx][r] : 0.f);
    }
  }
  if (bi == 0 && bj == 0 && threadIdx.x == 0) {
    const double de = 2.0 * dt * (2.0 * tl + dt) - sums[2] - 2.0 * sums[3];
    e_st[x] += -w * de / ne;
  }
}

// sig[e] += (1 - c[e]) (mean_x fl[x][e] - sdd[e])
__global__ void cv_tc_sigma_kernel(const float *__restrict__ fl, int ns, long long nn,
                                   const double *__restrict__ c, const double *__restrict__ sdd,
                                   double *__restrict__ sig) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn;
       e += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int x = 0; x < ns; ++x) acc += (double)fl[(long long)x * nn + e];
    sig[e] += (1.0 - c[e]) * (acc / ns - sdd[e]);
  }
}

// e_st[x] += -(w / ne) sum_ij (1 - c_ij) fl[x]_ij gb_ji, one block per pair
__global__ void __launch_bounds__(256) cv_tc_energy_kernel(const float *__restrict__ fl, int n,
                                                           const double *__restrict__ c,
                                                           const double *__restrict__ gb,
                                                           double w, double ne,
                                                           double *__restrict__ e_st) {
  const int x = blockIdx.x;
  const long long nn = (long long)n * n;
  const float *F = fl + x * nn;
  double q = 0.0;
  for (long long e = threadIdx.x; e < nn; e += blockDim.x) {
    const long long i = e / n, j = e - i * n;
    q += (1.0 - c[e]) * (double)F[e] * gb[j * n + i];
  }
  q = block_sum_d(q);
  if (threadIdx.x == 0) e_st[x] += -w * q / ne;
}

__global__ void reduce_tc_kernel(const float *__restrict__ part, int groups, long long nn,
                                   const double *__restrict__ base, double ns,
                                   double *__restrict__ sig) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn;
       e += (long long)gridDim.x * blockDim.x) {
    // four independent partial sums (loads in flight), added in a fixed order
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    int g = 0;
    for (; g + 4 <= groups; g += 4) {
      a0 += part[(long long)g * nn + e];
      a1 += part[(long long)(g + 1) * nn + e];
      a2 += part[(long long)(g + 2) * nn + e];
      a3 += part[(long long)(g + 3) * nn + e];
    }
    for (; g < groups; ++g) a0 += part[(long long)g * nn + e];
    const double acc = ((double)a0 + (double)a1) + ((double)a2 + (double)a3);
    sig[e] = base[e] + acc / ns;
  }
}

}  // namespace

cudaError_t chain_factors(int kind, const double *fac, int ns, int n, int ldp, void *xsl,
                          void *y3, cudaStream_t s) {
  const int grid = grid_cap((long long)ns * n * ldp, 256);
  if (kind == TC_BF16)
    factors_kernel<<<grid, 256, 0, s>>>(fac, ns, n, ldp, static_cast<__nv_bfloat16 *>(xsl),
                                        static_cast<__nv_bfloat16 *>(y3));
  else
    factors_kernel<<<grid, 256, 0, s>>>(fac, ns, n, ldp, static_cast<float *>(xsl),
                                        static_cast<float *>(y3));
  ++launch_counter();
  return cudaGetLastError();
}

cudaError_t chain_matrices(int kind, const double *src, int cnt, int n, int ldp, void *dst,
                           cudaStream_t s) {
  const int grid = grid_cap((long long)cnt * n * ldp, 256);
  if (kind == TC_BF16)
    matrices_kernel<<<grid, 256, 0, s>>>(src, cnt, n, ldp, static_cast<__nv_bfloat16 *>(dst));
  else
    matrices_kernel<<<grid, 256, 0, s>>>(src, cnt, n, ldp, static_cast<float *>(dst));
  ++launch_counter();
  return cudaGetLastError();
}

cudaError_t fold_tc(int kind, const float *xy, const float *dc, const float *cl, int ns, int n,
                    int ldp, double w, double ne, void *a6, void *ct, void *dct, void *clt,
                    double *e_st, double *part, cudaStream_t s) {
  const int nt = (n + 31) / 32;
  dim3 grid(nt, ns);
  fold_traces_kernel<<<grid, 256, 0, s>>>(xy, ns, n, part);
  ++launch_counter();
  RS_TRY(cudaGetLastError());
  if (ns > 65535) return cudaErrorInvalidValue;
  dim3 go((ldp + 31) / 32, nt, ns);
  if (kind == TC_BF16)
    fold_operands_kernel<<<go, 256, 0, s>>>(xy, dc, cl, ns, n, ldp, nt, part, w, ne,
                                              static_cast<__nv_bfloat16 *>(a6),
                                              static_cast<__nv_bfloat16 *>(ct),
                                              static_cast<__nv_bfloat16 *>(dct),
                                              static_cast<__nv_bfloat16 *>(clt), e_st);
  else
    fold_operands_kernel<<<go, 256, 0, s>>>(xy, dc, cl, ns, n, ldp, nt, part, w, ne,
                                              static_cast<float *>(a6), static_cast<float *>(ct),
                                              static_cast<float *>(dct),
                                              static_cast<float *>(clt), e_st);
  ++launch_counter();
  return cudaGetLastError();
}

cudaError_t cv_tc_apply(const float *fl, int ns, int n, const double *c, const double *sdd,
                        const double *gb, double w, double ne, double *sig, double *e_st,
                        cudaStream_t s) {
  const long long nn = (long long)n * n;
  cv_tc_sigma_kernel<<<grid_cap(nn, 256), 256, 0, s>>>(fl, ns, nn, c, sdd, sig);
  ++launch_counter();
  RS_TRY(cudaGetLastError());
  cv_tc_energy_kernel<<<ns, 256, 0, s>>>(fl, n, c, gb, w, ne, e_st);
  ++launch_counter();
  return cudaGetLastError();
}

cudaError_t reduce_tc(const float *part, int groups, int n, const double *base, double ns,
                      double *sig, cudaStream_t s) {
  const long long nn = (long long)n * n;
  reduce_tc_kernel<<<grid_cap(nn, 256), 256, 0, s>>>(part, groups, nn, base, ns, sig);
  ++launch_counter();
  return cudaGetLastError();
}

}  // namespace rssri
