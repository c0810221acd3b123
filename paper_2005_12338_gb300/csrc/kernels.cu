// Non-GEMM kernels of the RS-SRI-GF2 path.  Every reduction has a fixed
// order (per-thread strided partials, then a fixed shuffle/shared-memory
// tree), so the library is bitwise reproducible; maxima and integer counts
// are exact regardless of order.
#include <algorithm>

#include "kernels.cuh"

namespace rssri {
namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(FULL, v, o));
  return v;
}
__device__ __forceinline__ long long warp_suml(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
  return v;
}

// Block-wide sum / max; the result is returned to every thread.  blockDim.x
// must be a multiple of 32 and at most 1024.
__device__ double block_sum(double v) {
  __shared__ double sh[32];
  __syncthreads();
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    double x = (l < nw) ? sh[l] : 0.0;
    x = warp_sum(x);
    if (l == 0) sh[0] = x;
  }
  __syncthreads();
  return sh[0];
}
__device__ double block_max(double v) {
  __shared__ double sh[32];
  __syncthreads();
  v = warp_max(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    double x = (l < nw) ? sh[l] : 0.0;
    x = warp_max(x);
    if (l == 0) sh[0] = x;
  }
  __syncthreads();
  return sh[0];
}
__device__ long long block_suml(long long v) {
  __shared__ long long sh[32];
  __syncthreads();
  v = warp_suml(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    long long x = (l < nw) ? sh[l] : 0;
    x = warp_suml(x);
    if (l == 0) sh[0] = x;
  }
  __syncthreads();
  return sh[0];
}

int grid_for(long long work, int threads, int cap = 152 * 32) {
  long long b = (work + threads - 1) / threads;
  return (int)std::max<long long>(1, std::min<long long>(b, cap));
}

// ------------------------------------------------------------------ S1 ----
__global__ void rowsum_abs_kernel(const double *__restrict__ V, int na, double *__restrict__ out) {
  const int i = blockIdx.x;
  double s = 0.0;
  for (int j = threadIdx.x; j < na; j += blockDim.x) s += fabs(V[(long long)i * na + j]);
  s = block_sum(s);
  if (threadIdx.x == 0) out[i] = s;
}

__global__ void absmax_partial_kernel(const double *__restrict__ x, long long len,
                                      double *__restrict__ part) {
  double m = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len;
       e += (long long)gridDim.x * blockDim.x)
    m = fmax(m, fabs(x[e]));
  m = block_max(m);
  if (threadIdx.x == 0) part[blockIdx.x] = m;
}

__global__ void max_final_kernel(const double *__restrict__ part, int np, double *__restrict__ out) {
  double m = 0.0;
  for (int e = threadIdx.x; e < np; e += blockDim.x) m = fmax(m, part[e]);
  m = block_max(m);
  if (threadIdx.x == 0) out[0] = m;
}

__global__ void ns_init_kernel(const double *__restrict__ V, int na, const double *__restrict__ scal,
                               double *__restrict__ Y, double *__restrict__ Z) {
  const double c = scal[0];
  const long long nn = (long long)na * na;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / na, j = e - i * na;
    Y[e] = V[e] / c;
    Z[e] = (i == j) ? 1.0 : 0.0;
  }
}

__global__ void ns_tbuild_kernel(const double *__restrict__ P, int na, double *__restrict__ T,
                                 double *__restrict__ part) {
  const long long nn = (long long)na * na;
  double m = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / na, j = e - i * na;
    const double d = (i == j) ? 1.0 : 0.0;
    const double p = P[e];
    T[e] = 0.5 * (3.0 * d - p);
    m = fmax(m, fabs(p - d));
  }
  m = block_max(m);
  if (threadIdx.x == 0) part[blockIdx.x] = m;
}

__global__ void ns_finish_kernel(const double *__restrict__ Z, int na, const double *__restrict__ scal,
                                 double *__restrict__ W) {
  const double r = 1.0 / sqrt(scal[0]);
  const long long nn = (long long)na * na;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / na, j = e - i * na;
    W[e] = 0.5 * (Z[e] + Z[j * na + i]) * r;
  }
}

// ------------------------------------------------------------------ S2 ----
__global__ void eri_check_kernel(const double *__restrict__ eri3, int n, int naux,
                                 int *__restrict__ flags) {
  const long long total = (long long)n * n * naux;
  int bad_sym = 0, bad_fin = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const double x = eri3[e];
    if (!isfinite(x)) bad_fin = 1;
    const long long p = e / naux;
    const int a = (int)(e - p * naux);
    const int i = (int)(p / n), j = (int)(p - (long long)i * n);
    if (i < j && x != eri3[((long long)j * n + i) * naux + a]) bad_sym = 1;
  }
  if (__any_sync(FULL, bad_sym) && (threadIdx.x & 31) == 0) atomicOr(&flags[0], 1);
  if (__any_sync(FULL, bad_fin) && (threadIdx.x & 31) == 0) atomicOr(&flags[1], 1);
}

__global__ void eri_colmax_kernel(const double *__restrict__ eri3, int n, int naux,
                                  double *__restrict__ colmax) {
  const int j = blockIdx.x;
  const long long len = (long long)n * naux;
  const double *row = eri3 + (long long)j * len;
  double m = 0.0;
  for (long long e = threadIdx.x; e < len; e += blockDim.x) m = fmax(m, fabs(row[e]));
  m = block_max(m);
  if (threadIdx.x == 0) colmax[j] = m;
}

__device__ __forceinline__ double screen_threshold(double eps_prime, int n, double mi, double mj) {
  // Eq. 11, applied with the smaller of the two orbital-index maxima.
  return (eps_prime / (double)n) * fmin(mi, mj);
}

__global__ void eri_pair_count_kernel(const double *__restrict__ eri3, int n, int naux,
                                      const double *__restrict__ colmax, double eps_prime,
                                      int *__restrict__ cnt) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long pair = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
  if (pair >= (long long)n * n) return;
  const int i = (int)(pair / n), j = (int)(pair - (long long)i * n);
  const double thr = screen_threshold(eps_prime, n, colmax[i], colmax[j]);
  const double *row = eri3 + pair * naux;
  int c = 0;
  for (int a = lane; a < naux; a += 32) c += (fabs(row[a]) >= thr) ? 1 : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(FULL, c, o);
  if (lane == 0) cnt[pair] = c;
}

__global__ void eri_gather_rows_kernel(const double *__restrict__ eri3, int n, int naux,
                                       const double *__restrict__ colmax, double eps_prime,
                                       const int *__restrict__ pairs, double *__restrict__ out) {
  const int p = blockIdx.x;
  const int pair = pairs[p];
  const int i = pair / n, j = pair - i * n;
  const double thr = screen_threshold(eps_prime, n, colmax[i], colmax[j]);
  const double *row = eri3 + (long long)pair * naux;
  double *o = out + (long long)p * naux;
  for (int a = threadIdx.x; a < naux; a += blockDim.x) {
    const double x = row[a];
    o[a] = (fabs(x) >= thr) ? x : 0.0;
  }
}

// -------------------------------------------------------------- compact ---
constexpr int CT = 256, CPT = 4, CB = CT * CPT;

__global__ void compact_count_kernel(const int *__restrict__ cnt, int len, int *__restrict__ bcount,
                                     long long *__restrict__ bsum) {
  const int base = blockIdx.x * CB + threadIdx.x * CPT;
  int c = 0;
  long long s = 0;
#pragma unroll
  for (int r = 0; r < CPT; ++r) {
    const int e = base + r;
    if (e < len) {
      const int v = cnt[e];
      c += v > 0;
      s += v;
    }
  }
  const double cd = block_sum((double)c);  // exact: small integers
  const long long sl = block_suml(s);
  if (threadIdx.x == 0) {
    bcount[blockIdx.x] = (int)cd;
    bsum[blockIdx.x] = sl;
  }
}

__global__ void compact_scan_kernel(const int *__restrict__ bcount, const long long *__restrict__ bsum,
                                    int nb, int *__restrict__ boff, int *__restrict__ count,
                                    long long *__restrict__ sum64) {
  // one block of 1024 threads; chunks of 1024 block counts with a carry
  __shared__ int wsum[32];
  __shared__ int carry;
  __shared__ long long lcarry;
  if (threadIdx.x == 0) { carry = 0; lcarry = 0; }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c0 = 0; c0 < nb; c0 += 1024) {
    const int e = c0 + threadIdx.x;
    const int v = (e < nb) ? bcount[e] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(FULL, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int w = wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, w, o);
        if (lane >= o) w += y;
      }
      wsum[lane] = w;
    }
    __syncthreads();
    const int excl = x - v + (warp > 0 ? wsum[warp - 1] : 0);
    if (e < nb) boff[e] = carry + excl;
    const long long ls = block_suml((e < nb) ? bsum[e] : 0);
    __syncthreads();
    if (threadIdx.x == 0) {
      carry += wsum[31];
      lcarry += ls;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    count[0] = carry;
    sum64[0] = lcarry;
  }
}

__global__ void compact_write_kernel(const int *__restrict__ cnt, int len, const int *__restrict__ boff,
                                     int *__restrict__ idx) {
  __shared__ int wsum[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int base = blockIdx.x * CB + threadIdx.x * CPT;
  int f[CPT];
  int c = 0;
#pragma unroll
  for (int r = 0; r < CPT; ++r) {
    const int e = base + r;
    f[r] = (e < len && cnt[e] > 0) ? 1 : 0;
    c += f[r];
  }
  int x = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = (lane < (CT >> 5)) ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(FULL, w, o);
      if (lane >= o) w += y;
    }
    if (lane < (CT >> 5)) wsum[lane] = w;
  }
  __syncthreads();
  int pos = boff[blockIdx.x] + x - c + (warp > 0 ? wsum[warp - 1] : 0);
#pragma unroll
  for (int r = 0; r < CPT; ++r)
    if (f[r]) idx[pos++] = base + r;
}

// ------------------------------------------------------------------ S3 ----
__global__ void kl_cut_kernel(double *__restrict__ rows, int naux, const double *__restrict__ kmax,
                              double eps, int *__restrict__ cnt) {
  const int p = blockIdx.x;
  const double thr = eps * kmax[0];  // Eq. 13: eps times the global maximum
  double *r = rows + (long long)p * naux;
  double c = 0.0;
  for (int q = threadIdx.x; q < naux; q += blockDim.x) {
    const double x = r[q];
    if (fabs(x) >= thr) c += (x != 0.0) ? 1.0 : 0.0;
    else r[q] = 0.0;
  }
  c = block_sum(c);
  if (threadIdx.x == 0) cnt[p] = (int)c;
}

__global__ void gather_rows_kernel(const double *__restrict__ src, const int *__restrict__ idx,
                                   int ncols, double *__restrict__ dst) {
  const int r = blockIdx.x;
  const double *s = src + (long long)idx[r] * ncols;
  double *d = dst + (long long)r * ncols;
  for (int c = threadIdx.x; c < ncols; c += blockDim.x) d[c] = s[c];
}

__global__ void gather_int_kernel(const int *__restrict__ vals, const int *__restrict__ idx, int P,
                                  int *__restrict__ dst) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < P; r += gridDim.x * blockDim.x)
    dst[r] = vals[idx[r]];
}

__global__ void pair_csr_kernel(const int *__restrict__ pij, int P, int n, int *__restrict__ rowptr,
                                int *__restrict__ prow, int *__restrict__ pcol) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t <= n) {  // first pair with row >= t
    const long long key = (long long)t * n;
    int lo = 0, hi = P;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if ((long long)pij[mid] < key) lo = mid + 1;
      else hi = mid;
    }
    rowptr[t] = lo;
  }
  for (int a = t; a < P; a += gridDim.x * blockDim.x) {
    prow[a] = pij[a] / n;
    pcol[a] = pij[a] - prow[a] * n;
  }
}

__global__ void scatter_pairs_kernel(const double *__restrict__ src, int ns, int P,
                                     const int *__restrict__ pij, long long dst_stride,
                                     double *__restrict__ dst) {
  const long long total = (long long)ns * P;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long x = e / P;
    const int p = (int)(e - x * P);
    dst[x * dst_stride + pij[p]] = src[e];
  }
}

// ------------------------------------------------------------------ S4 ----
__global__ void rademacher_kernel(unsigned long long seed, int set, long long xi_offset, int ns,
                                  int naux, double *__restrict__ theta) {
  const long long total = (long long)ns * naux;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long x = e / naux;
    const int q = (int)(e - x * naux);
    const unsigned long long ctr = ((unsigned long long)set << 60) |
                                   ((unsigned long long)(xi_offset + x) << 20) |
                                   (unsigned long long)q;
    // first output of SplitMix64 (Steele, Lea & Flood 2014) from state seed ^ ctr
    unsigned long long z = (seed ^ ctr) + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    theta[e] = (z >> 63) ? -1.0 : 1.0;
  }
}

// ------------------------------------------------------------------ S6 ----
__global__ void green_scale_kernel(const double *__restrict__ C, const double *__restrict__ e,
                                   int n, int off, int m, double mu, const double *__restrict__ tau,
                                   int ntau, int sign, double *__restrict__ cs) {
  const long long total = (long long)ntau * n * m;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const long long ti = k / ((long long)n * m);
    const long long r = k - ti * n * m;
    const int i = (int)(r / m), a = (int)(r - (long long)i * m);
    const double arg = (e[off + a] - mu) * tau[ti];
    cs[k] = C[(long long)i * n + off + a] * exp(sign > 0 ? arg : -arg);
  }
}

// ------------------------------------------------------------------ S7 ----
// Warp per output row pair (m, j): lanes run over the auxiliary index Q, QC
// fp64 accumulators per lane (32*QC values of Q per pass).  QC is chosen so
// that the passes cover N_aux with little padding (the DFMA pipe spends its
// cycles on padded lanes too).
template <int QC>
__global__ void __launch_bounds__(128) dd_spmm_kernel(
    const int *__restrict__ rowptr, const int *__restrict__ pcol, const double *__restrict__ D,
    int P, const double *__restrict__ At, int n, int naux, double *__restrict__ T) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * 4 + warp;
  const int m = blockIdx.y;
  if (j >= n) return;
  const int a0 = rowptr[m], a1 = rowptr[m + 1];
  const int b0 = rowptr[j], b1 = rowptr[j + 1];
  for (int q0 = 0; q0 < naux; q0 += 32 * QC) {
    double acc[QC];
#pragma unroll
    for (int c = 0; c < QC; ++c) acc[c] = 0.0;
    const int qv = naux - q0 - lane;  // lanes with q0 + lane + 32c < naux
    for (int a = a0; a < a1; ++a) {
      const double *Drow = D + (long long)a * P;
      const double *Ak = At + (long long)pcol[a] * n * naux + q0 + lane;
      for (int b = b0; b < b1; ++b) {
        const double d = Drow[b];
        const double *ap = Ak + (long long)pcol[b] * naux;
#pragma unroll
        for (int c = 0; c < QC; ++c)
          if (32 * c < qv) acc[c] = fma(d, ap[32 * c], acc[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < QC; ++c)
      if (32 * c < qv) T[((long long)m * naux + q0 + lane + 32 * c) * n + j] = acc[c];
  }
}

__global__ void dd_fold_kernel(const int *__restrict__ prow, const int *__restrict__ pcol,
                               const double *__restrict__ L, int P, int n, int naux,
                               double *__restrict__ T) {
  const long long total = (long long)P * naux;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long a = e / naux;
    const int q = (int)(e - a * naux);
    T[((long long)prow[a] * naux + q) * n + pcol[a]] -= 2.0 * L[e];
  }
}

// ------------------------------------------------------------------ S8 ----
// One block per batch entry.  Tr(B B) = sum_ij B_ij B_ji is taken over pairs of
// 32 x 32 tiles staged in shared memory (both tiles read coalesced), then the
// entry is overwritten with sgn (2 t I - B), or written as (hi, lo) float pairs
// into Bhl when that is given (the double-float chain's next operand).
__global__ void chain_fold_kernel(double *__restrict__ Bm, int npos, int n, double *__restrict__ t,
                                  double *__restrict__ s2, float2 *__restrict__ Bhl) {
  __shared__ double ta[32][33], tb[32][33];
  const int b = blockIdx.x;
  const long long nn = (long long)n * n;
  double *B = Bm + (long long)b * nn;
  double tl = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) tl += B[(long long)i * n + i];
  const double tr = block_sum(tl);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5, nty = blockDim.x >> 5;
  const int ntile = (n + 31) / 32;
  double sl = 0.0;
  for (int bi = 0; bi < ntile; ++bi)
    for (int bj = 0; bj < ntile; ++bj) {
      __syncthreads();
      for (int r = ty; r < 32; r += nty) {
        const int i = bi * 32 + r, j = bj * 32 + tx;        // tile (bi, bj)
        const int i2 = bj * 32 + r, j2 = bi * 32 + tx;      // tile (bj, bi)
        ta[r][tx] = (i < n && j < n) ? B[(long long)i * n + j] : 0.0;
        tb[r][tx] = (i2 < n && j2 < n) ? B[(long long)i2 * n + j2] : 0.0;
      }
      __syncthreads();
      for (int r = ty; r < 32; r += nty) sl += ta[r][tx] * tb[tx][r];  // B_ij B_ji
    }
  const double ss = block_sum(sl);  // ends with a barrier: all reads are done
  const double sg = (b < npos) ? 1.0 : -1.0;
  for (long long e = threadIdx.x; e < nn; e += blockDim.x) {
    const long long i = e / n, j = e - i * n;
    const double v = sg * (((i == j) ? 2.0 * tr : 0.0) - B[e]);
    if (Bhl) {
      const float hi = __double2float_rn(v);
      Bhl[(long long)b * nn + e] = make_float2(hi, __double2float_rn(v - (double)hi));
    } else {
      B[e] = v;
    }
  }
  if (threadIdx.x == 0) {
    t[b] = tr;
    s2[b] = ss;
  }
}

// the kinds of one sample pair are summed first (they cancel to the small
// stochastic part), then the pairs in order
__global__ void sigma_accumulate_kernel(const double *__restrict__ BC, int nh, int nkind, long long nn,
                                        double ns_div, const double *__restrict__ base, int init,
                                        double *__restrict__ sig) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn;
       e += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int x = 0; x < nh; ++x) {
      double v = BC[(long long)x * nn + e];
      for (int k = 1; k < nkind; ++k) v += BC[(long long)(k * nh + x) * nn + e];
      acc += v;
    }
    const double add = acc / ns_div;
    sig[e] = init ? base[e] + add : sig[e] + add;
  }
}

// kinds k < kpos enter with +, the others with -: Tr(F Gb) = 2 t^2 - Tr(B B)
__global__ void pair_energy_kernel(const double *__restrict__ t, const double *__restrict__ s2,
                                   int nh, int nkind, int kpos, double w, double ne,
                                   double *__restrict__ e_st) {
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nh; x += gridDim.x * blockDim.x) {
    double de = 0.0;
    for (int k = 0; k < nkind; ++k) {
      const double v = 2.0 * t[k * nh + x] * t[k * nh + x] - s2[k * nh + x];
      de += k < kpos ? v : -v;
    }
    e_st[x] += -w * de / ne;
  }
}

// ------------------------------------------- literal estimator (Eq. 25) --
// out[e][s] = in[s][e] for s < S, e < nn (32 x 32 tiles through shared memory)
__global__ void lit_qfast_kernel(const double *__restrict__ in, int S, long long nn,
                                 double *__restrict__ out) {
  __shared__ double tile[32][33];
  const long long e0 = (long long)blockIdx.x * 32;
  const int s0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  for (int r = ty; r < 32; r += 8) {
    const int sv = s0 + r;
    const long long e = e0 + tx;
    tile[r][tx] = (sv < S && e < nn) ? in[(long long)sv * nn + e] : 0.0;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const long long e = e0 + r;
    const int sv = s0 + tx;
    if (e < nn && sv < S) out[e * S + sv] = tile[tx][r];
  }
}

// W[s][m][j] = -Tk[m][s][j]
__global__ void lit_w_kernel(const double *__restrict__ Tk, int S, int n, double *__restrict__ W) {
  const long long total = (long long)S * n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long j = e % n, ms = e / n;  // ms = m * S + s
    const long long m = ms / S, sv = ms - m * S;
    W[(sv * n + m) * n + j] = -Tk[e];
  }
}

// W[s][prow a][pcol a] += 2 JP[a][s] (each target is written by one thread)
__global__ void lit_direct_kernel(const double *__restrict__ JP, const int *__restrict__ pij, int P,
                                  int S, long long nn, double *__restrict__ W) {
  const long long total = (long long)P * S;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long a = e / S, sv = e - a * S;
    W[sv * nn + pij[a]] += 2.0 * JP[e];
  }
}

// Per sample x (one block): z = sum_side sgn(side) Z[side][x], added into the
// first chain slot, and e_st[x] += -w Tr(z Gb) / ne.  Sides 0 and 2 enter
// with +, sides 1 and 3 with -.
__global__ void lit_add_kernel(const double *__restrict__ Z, int cnt, int n,
                               const double *__restrict__ Gb, double w, double ne,
                               double *__restrict__ F0, double *__restrict__ e_st) {
  const int x = blockIdx.x;
  const long long nn = (long long)n * n;
  double part = 0.0;
  for (long long e = threadIdx.x; e < nn; e += blockDim.x) {
    const double z = Z[(0LL * cnt + x) * nn + e] - Z[(1LL * cnt + x) * nn + e] +
                     Z[(2LL * cnt + x) * nn + e] - Z[(3LL * cnt + x) * nn + e];
    F0[(long long)x * nn + e] += z;
    const long long i = e / n, j = e - i * n;
    part += z * Gb[j * n + i];
  }
  const double de = block_sum(part);
  if (threadIdx.x == 0) e_st[x] += -w * de / ne;
}

// ------------------------------------------------------------------ S9 ----
__global__ void trace_prod_kernel(const double *__restrict__ X, const double *__restrict__ Y, int n,
                                  double *__restrict__ out) {
  const int ti = blockIdx.x;
  const long long nn = (long long)n * n;
  const double *x = X + ti * nn, *y = Y + ti * nn;
  double s = 0.0;
  for (long long e = threadIdx.x; e < nn; e += blockDim.x) {
    const long long i = e / n, j = e - i * n;
    s += x[e] * y[j * n + i];
  }
  s = block_sum(s);
  if (threadIdx.x == 0) out[ti] = s;
}

__global__ void energy_finalize_kernel(const double *__restrict__ w, const double *__restrict__ trdd,
                                       const double *__restrict__ tr, int ntau, double ne,
                                       const double *__restrict__ e_st, int ns,
                                       double *__restrict__ e_pair, double *__restrict__ res) {
  __shared__ double sh_edd, sh_e;
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < ntau; ++k) {
      a += w[k] * trdd[k];
      b += w[k] * tr[k];
    }
    sh_edd = -a / ne;
    sh_e = -b / ne;
  }
  __syncthreads();
  const double edd = sh_edd;
  double s = 0.0;
  for (int x = threadIdx.x; x < ns; x += blockDim.x) {
    const double v = edd + e_st[x];
    e_pair[x] = v;
    s += v;
  }
  const double mean = block_sum(s) / ns;
  double q = 0.0;
  for (int x = threadIdx.x; x < ns; x += blockDim.x) {
    const double d = (edd + e_st[x]) - mean;
    q += d * d;
  }
  const double ss = block_sum(q);
  if (threadIdx.x == 0) {
    res[0] = edd;
    res[1] = sh_e;
    res[2] = mean;
    res[3] = (ns > 1) ? sqrt(ss / (ns - 1) / ns) : 0.0;
  }
}

// ----------------------------------------------------------------- S10 ----
__global__ void symmetrize_kernel(const double *__restrict__ in, int n, long long total,
                                  double *__restrict__ out) {
  const long long nn = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long t = e / nn, r = e - t * nn;
    const long long i = r / n, j = r - i * n;
    out[e] = 0.5 * (in[e] + in[t * nn + j * n + i]);
  }
}

__global__ void nonfinite_kernel(const double *__restrict__ x, long long len, int *__restrict__ flag) {
  int bad = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len;
       e += (long long)gridDim.x * blockDim.x)
    if (!isfinite(x[e])) bad = 1;
  if (__any_sync(FULL, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

}  // namespace

// ================================================================ launchers
long long &launch_counter() {
  static thread_local long long count = 0;
  return count;
}

#define RS_LAUNCHED()            \
  do {                           \
    ++launch_counter();          \
    RS_TRY(cudaGetLastError());  \
  } while (0)

cudaError_t absmax(const double *x, long long len, double *out, double *part, cudaStream_t s) {
  const int nb = std::min(grid_for(len, 256), 1024);
  absmax_partial_kernel<<<nb, 256, 0, s>>>(x, len, part);
  RS_LAUNCHED();
  max_final_kernel<<<1, 1024, 0, s>>>(part, nb, out);
  RS_LAUNCHED();
  return cudaSuccess;
}

cudaError_t ns_init(const double *V, int na, double *Y, double *Z, double *scal, double *part,
                    cudaStream_t s) {
  rowsum_abs_kernel<<<na, 256, 0, s>>>(V, na, part);
  RS_LAUNCHED();
  max_final_kernel<<<1, 1024, 0, s>>>(part, na, scal);
  RS_LAUNCHED();
  ns_init_kernel<<<grid_for((long long)na * na, 256), 256, 0, s>>>(V, na, scal, Y, Z);
  RS_LAUNCHED();
  return cudaSuccess;
}

cudaError_t ns_tbuild(const double *P, int na, double *T, double *scal, double *part,
                      cudaStream_t s) {
  const int nb = std::min(grid_for((long long)na * na, 256), 1024);
  ns_tbuild_kernel<<<nb, 256, 0, s>>>(P, na, T, part);
  RS_LAUNCHED();
  max_final_kernel<<<1, 1024, 0, s>>>(part, nb, scal + 1);
  RS_LAUNCHED();
  return cudaSuccess;
}

cudaError_t ns_finish(const double *Z, int na, const double *scal, double *W, cudaStream_t s) {
  ns_finish_kernel<<<grid_for((long long)na * na, 256), 256, 0, s>>>(Z, na, scal, W);
  RS_LAUNCHED();
  return cudaSuccess;
}

cudaError_t eri_check(const double *eri3, int n, int naux, int *flags, cudaStream_t s) {
  eri_check_kernel<<<grid_for((long long)n * n * naux, 256), 256, 0, s>>>(eri3, n, naux, flags);
  RS_LAUNCHED();
  return cudaSuccess;
}

cudaError_t eri_colmax(const double *eri3, int n, int naux, double *colmax, cudaStream_t s) {
  eri_colmax_kernel<<<n, 512, 0, s>>>(eri3, n, naux, colmax);
  RS_LAUNCHED();
  return cudaSuccess;
}

cudaError_t eri_pair_count(const double *eri3, int n, int naux, const double *colmax,
                           double eps_prime, int *cnt, cudaStream_t s) {
  const long long pairs = (long long)n * n;
  eri_pair_count_kernel<<<(int)((pairs + 7) / 8), 256, 0, s>>>(eri3, n, naux, colmax, eps_prime,
                                                               cnt);
  RS_LAUNCHED();
  return cudaSuccess;
}

cudaError_t eri_gather_rows(const double *eri3, int n, int naux, const double *colmax,
                            double eps_prime, const int *pairs, int P, double *out,
                            cudaStream_t s) {
  if (P <= 0) return cudaSuccess;
  eri_gather_rows_kernel<<<P, 128, 0, s>>>(eri3, n, naux, colmax, eps_prime, pairs, out);
  RS_LAUNCHED();
  return cudaSuccess;
}

size_t compact_scratch_bytes(int len) {
  const size_t nb = (size_t)std::max(1, ceil_div(len, CB));
  return nb * (2 * sizeof(int) + sizeof(long long)) + 64;
}

cudaError_t compact(const int *cnt, int len, int *idx, int *count, long long *sum64, void *scratch,
                    cudaStream_t s) {
  const int nb = std::max(1, ceil_div(len, CB));
  long long *bsum = reinterpret_cast<long long *>(scratch);
  int *bcount = reinterpret_cast<int *>(bsum + nb);
  int *boff = bcount + nb;
  compact_count_kernel<<<nb, CT, 0, s>>>(cnt, len, bcount, bsum);
  RS_LAUNCHED();
  compact_scan_kernel<<<1, 1024, 0, s>>>(bcount, bsum, nb, boff, count, sum64);
  RS_LAUNCHED();
  compact_write_kernel<<<nb, CT, 0, s>>>(cnt, len, boff, idx);
  RS_LAUNCHED();
  return cudaSuccess;
}

cudaError_t kl_cut(double *rows, int P, int naux, const double *kmax, double eps, int *cnt,
                   cudaStream_t s) {
  if (P <= 0) return cudaSuccess;
  kl_cut_kernel<<<P, 128, 0, s>>>(rows, naux, kmax, eps, cnt);
  RS_LAUNCHED();
  return cudaSuccess;
}

cudaError_t gather_rows(const double *src, const int *idx, int P, int ncols, double *dst,
                        cudaStream_t s) {
  if (P <= 0) return cudaSuccess;
  gather_rows_kernel<<<P, 128, 0, s>>>(src, idx, ncols, dst);
  RS_LAUNCHED();
  return cudaSuccess;
}

cudaError_t gather_int(const int *vals, const int *idx, int P, int *dst, cudaStream_t s) {
  if (P <= 0) return cudaSuccess;
  gather_int_kernel<<<grid_for(P, 256), 256, 0, s>>>(vals, idx, P, dst);
  RS_LAUNCHED();
  return cudaSuccess;
}

cudaError_t pair_csr(const int *pair_ij, int P, int n, int *rowptr, int *prow, int *pcol,
                     cudaStream_t s) {
  const int work = std::max(P, n + 1);
  pair_csr_kernel<<<grid_for(work, 256, 1 << 20), 256, 0, s>>>(pair_ij, P, n, rowptr, prow, pcol);
  RS_LAUNCHED();
  return cudaSuccess;
}

cudaError_t scatter_pairs(const double *src, int ns, int P, const int *pair_ij, long long nn,
                          long long dst_stride, double *dst, cudaStream_t s) {
  (void)nn;
  if (P <= 0 || ns <= 0) return cudaSuccess;
  scatter_pairs_kernel<<<grid_for((long long)ns * P, 256), 256, 0, s>>>(src, ns, P, pair_ij,
                                                                         dst_stride, dst);
  RS_LAUNCHED();
  return cudaSuccess;
}

cudaError_t rademacher(unsigned long long seed, int set, long long xi_offset, int ns, int naux,
                       double *theta, cudaStream_t s) {
  rademacher_kernel<<<grid_for((long long)ns * naux, 256), 256, 0, s>>>(seed, set, xi_offset, ns,
                                                                         naux, theta);
  RS_LAUNCHED();
  return cudaSuccess;
}

cudaError_t green_scale(const double *C, const double *e, int n, int off, int m, double mu,
                        const double *tau, int ntau, int sign, double *cs, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  green_scale_kernel<<<grid_for((long long)ntau * n * m, 256), 256, 0, s>>>(C, e, n, off, m, mu,
                                                                             tau, ntau, sign, cs);
  RS_LAUNCHED();
  return cudaSuccess;
}

cudaError_t dd_exchange_spmm(const int *rowptr, const int *pcol, const double *D, int P,
                             const double *At, int n, int naux, double *T, cudaStream_t s) {
  // accumulators per lane: fewest padded lanes over ceil(naux / (32 QC)) passes
  static const int kQC[] = {1, 2, 3, 4, 5, 6, 8, 10, 12, 16, 20, 24};
  int best = 8;
  long long best_lanes = -1;
  for (int qc : kQC) {
    const long long passes = (naux + 32LL * qc - 1) / (32LL * qc);
    const long long lanes = passes * 32 * qc + passes * 64;  // small cost per pass
    if (best_lanes < 0 || lanes < best_lanes) {
      best_lanes = lanes;
      best = qc;
    }
  }
  dim3 grid(ceil_div(n, 4), n);
#define RS_SPMM(QC) \
  case QC: dd_spmm_kernel<QC><<<grid, 128, 0, s>>>(rowptr, pcol, D, P, At, n, naux, T); break;
  switch (best) {
    RS_SPMM(1) RS_SPMM(2) RS_SPMM(3) RS_SPMM(4) RS_SPMM(5) RS_SPMM(6) RS_SPMM(8) RS_SPMM(10)
    RS_SPMM(12) RS_SPMM(16) RS_SPMM(20) RS_SPMM(24)
    default: return cudaErrorInvalidValue;
  }
#undef RS_SPMM
  RS_LAUNCHED();
  return cudaSuccess;
}

cudaError_t dd_fold_direct(const int *prow, const int *pcol, const double *L, int P, int n,
                           int naux, double *T, cudaStream_t s) {
  if (P <= 0) return cudaSuccess;
  dd_fold_kernel<<<grid_for((long long)P * naux, 256), 256, 0, s>>>(prow, pcol, L, P, n, naux, T);
  RS_LAUNCHED();
  return cudaSuccess;
}

cudaError_t chain_fold(double *Bm, int nb, int npos, int n, double *t, double *s2,
                       float2 *Bhl, cudaStream_t s) {
  chain_fold_kernel<<<nb, 256, 0, s>>>(Bm, npos, n, t, s2, Bhl);
  RS_LAUNCHED();
  return cudaSuccess;
}

cudaError_t sigma_accumulate(const double *BC, int nh, int nkind, int n, double ns_div,
                             const double *base, int init, double *sig, cudaStream_t s) {
  const long long nn = (long long)n * n;
  sigma_accumulate_kernel<<<grid_for(nn, 256), 256, 0, s>>>(BC, nh, nkind, nn, ns_div, base, init,
                                                             sig);
  RS_LAUNCHED();
  return cudaSuccess;
}

cudaError_t pair_energy(const double *t, const double *s2, int nh, int nkind, int kpos, double w,
                        double ne, double *e_st, cudaStream_t s) {
  pair_energy_kernel<<<grid_for(nh, 256), 256, 0, s>>>(t, s2, nh, nkind, kpos, w, ne, e_st);
  RS_LAUNCHED();
  return cudaSuccess;
}

cudaError_t lit_qfast(const double *in, int S, long long nn, double *out, cudaStream_t s) {
  if (S <= 0 || nn <= 0) return cudaSuccess;
  dim3 grid((unsigned)((nn + 31) / 32), (S + 31) / 32);
  if (grid.y > 65535) return cudaErrorInvalidValue;
  lit_qfast_kernel<<<grid, 256, 0, s>>>(in, S, nn, out);
  RS_LAUNCHED();
  return cudaSuccess;
}

cudaError_t lit_w(const double *Tk, int S, int n, const double *JP, const int *pij, int P,
                  double *W, cudaStream_t s) {
  const long long total = (long long)S * n * n;
  lit_w_kernel<<<grid_for(total, 256), 256, 0, s>>>(Tk, S, n, W);
  RS_LAUNCHED();
  if (P > 0) {
    lit_direct_kernel<<<grid_for((long long)P * S, 256), 256, 0, s>>>(JP, pij, P, S,
                                                                      (long long)n * n, W);
    RS_LAUNCHED();
  }
  return cudaSuccess;
}

cudaError_t lit_add(const double *Z, int cnt, int n, const double *Gb, double w, double ne,
                    double *F0, double *e_st, cudaStream_t s) {
  lit_add_kernel<<<cnt, 256, 0, s>>>(Z, cnt, n, Gb, w, ne, F0, e_st);
  RS_LAUNCHED();
  return cudaSuccess;
}

cudaError_t trace_prod(const double *X, const double *Y, int n, int ntau, double *out,
                       cudaStream_t s) {
  trace_prod_kernel<<<ntau, 256, 0, s>>>(X, Y, n, out);
  RS_LAUNCHED();
  return cudaSuccess;
}

cudaError_t energy_finalize(const double *tau_w, const double *trdd, const double *tr, int ntau,
                            double ne, const double *e_st, int ns, double *e_pair, double *res,
                            cudaStream_t s) {
  energy_finalize_kernel<<<1, 256, 0, s>>>(tau_w, trdd, tr, ntau, ne, e_st, ns, e_pair, res);
  RS_LAUNCHED();
  return cudaSuccess;
}

cudaError_t symmetrize(const double *in, int n, int ntau, double *out, cudaStream_t s) {
  const long long total = (long long)ntau * n * n;
  symmetrize_kernel<<<grid_for(total, 256), 256, 0, s>>>(in, n, total, out);
  RS_LAUNCHED();
  return cudaSuccess;
}

cudaError_t nonfinite_check(const double *x, long long len, int *flag, cudaStream_t s) {
  if (len <= 0) return cudaSuccess;
  nonfinite_kernel<<<grid_for(len, 256), 256, 0, s>>>(x, len, flag);
  RS_LAUNCHED();
  return cudaSuccess;
}

}  // namespace rssri
