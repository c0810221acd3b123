// Arithmetic-pipe peaks of the GPU this library runs on, measured with CUDA
// events: the ceilings against which the fp64 and double-float kernels of
// the path are reported.  Each measurement runs compute-only kernels on
// every SM in several shapes (independent dependency chains per thread x
// resident warps per SM, with shared or distinct operand registers) and
// reports the best rate, so that the figure is the pipe's and not one shape's.
//
//   RSSRI_PEAK_DFMA   fp64 fused multiply-add (the DFMA pipe)
//   RSSRI_PEAK_DMMA   fp64 mma.sync m8n8k4 (the fp64 tensor path of mma.sync)
//   RSSRI_PEAK_FFMA   fp32 fused multiply-add (the pipe the double-float form uses)
#include <algorithm>

#include "common.cuh"
#include "rssri_peak.h"

namespace {

// CH independent chains per thread; DISTINCT: each chain has its own
// multiplier and addend registers (else all chains share two registers).
template <class T, int CH, bool DISTINCT>
__global__ void fma_chains(T *out, T a, T b, int iters) {
  T x[CH], y[CH], z[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    y[c] = a + (T)c * (T)1e-9;
    z[c] = b + (T)c * (T)1e-12;
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int c = 0; c < CH; ++c) x[c] = DISTINCT ? fma(x[c], y[c], z[c]) : fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += x[c];
  // never true for the arguments the launcher passes; keeps the chains live
  if (s == (T)-12345.0) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// D = A B + D with A 8x4, B 4x8, D 8x8 (fp64), per warp; CH independent
// accumulators.
template <int CH>
__global__ void dmma_chains(double *out, double a, double b, int iters) {
  double d[CH][2];
#pragma unroll
  for (int c = 0; c < CH; ++c) d[c][0] = d[c][1] = 0.0;
  const double av = a * (threadIdx.x & 3), bv = b * (threadIdx.x >> 3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int c = 0; c < CH; ++c)
        asm volatile(
            "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
            : "+d"(d[c][0]), "+d"(d[c][1])
            : "d"(av), "d"(bv));
  }
  double s = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += d[c][0] + d[c][1];
  if (s == -12345.0) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

struct Shape {
  void (*fn)(void *, int, int, int);  // launcher: (out, blocks, threads, iters)
  int ch;
  double flop_per_thread_iter;  // per thread and outer iteration
};

template <class T, int CH, bool D>
void launch_fma(void *out, int blocks, int threads, int iters) {
  fma_chains<T, CH, D><<<blocks, threads>>>((T *)out, (T)0.999999, (T)1e-7, iters);
}
template <int CH>
void launch_dmma(void *out, int blocks, int threads, int iters) {
  dmma_chains<CH><<<blocks, threads>>>((double *)out, 1e-3, 1e-3, iters);
}

// Time one shape: one warm-up launch, then 3 timed; returns TFLOP/s (0 on error).
double time_shape(const Shape &sh, void *out, int blocks, int threads, int iters, double *ms_out) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return 0.0;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return 0.0;
  }
  sh.fn(out, blocks, threads, iters);
  cudaEventRecord(e0);
  const int reps = 3;
  for (int r = 0; r < reps; ++r) sh.fn(out, blocks, threads, iters);
  cudaEventRecord(e1);
  float ms = 0;
  const bool ok = cudaEventSynchronize(e1) == cudaSuccess &&
                  cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
                  cudaGetLastError() == cudaSuccess && ms > 0.f;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok) return 0.0;
  if (ms_out) *ms_out = ms / reps;
  return sh.flop_per_thread_iter * iters * (double)blocks * threads * reps / (ms * 1e-3) / 1e12;
}

}  // namespace

extern "C" int rssri_peak_measure(int which, int device, double *tflops, double *ms_out) {
  if (!tflops || (which != RSSRI_PEAK_DFMA && which != RSSRI_PEAK_DMMA &&
                  which != RSSRI_PEAK_FFMA))
    return RSSRI_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return RSSRI_ERR_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return RSSRI_ERR_CUDA;
  void *out = nullptr;
  if (cudaMalloc(&out, (size_t)sms * 2048 * sizeof(double)) != cudaSuccess) return RSSRI_ERR_OOM;
  // fma: 2 flop x CH chains x 16 unrolled per iteration; dmma: 512 flop per warp
  // instruction = 16 per thread, x CH x 4 unrolled
  Shape dfma[] = {{launch_fma<double, 4, false>, 4, 2.0 * 4 * 16},
                  {launch_fma<double, 8, false>, 8, 2.0 * 8 * 16},
                  {launch_fma<double, 8, true>, 8, 2.0 * 8 * 16},
                  {launch_fma<double, 16, true>, 16, 2.0 * 16 * 16}};
  Shape ffma[] = {{launch_fma<float, 4, false>, 4, 2.0 * 4 * 16},
                  {launch_fma<float, 8, false>, 8, 2.0 * 8 * 16},
                  {launch_fma<float, 8, true>, 8, 2.0 * 8 * 16},
                  {launch_fma<float, 16, true>, 16, 2.0 * 16 * 16}};
  Shape dmma[] = {{launch_dmma<4>, 4, 16.0 * 4 * 4}, {launch_dmma<8>, 8, 16.0 * 8 * 4}};
  Shape *shapes = which == RSSRI_PEAK_DFMA ? dfma : which == RSSRI_PEAK_FFMA ? ffma : dmma;
  const int nshape = which == RSSRI_PEAK_DMMA ? 2 : 4;
  // about 10 ms per launch at the pipe's rate
  const long long per_sm_flop = which == RSSRI_PEAK_FFMA ? 5000000000LL : 100000000LL;
  double best = 0.0, best_ms = 0.0;
  for (int k = 0; k < nshape; ++k)
    for (int warps : {16, 32, 64}) {  // resident warps per SM
      const int threads = 256, blocks = sms * warps * 32 / threads;
      const int iters = (int)std::max<long long>(
          1, per_sm_flop / (long long)(shapes[k].flop_per_thread_iter * warps * 32));
      double ms = 0.0;
      const double tf = time_shape(shapes[k], out, blocks, threads, iters, &ms);
      if (tf > best) {
        best = tf;
        best_ms = ms;
      }
    }
  cudaFree(out);
  if (!(best > 0.0)) return RSSRI_ERR_CUDA;
  *tflops = best;
  if (ms_out) *ms_out = best_ms;
  return RSSRI_OK;
}
