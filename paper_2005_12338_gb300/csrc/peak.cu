// Arithmetic-pipe peaks of the GPU this library runs on, measured with CUDA
// events: the ceilings against which the fp64 and double-float kernels of
// the path are reported.  Each kernel runs independent dependency chains
// (enough of them per thread, and enough warps per SM, to hide the pipe's
// latency) on every SM; the result is flops / elapsed time.
//
//   RSSRI_PEAK_DFMA   fp64 fused multiply-add (the DFMA pipe)
//   RSSRI_PEAK_DMMA   fp64 mma.sync m8n8k4 (the fp64 tensor path of mma.sync)
//   RSSRI_PEAK_FFMA   fp32 fused multiply-add (the pipe the double-float form uses)
#include <cstdio>

#include "common.cuh"
#include "rssri_peak.h"

namespace {

constexpr int CHAINS = 8;

template <class T>
__global__ void __launch_bounds__(256) fma_chains(T *out, T a, T b, int iters) {
  T x[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int c = 0; c < CHAINS; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += x[c];
  // never true for the arguments the launcher passes; keeps the chains live
  if (s == (T)-12345.0) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// D = A B + D with A 8x4, B 4x8, D 8x8 (fp64), per warp; CHAINS independent
// accumulators.
__global__ void __launch_bounds__(256) dmma_chains(double *out, double a, double b, int iters) {
  double d[CHAINS][2];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) d[c][0] = d[c][1] = 0.0;
  const double av = a * (threadIdx.x & 3), bv = b * (threadIdx.x >> 3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int c = 0; c < CHAINS; ++c)
        asm volatile(
            "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
            : "+d"(d[c][0]), "+d"(d[c][1])
            : "d"(av), "d"(bv));
  }
  double s = 0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += d[c][0] + d[c][1];
  if (s == -12345.0) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
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
  const int threads = 256, blocks = sms * 8;  // 64 warps per SM
  // fp64 pipes are ~64x slower than fp32: fewer iterations there
  const int iters = which == RSSRI_PEAK_FFMA ? 4096 : which == RSSRI_PEAK_DFMA ? 256 : 256;
  void *out = nullptr;
  if (cudaMalloc(&out, (size_t)blocks * threads * sizeof(double)) != cudaSuccess)
    return RSSRI_ERR_OOM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto launch = [&]() {
    if (which == RSSRI_PEAK_DFMA)
      fma_chains<double><<<blocks, threads>>>((double *)out, 0.999999, 1e-7, iters);
    else if (which == RSSRI_PEAK_FFMA)
      fma_chains<float><<<blocks, threads>>>((float *)out, 0.999999f, 1e-7f, iters);
    else
      dmma_chains<<<blocks, threads>>>((double *)out, 1e-3, 1e-3, iters);
  };
  launch();  // warm-up (clocks ramp, module load)
  cudaEventRecord(e0);
  const int reps = 5;
  for (int r = 0; r < reps; ++r) launch();
  cudaEventRecord(e1);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess || ms <= 0.f) return RSSRI_ERR_CUDA;
  double flops;
  if (which == RSSRI_PEAK_DMMA)
    flops = 2.0 * 8 * 8 * 4 * CHAINS * 4.0 * iters * (blocks * threads / 32.0) * reps;
  else
    flops = 2.0 * CHAINS * 16.0 * iters * (double)blocks * threads * reps;
  *tflops = flops / (ms * 1e-3) / 1e12;
  if (ms_out) *ms_out = ms / reps;
  return RSSRI_OK;
}
