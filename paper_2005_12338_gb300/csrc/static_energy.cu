// rssri_energy_static: the Eq. 26 energy of a caller-held self-energy, for
// callers that may not allocate device memory.
//
// Some callers cannot call cudaMalloc: code running while a stream is being
// captured into a CUDA graph (an allocation there breaks the capture), hosts
// that hand every byte of device memory to their own pool allocator and forbid
// libraries from allocating behind their back, and real-time loops that must
// not hit the allocator's synchronisation.  This entry point creates no handle
// and allocates nothing: its only scratch (one partial trace per tau point) is
// a file-scope __device__ array of fixed size, loaded with the library and
// held by every GPU that loads it until the process exits.
#include <mutex>

#include "kernels.cuh"

namespace {

// One fp64 slot per tau point; RSSRI_STATIC_MAX_TAU slots (32 KiB).
static __device__ __align__(256) double g_energy_scratch[RSSRI_STATIC_MAX_TAU];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  The symbol's
// host-side name is only a stand-in: the address must come from
// cudaGetSymbolAddress with that device current.  Looked up once per device.
cudaError_t scratch_on_current_device(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_energy_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// e_corr = -(sum_t w_t tr[t]) / ne, summed in tau order (the same order as
// the energy of rssri_sigma).
__global__ void static_energy_finalize_kernel(const double *__restrict__ tau_w,
                                              const double *__restrict__ tr, int ntau, double ne,
                                              double *__restrict__ e_corr) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double b = 0.0;
  for (int k = 0; k < ntau; ++k) b += tau_w[k] * tr[k];
  e_corr[0] = -b / ne;
}

}  // namespace

extern "C" int rssri_energy_static(const double *sigma, const double *gb, const double *tau_w,
                                   int n, int n_tau, int n_occ, double *e_corr, void *stream) {
  if (!sigma || !gb || !tau_w || !e_corr) return RSSRI_ERR_INVALID_ARG;
  if (n < 1 || n > 4096 || n_occ < 1 || n_tau < 1) return RSSRI_ERR_INVALID_ARG;
  if (n_tau > RSSRI_STATIC_MAX_TAU) return RSSRI_ERR_INVALID_ARG;  // beyond the static scratch
  double *scratch = nullptr;
  cudaError_t e = scratch_on_current_device(&scratch);
  if (e != cudaSuccess) return RSSRI_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // every slot read below is written first by this call, so nothing needs clearing
  e = rssri::trace_prod(sigma, gb, n, n_tau, scratch, s);
  if (e != cudaSuccess) return RSSRI_ERR_CUDA;
  static_energy_finalize_kernel<<<1, 32, 0, s>>>(tau_w, scratch, n_tau, 2.0 * n_occ, e_corr);
  e = cudaGetLastError();
  return e == cudaSuccess ? RSSRI_OK : RSSRI_ERR_CUDA;
}
