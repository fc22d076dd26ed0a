// noalloc.cu -- GetError for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc or cudaMallocAsync: code embedded in a host
// framework whose own allocator owns the whole device memory budget, code that must not
// allocate while another component captures CUDA graphs on the device, or real-time
// loops that cannot afford an allocation's implicit synchronisation.  For them this file
// offers spring_fourier_error_noalloc: the same computation as spring_fourier_error, with
// its scratch (the transformed images and the per-block partial sums) in one file-scope
// device array of fixed size instead of allocated memory.
//
// The array is a static device symbol: every GPU that loads the library holds it
// (SPRING_NOALLOC_SCRATCH_BYTES) until the process exits.  Host code cannot use the
// symbol's name as a device address, so on the first call on each device (with that
// device current) the address is looked up once with cudaGetSymbolAddress and cached; the
// same set-up copies the twiddle table into a second static array.  That first call
// must therefore come before any stream capture on the device.
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace spring {

static __device__ __align__(256) unsigned char g_noalloc_scratch[SPRING_NOALLOC_SCRATCH_BYTES];
static __device__ __align__(256) float2 g_noalloc_twiddle[TW_TOTAL];

struct NoallocDevice {
  bool ready = false;
  unsigned char* scratch = nullptr;
  float2* tw = nullptr;
};
static std::mutex g_noalloc_mu;
static NoallocDevice g_noalloc_dev[64];

// once per device, with that device current: symbol addresses and the twiddle table
static spring_status noalloc_setup(NoallocDevice** out) {
  int dev = 0;
  SPRING_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return invalid("device index out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  NoallocDevice& d = g_noalloc_dev[dev];
  if (!d.ready) {
    void* p = nullptr;
    SPRING_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    d.scratch = static_cast<unsigned char*>(p);
    SPRING_CUDA(cudaGetSymbolAddress(&p, g_noalloc_twiddle));
    d.tw = static_cast<float2*>(p);
    std::vector<float2> tw(TW_TOTAL);
    fill_twiddles(tw.data());
    SPRING_CUDA(cudaMemcpyToSymbol(g_noalloc_twiddle, tw.data(), sizeof(float2) * TW_TOTAL));
    d.ready = true;
  }
  *out = &d;
  return SPRING_OK;
}

}  // namespace spring

using namespace spring;

extern "C" spring_status spring_fourier_error_noalloc(const void* x, const uint8_t* S, const float* M,
                                                     int batch, int n, double* err, void* stream) {
  if (!valid_n(n)) return invalid("unsupported pattern side " + std::to_string(n));
  if (batch < 0) return invalid("negative batch");
  if (batch == 0) return SPRING_OK;
  if (!x || !S || !M || !err) return invalid("null pointer");
  const size_t nn = (size_t)n * n;
  const size_t work = sizeof(float2) * nn * (size_t)batch;
  const size_t part = sizeof(double) * 2 * (size_t)batch * err_strips(n);
  const size_t part_off = (work + 255) & ~(size_t)255;
  if (part_off + part > SPRING_NOALLOC_SCRATCH_BYTES)
    return invalid("batch x N x N too large for the fixed scratch: needs " +
                   std::to_string(part_off + part) + " bytes, the maximum is " +
                   std::to_string((size_t)SPRING_NOALLOC_SCRATCH_BYTES));
  NoallocDevice* d = nullptr;
  SPRING_TRY(noalloc_setup(&d));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  float2* wb = reinterpret_cast<float2*>(d->scratch);
  double* partials = reinterpret_cast<double*>(d->scratch + part_off);
  // every byte read below is written first by this call: no clearing needed
  SPRING_TRY(launch_row_fft_tw(n, -1, static_cast<const float2*>(x), wb, S, batch, 1.0f, d->tw, s));
  SPRING_TRY(launch_col_err_tw(n, wb, M, batch, partials, d->tw, s));
  return launch_err_finalize(n, partials, batch, err, nullptr, s);
}
