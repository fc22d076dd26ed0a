// ops.cu -- runtime plumbing of libspring and the operator-level C ABI (include/spring.h).
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda.h>

#include "internal.h"
#include "tma.cuh"

namespace spring {

// ------------------------------------------------------------------ errors
static thread_local std::string t_err;

void set_error(const std::string& msg) { t_err = msg; }

spring_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  std::string m = std::string(what) + " failed: " + cudaGetErrorString(e) + " (" + file + ":" +
                  std::to_string(line) + ")";
  set_error(m);
  if (e == cudaErrorMemoryAllocation) return SPRING_E_NOMEM;
  return SPRING_E_CUDA;
}

spring_status invalid(const std::string& msg) {
  set_error(msg);
  return SPRING_E_INVALID;
}

// ------------------------------------------------------------------ launch accounting
struct KStat {
  std::atomic<uint64_t> launches{0};
  std::atomic<uint64_t> timed{0};
  double total_ms = 0.0;
  double bytes = 0.0;        // algorithmic bytes of the last launch
  double timed_bytes = 0.0;  // summed over the timed launches
};
static KStat g_kstat[SPRING_KC_COUNT];
static std::atomic<uint64_t> g_launches{0};
static std::atomic<int> g_timing{0};
static std::mutex g_tmu;
struct Pending {
  int kc;
  cudaEvent_t a, b;
  double bytes;
};
static std::vector<Pending> g_pending;
static std::vector<cudaEvent_t> g_event_pool;
static thread_local cudaEvent_t t_begin_event = nullptr;

static cudaEvent_t take_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

static bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &st);
  return st != cudaStreamCaptureStatusNone;
}

void launch_begin(int kc, cudaStream_t s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  const uint64_t idx = g_kstat[kc].launches.fetch_add(1, std::memory_order_relaxed);
  t_begin_event = nullptr;
  const int stride = g_timing.load(std::memory_order_relaxed);
  if (stride > 0 && idx % (uint64_t)stride == 0 && kc != SPRING_KC_OTHER && !capturing(s)) {
    std::lock_guard<std::mutex> lk(g_tmu);
    t_begin_event = take_event();
    cudaEventRecord(t_begin_event, s);
  }
}

void launch_end(int kc, cudaStream_t s, double bytes) {
  g_kstat[kc].bytes = bytes;
  if (t_begin_event) {
    std::lock_guard<std::mutex> lk(g_tmu);
    cudaEvent_t b = take_event();
    cudaEventRecord(b, s);
    g_pending.push_back({kc, t_begin_event, b, bytes});
    t_begin_event = nullptr;
  }
}

static void drain_pending() {
  std::lock_guard<std::mutex> lk(g_tmu);
  for (auto& p : g_pending) {
    cudaEventSynchronize(p.b);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      g_kstat[p.kc].total_ms += ms;
      g_kstat[p.kc].timed_bytes += p.bytes;
      g_kstat[p.kc].timed.fetch_add(1);
    }
    g_event_pool.push_back(p.a);
    g_event_pool.push_back(p.b);
  }
  g_pending.clear();
}

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!cached[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = v > 0 ? v : 1;
  }
  return cached[dev];
}

// ------------------------------------------------------------------ device tables
static std::mutex g_tab_mu;
static DeviceTables g_tabs[64];
static bool g_tab_ok[64];

spring_status device_tables(DeviceTables* out) {
  int dev = 0;
  SPRING_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return invalid("device index out of range");
  if (g_tab_ok[dev]) {
    *out = g_tabs[dev];
    return SPRING_OK;
  }
  std::lock_guard<std::mutex> lk(g_tab_mu);
  if (!g_tab_ok[dev]) {
    std::vector<float2> tw(TW_TOTAL);
    fill_twiddles(tw.data());
    std::vector<long long> rc(1024), rs(1024);
    for (int k = 0; k < 1024; ++k) {
      const double th = (3.14159265358979323846 / 2.0) * (double)k / 1024.0;
      rc[k] = std::llround(std::cos(th) * 1073741824.0);
      rs[k] = std::llround(std::sin(th) * 1073741824.0);
    }
    char* mem = nullptr;
    const size_t tw_bytes = sizeof(float2) * TW_TOTAL, r_bytes = sizeof(long long) * 1024;
    SPRING_CUDA(cudaMalloc(&mem, tw_bytes + 2 * r_bytes + 256));
    SPRING_CUDA(cudaMemset(mem + tw_bytes + 2 * r_bytes, 0, 256));
    SPRING_CUDA(cudaMemcpy(mem, tw.data(), tw_bytes, cudaMemcpyHostToDevice));
    SPRING_CUDA(cudaMemcpy(mem + tw_bytes, rc.data(), r_bytes, cudaMemcpyHostToDevice));
    SPRING_CUDA(cudaMemcpy(mem + tw_bytes + r_bytes, rs.data(), r_bytes, cudaMemcpyHostToDevice));
    g_tabs[dev].tw = reinterpret_cast<const float2*>(mem);
    g_tabs[dev].rot_cos = reinterpret_cast<const long long*>(mem + tw_bytes);
    g_tabs[dev].rot_sin = reinterpret_cast<const long long*>(mem + tw_bytes + r_bytes);
    g_tabs[dev].status = reinterpret_cast<int*>(mem + tw_bytes + 2 * r_bytes);
    g_tab_ok[dev] = true;
  }
  *out = g_tabs[dev];
  return SPRING_OK;
}

spring_status take_device_status(int* out) {
  DeviceTables tb;
  SPRING_TRY(device_tables(&tb));
  int v = 0;
  SPRING_CUDA(cudaMemcpy(&v, tb.status, sizeof(int), cudaMemcpyDeviceToHost));
  if (v) SPRING_CUDA(cudaMemset(tb.status, 0, sizeof(int)));
  *out = v;
  return SPRING_OK;
}

spring_status check_device_waits() {
  int v = 0;
  SPRING_TRY(take_device_status(&v));
  if (v & 2) {
    set_error("a bounded device-side wait timed out (a TMA copy did not complete)");
    return SPRING_E_TIMEOUT;
  }
  return SPRING_OK;
}

// One block waits on an mbarrier that expects two arrivals and gets none: the bounded
// wait gives up after `cycles`, records the timed-out wait in the device status word
// exactly as the TMA column pass does, and returns.
__global__ void k_wait_check(int* status, long long cycles) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 2);
  mbar_fence_init();
  if (!mbar_wait_bounded(&bar, 0u, cycles)) atomicOr(status, 2);
}

// ------------------------------------------------------------------ TMA descriptors
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

spring_status encode_tmap_f32_3d(void* map, const void* base, int dim0, int dim1, int dim2, int box0,
                                 int box1) {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    SPRING_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    if (!p || q != cudaDriverEntryPointSuccess) {
      set_error("cuTensorMapEncodeTiled is not available from the driver");
      return SPRING_E_CUDA;
    }
    fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  const cuuint64_t dims[3] = {(cuuint64_t)dim0, (cuuint64_t)dim1, (cuuint64_t)dim2};
  const cuuint64_t strides[2] = {(cuuint64_t)dim0 * 4, (cuuint64_t)dim0 * dim1 * 4};
  const cuuint32_t box[3] = {(cuuint32_t)box0, (cuuint32_t)box1, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(reinterpret_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base),
                  dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
    return SPRING_E_CUDA;
  }
  return SPRING_OK;
}

// ------------------------------------------------------------------ scratch
spring_status Scratch::alloc(size_t bytes, cudaStream_t stream) {
  s = stream;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMallocAsync(&p, bytes, stream);
  if (e != cudaSuccess) {
    p = nullptr;
    cudaGetLastError();
    set_error(std::string("device scratch allocation of ") + std::to_string(bytes) +
              " bytes failed: " + cudaGetErrorString(e));
    return SPRING_E_NOMEM;
  }
  return SPRING_OK;
}

// ------------------------------------------------------------------ composite transforms
spring_status fft2_unitary(int n, int dir, const float2* in, float2* out, const uint8_t* Smul,
                           int batch, cudaStream_t s) {
  if (batch < 1) return SPRING_OK;
  const float inv = 1.0f / (float)n;
  if (dir < 0) {
    SPRING_TRY(launch_row_fft(n, -1, in, out, Smul, batch, 1.0f, s));
    SPRING_TRY(launch_col_fft(n, -1, out, batch, inv, s));
  } else {
    if (in != out)
      SPRING_CUDA(cudaMemcpyAsync(out, in, sizeof(float2) * (size_t)batch * n * n,
                                  cudaMemcpyDeviceToDevice, s));
    SPRING_TRY(launch_col_fft(n, +1, out, batch, inv, s));
    SPRING_TRY(launch_row_fft(n, +1, out, out, nullptr, batch, 1.0f, s));
  }
  return SPRING_OK;
}

static spring_status check_n(int n, int batch) {
  if (!valid_n(n)) return invalid("unsupported pattern side " + std::to_string(n));
  if (batch < 0) return invalid("negative batch");
  return SPRING_OK;
}

}  // namespace spring

using namespace spring;

#define ST(x) reinterpret_cast<cudaStream_t>(x)

extern "C" {

int spring_abi_version(void) { return SPRING_ABI_VERSION; }

spring_status spring_check_wait_timeout(long long cycles) {
  if (cycles < 1 || cycles > (1LL << 32)) return invalid("cycles must be in [1, 2^32]");
  DeviceTables tb;
  SPRING_TRY(device_tables(&tb));
  int stale = 0;
  SPRING_TRY(take_device_status(&stale));  // start from a clear word
  k_wait_check<<<1, 32>>>(tb.status, cycles);
  SPRING_CHECK_LAUNCH();
  SPRING_CUDA(cudaDeviceSynchronize());
  return check_device_waits();
}

const char* spring_status_string(spring_status s) {
  switch (s) {
    case SPRING_OK: return "ok";
    case SPRING_E_INVALID: return "invalid argument";
    case SPRING_E_NOMEM: return "out of device memory or HBM budget";
    case SPRING_E_CUDA: return "CUDA error";
    case SPRING_E_BUSY: return "busy";
    case SPRING_E_TIMEOUT: return "timeout";
    case SPRING_E_NOT_FOUND: return "not found";
    case SPRING_E_NUMERIC: return "non-finite value in a reduction";
    case SPRING_E_CANCELLED: return "cancelled";
  }
  return "unknown status";
}

const char* spring_last_error(void) { return t_err.c_str(); }

void spring_stats_reset(void) {
  drain_pending();
  std::lock_guard<std::mutex> lk(g_tmu);
  for (auto& k : g_kstat) {
    k.launches = 0;
    k.timed = 0;
    k.total_ms = 0.0;
    k.timed_bytes = 0.0;
  }
  g_launches = 0;
}

void spring_stats_enable_timing(int on) { g_timing = on > 0 ? on : 0; }

void spring_stats_get(int kc, spring_kernel_stat* out) {
  if (!out) return;
  std::memset(out, 0, sizeof(*out));
  if (kc < 0 || kc >= SPRING_KC_COUNT) return;
  drain_pending();
  std::lock_guard<std::mutex> lk(g_tmu);
  out->launches = g_kstat[kc].launches;
  out->timed = g_kstat[kc].timed;
  out->total_ms = g_kstat[kc].total_ms;
  out->bytes_per_launch = out->timed ? g_kstat[kc].timed_bytes / (double)out->timed : g_kstat[kc].bytes;
}

uint64_t spring_launch_count(void) { return g_launches.load(); }

spring_status spring_fft2(void* data, int batch, int n, int inverse, void* stream) {
  SPRING_TRY(check_n(n, batch));
  if (!data && batch) return invalid("null data");
  float2* d = static_cast<float2*>(data);
  return fft2_unitary(n, inverse ? +1 : -1, d, d, nullptr, batch, ST(stream));
}

spring_status spring_project_modulus(const void* x, void* out, const float* M, int batch, int n,
                                     void* stream) {
  SPRING_TRY(check_n(n, batch));
  if (batch == 0) return SPRING_OK;
  if (!x || !out || !M) return invalid("null pointer");
  cudaStream_t s = ST(stream);
  float2* o = static_cast<float2*>(out);
  SPRING_TRY(launch_row_fft(n, -1, static_cast<const float2*>(x), o, nullptr, batch, 1.0f, s));
  SPRING_TRY(launch_col_pm(n, o, M, batch, s));
  return launch_row_fft(n, +1, o, o, nullptr, batch, 1.0f, s);
}

spring_status spring_iterate(void* x, const uint8_t* S, const float* M, int batch, int n,
                             int algorithm, float beta, float chi, int n_iter, void* stream) {
  SPRING_TRY(check_n(n, batch));
  if (algorithm < 0 || algorithm > 2) return invalid("algorithm must be 0, 1 or 2");
  if (n_iter < 0) return invalid("negative iteration count");
  if (batch == 0 || n_iter == 0) return SPRING_OK;
  if (!x || !S || !M) return invalid("null pointer");
  if (reinterpret_cast<uintptr_t>(x) & 15u) return invalid("x must be 16-byte aligned");
  cudaStream_t s = ST(stream);
  Scratch w;
  const size_t wbytes = sizeof(float2) * (size_t)batch * n * n, sbytes = ((size_t)batch * n * n / 8 + 255) & ~(size_t)255;
  const bool split = iteration_path(n) == 2;
  SPRING_TRY(w.alloc(wbytes + sbytes + (split ? sizeof(float) * (size_t)n * n : 0), s));
  uint32_t* Sb = reinterpret_cast<uint32_t*>(static_cast<char*>(w.p) + wbytes);
  SPRING_TRY(launch_pack_support(S, Sb, (long long)batch * n * n, s));
  float2* xs = static_cast<float2*>(x);
  if (split) {  // the split passes (sides 192-1024)
    float* Mp = reinterpret_cast<float*>(static_cast<char*>(w.p) + wbytes + sbytes);
    SPRING_TRY(launch_split_modulus(n, M, Mp, 1, s));
    SPRING_TRY(launch_row_split(n, algorithm, true, w.as<float2>(), xs, nullptr, batch, beta, chi, s));
    return iterate_split(n, algorithm, w.as<float2>(), xs, Sb, Mp, batch, 0, beta, chi, n_iter, s);
  }
  SPRING_TRY(launch_row_fft(n, -1, xs, w.as<float2>(), nullptr, batch, 1.0f, s));
  for (int it = 0; it < n_iter; ++it) {
    SPRING_TRY(launch_col_pm(n, w.as<float2>(), M, batch, s));
    SPRING_TRY(launch_row_iter(n, algorithm, w.as<float2>(), xs, Sb, batch, beta, chi,
                               it + 1 < n_iter, s));
  }
  return SPRING_OK;
}

spring_status spring_iterate_fused(void* x, const uint8_t* S, const float* M, int batch, int n,
                                   int algorithm, float beta, float chi, int n_iter, void* stream) {
  SPRING_TRY(check_n(n, batch));
  if (algorithm < 0 || algorithm > 2) return invalid("algorithm must be 0, 1 or 2");
  if (n_iter < 0) return invalid("negative iteration count");
  bool ok = false;
  SPRING_TRY(cluster_supported(n, &ok));
  if (!ok) return invalid("the on-chip iteration kernel does not cover this side on this device");
  if (batch == 0 || n_iter == 0) return SPRING_OK;
  if (!x || !S || !M) return invalid("null pointer");
  return launch_cluster_iter(n, algorithm, static_cast<float2*>(x), S, M, batch, beta, chi, n_iter, ST(stream));
}

spring_status spring_modulus_encode(const float* I, const uint8_t* mask, const uint8_t* sat, int n,
                                    const spring_bounds* b, float* M, void* stream) {
  SPRING_TRY(check_n(n, 1));
  if (!I || !mask || !M) return invalid("null pointer");
  if (b && b->eta > 0.f && !(b->max_missing >= 0.f && b->max_saturated >= 0.f && std::isfinite(b->eta)))
    return invalid("bounds: eta must be finite and the fractions >= 0");
  cudaStream_t s = ST(stream);
  Scratch ring;
  if (b && b->eta > 0.f) SPRING_TRY(ring.alloc(sizeof(double) * (size_t)ring_count(n), s));
  return launch_modulus_encode(n, I, mask, sat, b, ring.as<double>(), M, s);
}

spring_status spring_iterate_ex(void* x, const uint8_t* S, const float* M, int batch, int n,
                                int algorithm, float beta, float chi, int n_iter, int precision,
                                void* stream) {
  if (precision == 0) return spring_iterate(x, S, M, batch, n, algorithm, beta, chi, n_iter, stream);
  if (precision != 1) return invalid("precision must be 0 or 1");
  SPRING_TRY(check_n(n, batch));
  if (algorithm < 0 || algorithm > 2) return invalid("algorithm must be 0, 1 or 2");
  if (n_iter < 0) return invalid("negative iteration count");
  if (batch == 0 || n_iter == 0) return SPRING_OK;
  if (!x || !S || !M) return invalid("null pointer");
  cudaStream_t s = ST(stream);
  const long long total = (long long)batch * n * n;
  Scratch w;
  SPRING_TRY(w.alloc(sizeof(float2) * total + 256 + total / 8, s));
  void* wh = w.p;
  void* xh = static_cast<char*>(w.p) + total * 4;
  float* s16 = reinterpret_cast<float*>(static_cast<char*>(w.p) + total * 8);
  uint32_t* Sb = reinterpret_cast<uint32_t*>(static_cast<char*>(w.p) + total * 8 + 256);
  SPRING_TRY(launch_pack_support(S, Sb, total, s));
  float2* xs = static_cast<float2*>(x);
  SPRING_TRY(launch_fp16_scale(n, M, s16, s));
  SPRING_TRY(launch_row_init16(n, xs, xh, wh, batch, s16, s));
  for (int it = 0; it < n_iter; ++it) {
    SPRING_TRY(launch_col_pm16(n, wh, M, batch, s16, s));
    SPRING_TRY(launch_row_iter16(n, algorithm, wh, xh, Sb, batch, beta, chi, s16, s));
  }
  return launch_half_to_float(xh, xs, total, s16, s);
}

spring_status spring_smooth(const void* x, float* out, int batch, int n, float sigma, void* stream) {
  SPRING_TRY(check_n(n, batch));
  if (batch == 0) return SPRING_OK;
  if (!x || !out) return invalid("null pointer");
  cudaStream_t s = ST(stream);
  Scratch tmp;
  SPRING_TRY(tmp.alloc(sizeof(float) * (size_t)batch * n * n, s));
  return launch_smooth(n, static_cast<const float2*>(x), tmp.as<float>(), out, batch, sigma, nullptr, s);
}

spring_status spring_update_support(const void* x, uint8_t* S, int batch, int n, float sigma,
                                    float tau, void* stream) {
  SPRING_TRY(check_n(n, batch));
  if (batch == 0) return SPRING_OK;
  if (!x || !S) return invalid("null pointer");
  cudaStream_t s = ST(stream);
  const size_t nn = (size_t)n * n;
  Scratch tmp;
  SPRING_TRY(tmp.alloc(sizeof(float) * 2 * batch * nn + 256 + sizeof(unsigned) * batch, s));
  float* t0 = tmp.as<float>();
  float* t1 = t0 + batch * nn;
  unsigned* mx = reinterpret_cast<unsigned*>(t1 + batch * nn);
  SPRING_TRY(launch_smooth(n, static_cast<const float2*>(x), t0, t1, batch, sigma, mx, s));
  return launch_threshold(n, t1, mx, tau, S, batch, s);
}

spring_status spring_update_support_size(const void* x, uint8_t* S, int batch, int n, float sigma,
                                         const int64_t* alpha, void* stream) {
  SPRING_TRY(check_n(n, batch));
  if (batch == 0) return SPRING_OK;
  if (!x || !S || !alpha) return invalid("null pointer");
  cudaStream_t s = ST(stream);
  const size_t nn = (size_t)n * n;
  Scratch tmp;
  SPRING_TRY(tmp.alloc(sizeof(float) * 2 * batch * nn, s));
  float* t0 = tmp.as<float>();
  float* t1 = t0 + batch * nn;
  SPRING_TRY(launch_smooth(n, static_cast<const float2*>(x), t0, t1, batch, sigma, nullptr, s));
  return launch_select_area(n, t1, alpha, 1, S, batch, s, 1, t0);  // t0 is free after the smoothing
}

spring_status spring_fourier_error(const void* x, const uint8_t* S, const float* M, int batch, int n,
                                   double* err, void* stream) {
  SPRING_TRY(check_n(n, batch));
  if (batch == 0) return SPRING_OK;
  if (!x || !S || !M || !err) return invalid("null pointer");
  cudaStream_t s = ST(stream);
  const size_t nn = (size_t)n * n;
  const size_t part_bytes = sizeof(double) * 2 * (size_t)batch * err_strips(n);
  Scratch w;
  SPRING_TRY(w.alloc(sizeof(float2) * batch * nn + part_bytes, s));
  float2* wb = w.as<float2>();
  double* part = reinterpret_cast<double*>(wb + batch * nn);
  SPRING_TRY(launch_row_fft(n, -1, static_cast<const float2*>(x), wb, S, batch, 1.0f, s));
  SPRING_TRY(launch_col_err(n, wb, M, batch, part, s));
  return launch_err_finalize(n, part, batch, err, nullptr, s);
}

spring_status spring_area_stats(const uint8_t* S, const double* err, int P, int n, int g, int G,
                                int64_t* out, void* stream) {
  SPRING_TRY(check_n(n, P));
  if (P < 1 || !S || !out) return invalid("need P >= 1 and non-null S, out");
  cudaStream_t s = ST(stream);
  Scratch b;
  SPRING_TRY(b.alloc(sizeof(int32_t) * 4, s));
  SPRING_TRY(launch_argmin(err, P, b.as<int32_t>(), s));
  return launch_area_stats(n, S, b.as<int32_t>(), P, g, G, out, s);
}

spring_status spring_random_choice(uint64_t seed, int g, int P, int32_t* abc, void* stream) {
  if (!abc) return invalid("null pointer");
  return launch_random_choice(seed, g, P, abc, ST(stream));
}

spring_status spring_crossover_map(uint64_t seed, int g, int p, int n, int tile_min, int tile_max,
                                   float cp, uint8_t* map, void* stream) {
  SPRING_TRY(check_n(n, 1));
  if (!map) return invalid("null pointer");
  return launch_crossover_map(seed, g, p, n, tile_min, tile_max, cp, map, ST(stream));
}

// alignment of pairs (x[ix[q]] onto ref-spectrum index ir[q]) given spectra X of both
static spring_status align_pairs(int n, const float2* X, const int32_t* ix, const int32_t* ir,
                                 int npairs, const float* M, float2* A, float2* B, int32_t* info,
                                 float2* phasor, cudaStream_t s) {
  Scratch pk;
  SPRING_TRY(pk.alloc(peaks_scratch_bytes(n, npairs), s));
  SPRING_TRY(launch_xcorr_spectra(n, X, ix, ir, npairs, M, A, B, s));
  SPRING_TRY(fft2_unitary(n, +1, A, A, nullptr, npairs, s));
  SPRING_TRY(fft2_unitary(n, +1, B, B, nullptr, npairs, s));
  return launch_peaks(n, A, B, npairs, info, phasor, pk.p, s);
}

__global__ void k_iota_pairs(int n, int32_t* ix, int32_t* ir) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  ix[q] = q;
  ir[q] = n + q;
}

__global__ void k_phase_angle(const float2* ph, int n, float* out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) out[q] = atan2f(ph[q].y, ph[q].x);
}

spring_status spring_reshift(const void* x, const uint8_t* S, const void* ref, const float* M,
                             int batch, int n, void* x_out, uint8_t* S_out, int32_t* info,
                             float* phase, void* stream) {
  SPRING_TRY(check_n(n, batch));
  if (batch == 0) return SPRING_OK;
  if (!x || !ref || !M) return invalid("null pointer");
  if (S_out && !S) return invalid("S_out needs S");
  cudaStream_t s = ST(stream);
  const size_t nn = (size_t)n * n;
  // spectra of x (first batch images) and ref (next batch), correlations A, B
  Scratch w;
  const size_t img = sizeof(float2) * nn;
  SPRING_TRY(w.alloc(img * 4 * batch + sizeof(int32_t) * 5 * batch + sizeof(float2) * batch + 64, s));
  float2* X = w.as<float2>();
  float2* A = X + 2 * batch * nn;
  float2* B = A + batch * nn;
  int32_t* ix = reinterpret_cast<int32_t*>(B + batch * nn);
  int32_t* ir = ix + batch;
  int32_t* inf = ir + batch;
  float2* ph = reinterpret_cast<float2*>(inf + 3 * batch + (batch & 1));
  SPRING_TRY(fft2_unitary(n, -1, static_cast<const float2*>(x), X, nullptr, batch, s));
  SPRING_TRY(fft2_unitary(n, -1, static_cast<const float2*>(ref), X + batch * nn, nullptr, batch, s));
  launch_begin(SPRING_KC_OTHER, s);
  k_iota_pairs<<<div_up(batch, 128), 128, 0, s>>>(batch, ix, ir);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, 8.0 * batch);
  SPRING_TRY(align_pairs(n, X, ix, ir, batch, M, A, B, inf, ph, s));
  // ix as the source index of x: identity
  launch_begin(SPRING_KC_OTHER, s);
  k_iota_pairs<<<div_up(batch, 128), 128, 0, s>>>(batch, ix, ir);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, 8.0 * batch);
  SPRING_TRY(launch_apply_shift(n, static_cast<const float2*>(x), S, ix, batch, inf, ph,
                                static_cast<float2*>(x_out), S_out, s));
  if (info) SPRING_CUDA(cudaMemcpyAsync(info, inf, sizeof(int32_t) * 3 * batch, cudaMemcpyDeviceToDevice, s));
  if (phase) {
    launch_begin(SPRING_KC_OTHER, s);
    k_phase_angle<<<div_up(batch, 128), 128, 0, s>>>(ph, batch, phase);
    SPRING_CHECK_LAUNCH();
    launch_end(SPRING_KC_OTHER, s, 12.0 * batch);
  }
  return SPRING_OK;
}

spring_status spring_crossover(const void* pop_x, const uint8_t* pop_S, const float* M, int P, int n,
                               uint64_t seed, int g, float cw, float cp, int tile_min, int tile_max,
                               void* new_x, uint8_t* new_S, int32_t* parents, void* stream) {
  return spring_crossover_ca(pop_x, pop_S, M, P, n, seed, g, cw, cp, tile_min, tile_max, 0.0f, nullptr,
                             new_x, new_S, parents, stream);
}

spring_status spring_crossover_ca(const void* pop_x, const uint8_t* pop_S, const float* M, int P, int n,
                                  uint64_t seed, int g, float cw, float cp, int tile_min, int tile_max,
                                  float ca, const float* mavg, void* new_x, uint8_t* new_S, int32_t* parents,
                                  void* stream) {
  SPRING_TRY(check_n(n, P));
  if (P < 4) return invalid("population must be >= 4");
  if (!pop_x || !pop_S || !M || !new_x || !new_S) return invalid("null pointer");
  if (!(ca >= 0.f && ca <= 1.f)) return invalid("ca must be in [0, 1]");
  if (ca > 0.f && !mavg) return invalid("crossover averaging needs the average moduli");
  cudaStream_t s = ST(stream);
  const size_t nn = (size_t)n * n;
  Scratch w;
  const int Q = 3 * P;
  SPRING_TRY(w.alloc(sizeof(float2) * nn * (P + 2 * (size_t)P) + sizeof(int32_t) * (3 * Q + 3 * Q + 4) +
                         sizeof(float2) * Q + 64, s));
  float2* X = w.as<float2>();       // P spectra
  float2* A = X + P * nn;           // P correlation images per chunk
  float2* B = A + P * nn;
  int32_t* abc = reinterpret_cast<int32_t*>(B + P * nn);
  int32_t* ix = abc + Q;
  int32_t* ir = ix + Q;
  int32_t* inf = ir + Q;
  float2* ph = reinterpret_cast<float2*>(inf + 3 * Q + 2);
  SPRING_TRY(fft2_unitary(n, -1, static_cast<const float2*>(pop_x), X, nullptr, P, s));
  SPRING_TRY(launch_random_choice(seed, g, P, abc, s));
  SPRING_TRY(launch_pairs_crossover(P, abc, ix, ir, s));
  for (int c = 0; c < 3; ++c)
    SPRING_TRY(align_pairs(n, X, ix + c * P, ir + c * P, P, M, A, B, inf + 3 * c * P, ph + c * P, s));
  float2* nx = static_cast<float2*>(new_x);
  SPRING_TRY(launch_crossover_mix(n, X, abc, inf, ph, P, seed, g, cw, cp, tile_min, tile_max, ca, mavg, nx, s));
  SPRING_TRY(fft2_unitary(n, +1, nx, nx, nullptr, P, s));
  SPRING_TRY(launch_crossover_support(n, pop_S, abc, inf, P, new_S, s));
  if (parents) SPRING_CUDA(cudaMemcpyAsync(parents, abc, sizeof(int32_t) * Q, cudaMemcpyDeviceToDevice, s));
  return SPRING_OK;
}

spring_status spring_select(void* pop_x, uint8_t* pop_S, double* pop_err, const void* new_x,
                            const uint8_t* new_S, const double* new_err, int P, int n,
                            uint8_t* replaced, void* stream) {
  SPRING_TRY(check_n(n, P));
  if (P == 0) return SPRING_OK;
  if (!pop_x || !pop_S || !pop_err || !new_x || !new_S || !new_err) return invalid("null pointer");
  return launch_select(n, static_cast<float2*>(pop_x), pop_S, pop_err, static_cast<const float2*>(new_x),
                       new_S, new_err, P, replaced, ST(stream));
}

spring_status spring_average_moduli(const void* pop_x, const uint8_t* pop_S, const double* err, const float* M,
                                    int P, int n, float* mavg, void* stream) {
  SPRING_TRY(check_n(n, P));
  if (P < 1 || !pop_x || !pop_S || !M || !mavg) return invalid("null pointer or empty population");
  cudaStream_t s = ST(stream);
  const size_t nn = (size_t)n * n;
  Scratch w;
  SPRING_TRY(w.alloc(sizeof(float2) * nn * (3 * (size_t)P + 1) + nn + sizeof(int32_t) * (6 * P + 4) +
                         sizeof(float2) * P + 64, s));
  float2* X = w.as<float2>();
  float2* A = X + P * nn;
  float2* B = A + P * nn;
  float2* avg = B + P * nn;
  uint8_t* Savg = reinterpret_cast<uint8_t*>(avg + nn);
  int32_t* ix = reinterpret_cast<int32_t*>(Savg + nn + (4 - nn % 4) % 4);
  int32_t* ir = ix + P;
  int32_t* inf = ir + P;
  int32_t* best = inf + 3 * P;
  float2* ph = reinterpret_cast<float2*>(best + 2 + (P & 1));
  SPRING_TRY(fft2_unitary(n, -1, static_cast<const float2*>(pop_x), X, nullptr, P, s));
  SPRING_TRY(launch_argmin(err, P, best, s));
  SPRING_TRY(launch_pairs_onto_best(P, best, ix, ir, s));
  SPRING_TRY(align_pairs(n, X, ix, ir, P, M, A, B, inf, ph, s));
  SPRING_TRY(launch_average(n, static_cast<const float2*>(pop_x), pop_S, inf, ph, best, P, avg, Savg, s));
  SPRING_TRY(fft2_unitary(n, -1, avg, avg, nullptr, 1, s));
  return launch_average_moduli(n, X, avg, P, mavg, s);
}

spring_status spring_average(const void* pop_x, const uint8_t* pop_S, const double* err, const float* M,
                             int P, int n, void* avg, uint8_t* S_avg, void* stream) {
  SPRING_TRY(check_n(n, P));
  if (P < 1 || !pop_x || !pop_S || !M || !avg || !S_avg) return invalid("null pointer or empty population");
  cudaStream_t s = ST(stream);
  const size_t nn = (size_t)n * n;
  Scratch w;
  SPRING_TRY(w.alloc(sizeof(float2) * nn * 3 * P + sizeof(int32_t) * (6 * P + 4) + sizeof(float2) * P + 64, s));
  float2* X = w.as<float2>();
  float2* A = X + P * nn;
  float2* B = A + P * nn;
  int32_t* ix = reinterpret_cast<int32_t*>(B + P * nn);
  int32_t* ir = ix + P;
  int32_t* inf = ir + P;
  int32_t* best = inf + 3 * P;
  float2* ph = reinterpret_cast<float2*>(best + 2 + (P & 1));
  SPRING_TRY(fft2_unitary(n, -1, static_cast<const float2*>(pop_x), X, nullptr, P, s));
  SPRING_TRY(launch_argmin(err, P, best, s));
  SPRING_TRY(launch_pairs_onto_best(P, best, ix, ir, s));
  SPRING_TRY(align_pairs(n, X, ix, ir, P, M, A, B, inf, ph, s));
  return launch_average(n, static_cast<const float2*>(pop_x), pop_S, inf, ph, best, P,
                        static_cast<float2*>(avg), S_avg, s);
}

spring_status spring_initialize(uint64_t seed, const uint8_t* S0, const float* M, int n, int P,
                                int n_spheres, float gamma, float phi_max, void* x, void* stream) {
  SPRING_TRY(check_n(n, P));
  if (P == 0) return SPRING_OK;
  if (!S0 || !M || !x) return invalid("null pointer");
  if (!(gamma > 0.f)) return invalid("init_gamma must be > 0");
  cudaStream_t s = ST(stream);
  const size_t nn = (size_t)n * n;
  Scratch w;
  const size_t a = sizeof(float2) * nn * P, b = normalise_scratch_bytes(P), c = init_scratch_bytes(P, n_spheres);
  SPRING_TRY(w.alloc(a + b + c + 256, s));
  float2* X = w.as<float2>();
  double* part = reinterpret_cast<double*>(reinterpret_cast<char*>(w.p) + a);
  void* isc = reinterpret_cast<char*>(w.p) + a + b + 128;
  float2* xs = static_cast<float2*>(x);
  SPRING_TRY(launch_init_spheres(n, seed, S0, P, n_spheres, gamma, phi_max, xs, isc, s));
  SPRING_TRY(fft2_unitary(n, -1, xs, X, nullptr, P, s));
  return launch_normalise(n, X, M, P, xs, part, s);
}

}  // extern "C"
