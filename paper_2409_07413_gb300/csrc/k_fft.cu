// k_fft.cu -- launchers of the transform passes, the kernel-variant table and its
// autotuner.  The kernels themselves are in k_fft.cuh (one instantiation unit per side).
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <mutex>
#include <string>

#include "k_fft.cuh"

namespace spring {

extern template spring_status run_fft_op<64>(const FftOp&, cudaStream_t, bool);
extern template spring_status run_fft_op<96>(const FftOp&, cudaStream_t, bool);
extern template spring_status run_fft_op<128>(const FftOp&, cudaStream_t, bool);
extern template spring_status run_fft_op<192>(const FftOp&, cudaStream_t, bool);
extern template spring_status run_fft_op<256>(const FftOp&, cudaStream_t, bool);
extern template spring_status run_fft_op<384>(const FftOp&, cudaStream_t, bool);
extern template spring_status run_fft_op<512>(const FftOp&, cudaStream_t, bool);
extern template spring_status run_fft_op<768>(const FftOp&, cudaStream_t, bool);
extern template spring_status run_fft_op<1024>(const FftOp&, cudaStream_t, bool);

static spring_status prepare_once(int n);

static spring_status dispatch(int n, const FftOp& op, cudaStream_t s, bool prep = false) {
  if (!prep) SPRING_TRY(prepare_once(n));
  switch (n) {
    case 64: return run_fft_op<64>(op, s, prep);
    case 96: return run_fft_op<96>(op, s, prep);
    case 128: return run_fft_op<128>(op, s, prep);
    case 192: return run_fft_op<192>(op, s, prep);
    case 256: return run_fft_op<256>(op, s, prep);
    case 384: return run_fft_op<384>(op, s, prep);
    case 512: return run_fft_op<512>(op, s, prep);
    case 768: return run_fft_op<768>(op, s, prep);
    case 1024: return run_fft_op<1024>(op, s, prep);
  }
  return invalid("unsupported pattern side " + std::to_string(n));
}

static int side_index(int n) { return side_slot(n); }

// ------------------------------------------------------------------ variant table
// Launch-shape variants of the two per-iteration passes, per side (see k_fft.cuh); the
// defaults are the fastest measured on a GB300 at 33.5 M pixels per launch.
static std::mutex g_var_mu;
// (sides 64, 96, 128, 192, 256, 384, 512, 768, 1024)
static int g_row_var[N_SIDES] = {0, 6, 5, 6, 0, 6, 6, 6, 5};
static int g_col_var[N_SIDES] = {0, 1, 2, 1, 0, 0, 0, 1, 1};
static bool g_tuned[N_SIDES] = {};
// iteration path per side: 0 = the two passes through HBM, 1 = the on-chip cluster kernel
// (N <= 256, k_cluster.cu), 2 = the split passes (N = 192, 384, 512, 768, 1024: the column
// transform's first radix-Q stage in the row pass); chosen by the autotuner, until then the
// fastest measured on a GB300 (the split passes at all five)
static int g_path[N_SIDES] = {0, 0, 0, 2, 0, 2, 2, 2, 2};

int iteration_path(int n) {
  const int si = side_index(n);
  if (si < 0) return 0;
  std::lock_guard<std::mutex> lk(g_var_mu);
  return g_path[si];
}

static int row_variant(int n) {
  std::lock_guard<std::mutex> lk(g_var_mu);
  return g_row_var[side_index(n)];
}
static int col_variant_of(int n) {
  std::lock_guard<std::mutex> lk(g_var_mu);
  return g_col_var[side_index(n)];
}

// ------------------------------------------------------------------ launchers
spring_status launch_row_iter(int n, int alg, float2* w, float2* x, const uint32_t* Sb, long long batch,
                              float beta, float chi, bool zout, cudaStream_t s) {
  if (alg < 0 || alg > 2) return invalid("algorithm must be 0 (ER), 1 (HIO) or 2 (RAAR)");
  if (side_index(n) < 0) return invalid("unsupported pattern side");
  DeviceTables tb;
  SPRING_TRY(device_tables(&tb));
  FftOp op;
  op.kind = OP_ROW_ITER;
  op.alg = alg;
  op.variant = row_variant(n);
  op.kclass = SPRING_KC_ROW_ITER;
  op.ra.in = w;
  op.ra.out = w;
  op.ra.x = x;
  op.ra.Sb = Sb;
  op.ra.tw = tb.tw + tw_offset(n);
  op.ra.nrows = batch * n;
  op.ra.beta = beta;
  op.ra.chi_on = chi < 1.0f;
  op.ra.cchi = (float)((chi == 0.5f) ? 0.0 : std::cos((double)chi * 3.14159265358979323846));
  op.ra.zout = zout ? 1 : 0;
  // algorithmic bytes: w in, x_n in (not for ER), x_{n+1} out, w out, and the support bits
  op.bytes = (double)batch * n * n * (8.0 + (alg ? 8.0 : 0.0) + 8.0 + (zout ? 8.0 : 0.0) + 0.125);
  return dispatch(n, op, s);
}

spring_status launch_row_fft_tw(int n, int dir, const float2* in, float2* out, const uint8_t* Smul,
                                long long batch, float scale, const float2* tw_all, cudaStream_t s) {
  FftOp op;
  op.kind = dir < 0 ? OP_ROW_FWD : OP_ROW_INV;
  op.ra.in = in;
  op.ra.out = out;
  op.ra.S = Smul;
  op.ra.tw = tw_all + tw_offset(n);
  op.ra.nrows = batch * n;
  op.ra.scale = scale;
  op.bytes = (double)batch * n * n * (16.0 + (Smul ? 1.0 : 0.0));
  return dispatch(n, op, s);
}

spring_status launch_row_fft(int n, int dir, const float2* in, float2* out, const uint8_t* Smul,
                             long long batch, float scale, cudaStream_t s) {
  DeviceTables tb;
  SPRING_TRY(device_tables(&tb));
  return launch_row_fft_tw(n, dir, in, out, Smul, batch, scale, tb.tw, s);
}

spring_status launch_col_pm(int n, float2* w, const float* M, int batch, cudaStream_t s, int m_group, int img0) {
  if (side_index(n) < 0) return invalid("unsupported pattern side");
  DeviceTables tb;
  SPRING_TRY(device_tables(&tb));
  FftOp op;
  op.kind = OP_COL_PM;
  op.variant = col_variant_of(n);
  op.kclass = SPRING_KC_COL_PM;
  op.ca.data = w;
  op.ca.M = M;
  op.ca.tw = tb.tw + tw_offset(n);
  op.ca.batch = batch;
  op.ca.m_group = m_group;
  op.ca.img0 = img0;
  const double nm = m_group > 0 ? (double)((batch + m_group - 1) / m_group) : 1.0;
  op.bytes = (double)batch * n * n * 16.0 + nm * n * n * 4.0;
  return dispatch(n, op, s);
}

spring_status launch_col_fft(int n, int dir, float2* data, int batch, float scale, cudaStream_t s) {
  DeviceTables tb;
  SPRING_TRY(device_tables(&tb));
  FftOp op;
  op.kind = dir < 0 ? OP_COL_FWD : OP_COL_INV;
  op.ca.data = data;
  op.ca.tw = tb.tw + tw_offset(n);
  op.ca.batch = batch;
  op.ca.scale = scale;
  op.bytes = (double)batch * n * n * 16.0;
  return dispatch(n, op, s);
}

int err_strips(int n) { return n / ERR_W; }

spring_status launch_col_err_tw(int n, float2* w, const float* M, int batch, double* partials,
                                const float2* tw_all, cudaStream_t s, int m_group, bool skip_m2) {
  FftOp op;
  op.kind = OP_COL_ERR;
  op.ca.data = w;
  op.ca.M = M;
  op.ca.tw = tw_all + tw_offset(n);
  op.ca.batch = batch;
  op.ca.partials = partials;
  op.ca.m_group = m_group;
  op.ca.skip_m2 = skip_m2 ? 1 : 0;
  op.bytes = (double)batch * n * n * 8.0 + (double)n * n * 4.0;
  return dispatch(n, op, s);
}

spring_status launch_col_err(int n, float2* w, const float* M, int batch, double* partials,
                             cudaStream_t s, int m_group, bool skip_m2) {
  DeviceTables tb;
  SPRING_TRY(device_tables(&tb));
  return launch_col_err_tw(n, w, M, batch, partials, tb.tw, s, m_group, skip_m2);
}

__global__ void k_err_finalize(const double* __restrict__ partials, int strips, int batch,
                               double* __restrict__ err, int* __restrict__ status,
                               const double* __restrict__ m2, int m_group) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  double sn = 0.0, sd = 0.0;
  for (int s = 0; s < strips; ++s) {
    sn += partials[((size_t)b * strips + s) * 2 + 0];
    if (!m2) sd += partials[((size_t)b * strips + s) * 2 + 1];
  }
  if (m2) sd = m2[m_group > 0 ? b / m_group : 0];
  const double e = sd > 0.0 ? sqrt(sn / sd) : 0.0;
  if (!isfinite(e) && status) atomicOr(status, 1);
  err[b] = e;
}

spring_status launch_err_finalize(int n, const double* partials, int batch, double* err,
                                  int* status, cudaStream_t s, const double* m2, int m_group) {
  if (batch < 1) return SPRING_OK;
  launch_begin(SPRING_KC_OTHER, s);
  k_err_finalize<<<div_up(batch, 128), 128, 0, s>>>(partials, n / ERR_W, batch, err, status, m2, m_group);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, 16.0 * batch * (n / ERR_W));
  return SPRING_OK;
}

// The denominator of Eq. error_calc, sum of M^2 over the measured pixels, depends on the
// pattern only: one block per modulus array, FP64 partial sums per thread in a fixed
// order, then a fixed-order block reduction.
__global__ void k_m2_sum(const float* __restrict__ M, long long nn, double* __restrict__ m2) {
  const float* Mk = M + (size_t)blockIdx.x * nn;
  double acc = 0.0;
  for (long long i = threadIdx.x; i < nn; i += blockDim.x) {
    const float v = Mk[i];
    if (v >= 0.f) acc += (double)v * (double)v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  __shared__ double red[32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    m2[blockIdx.x] = t;
  }
}

spring_status launch_m2_sum(int n, const float* M, int K, double* m2, cudaStream_t s) {
  if (K < 1) return SPRING_OK;
  launch_begin(SPRING_KC_OTHER, s);
  k_m2_sum<<<K, 1024, 0, s>>>(M, (long long)n * n, m2);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, 4.0 * K * n * n);
  return SPRING_OK;
}

// ------------------------------------------------------------------ FP16 storage (precision 1)
// s16 = 2^e with sqrt(N) ||M||_2 w16_scale(N) 2^e in [2^12, 2^13).  For any row r and
// frequency k, |rowFFT(x)_rk| <= sum_j |x_rj| <= sqrt(N) ||x||_2, and the iterates keep
// ||x||_2 near ||M||_2 (P_M maps onto the measured norm), so every stored FP16 value stays
// about 8x below its largest finite value; the same power of two keeps small intensity
// scales away from the subnormal range.  One block; a fixed-order FP64 sum.
__global__ void k_fp16_scale(const float* __restrict__ M, int n, float* __restrict__ out) {
  __shared__ double part[256];
  double acc = 0.0;
  const long long nn = (long long)n * n;
  for (long long i = threadIdx.x; i < nn; i += blockDim.x) {
    const double m = M[i];
    if (m > 0.0) acc += m * m;
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) part[threadIdx.x] += part[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double v = sqrt((double)n) * sqrt(part[0]) * (double)w16_scale(n);
    int k = 0;
    float sc = 1.0f;
    if (v > 0.0 && isfinite(v)) {
      frexp(v, &k);  // v = f 2^k, f in [0.5, 1)
      const int e = max(-120, min(120, 13 - k));
      sc = ldexpf(1.0f, e);
    }
    *out = sc;
  }
}

spring_status launch_fp16_scale(int n, const float* M, float* s16, cudaStream_t s) {
  launch_begin(SPRING_KC_OTHER, s);
  k_fp16_scale<<<1, 256, 0, s>>>(M, n, s16);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, (double)n * n * 4.0);
  return SPRING_OK;
}

spring_status launch_row_iter16(int n, int alg, void* wh, void* xh, const uint32_t* Sb, long long batch,
                                float beta, float chi, const float* s16, cudaStream_t s) {
  if (alg < 0 || alg > 2) return invalid("algorithm must be 0 (ER), 1 (HIO) or 2 (RAAR)");
  DeviceTables tb;
  SPRING_TRY(device_tables(&tb));
  FftOp op;
  op.kind = OP_ROW_ITER16;
  op.alg = alg;
  op.kclass = SPRING_KC_ROW_ITER;
  op.ra.in = static_cast<const float2*>(wh);
  op.ra.out = static_cast<float2*>(wh);
  op.ra.x = static_cast<float2*>(xh);
  op.ra.Sb = Sb;
  op.ra.tw = tb.tw + tw_offset(n);
  op.ra.nrows = batch * n;
  op.ra.beta = beta;
  op.ra.chi_on = chi < 1.0f;
  op.ra.cchi = (float)((chi == 0.5f) ? 0.0 : std::cos((double)chi * 3.14159265358979323846));
  op.ra.zout = 1;
  op.ra.s16 = s16;
  op.bytes = (double)batch * n * n * (4.0 + (alg ? 4.0 : 0.0) + 4.0 + 4.0 + 0.125);  // support: 1 bit/px
  return dispatch(n, op, s);
}

spring_status launch_col_pm16(int n, void* wh, const float* M, int batch, const float* s16, cudaStream_t s) {
  DeviceTables tb;
  SPRING_TRY(device_tables(&tb));
  FftOp op;
  op.kind = OP_COL_PM16;
  op.kclass = SPRING_KC_COL_PM;
  op.ca.data = static_cast<float2*>(wh);
  op.ca.M = M;
  op.ca.tw = tb.tw + tw_offset(n);
  op.ca.batch = batch;
  op.ca.s16 = s16;
  op.bytes = (double)batch * n * n * 8.0 + (double)n * n * 4.0;
  return dispatch(n, op, s);
}

spring_status launch_row_init16(int n, const float2* x, void* xh, void* wh, long long batch, const float* s16,
                                cudaStream_t s) {
  DeviceTables tb;
  SPRING_TRY(device_tables(&tb));
  FftOp op;
  op.kind = OP_ROW_INIT16;
  op.ra.in = x;
  op.ra.out = static_cast<float2*>(wh);
  op.ra.xh = xh;
  op.ra.tw = tb.tw + tw_offset(n);
  op.ra.nrows = batch * n;
  op.ra.s16 = s16;
  op.bytes = (double)batch * n * n * 16.0;
  return dispatch(n, op, s);
}

// ------------------------------------------------------------------ split passes (N = 192, 384, 512, 768, 1024)
bool split_supported(int n) { return split_side(n); }

// the modulus in the split column pass's chunked layout: row k2 L + k1 of Mp is row
// Q k1 + k2 of M (K arrays of n x n)
__global__ void k_split_modulus(const float* __restrict__ M, float* __restrict__ Mp, int n, int Q, long long total) {
  const int L = n / Q;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long nn = (long long)n * n, q = i / nn, r = (i / n) % n, c = i % n;
    const long long k2 = r / L, k1 = r % L;
    Mp[i] = M[q * nn + (Q * k1 + k2) * n + c];
  }
}

spring_status launch_split_modulus(int n, const float* M, float* Mp, int K, cudaStream_t s) {
  if (!split_side(n)) return invalid("the split passes cover sides 192, 384, 512, 768 and 1024");
  const long long total = (long long)K * n * n;
  const long long blocks = div_up(total, 256) < 16LL * sm_count() ? div_up(total, 256) : 16LL * sm_count();
  launch_begin(SPRING_KC_OTHER, s);
  k_split_modulus<<<(int)blocks, 256, 0, s>>>(M, Mp, n, split_q_of(n), total);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, (double)total * 8.0);
  return SPRING_OK;
}

// the split row pass: fwd_only = the forward row transforms and first stage from x alone
spring_status launch_row_split(int n, int alg, bool fwd_only, float2* w, float2* x, const uint32_t* Sb,
                               long long batch, float beta, float chi, cudaStream_t s) {
  if (!split_side(n)) return invalid("the split passes cover sides 192, 384, 512, 768 and 1024");
  if (alg < 0 || alg > 2) return invalid("algorithm must be 0 (ER), 1 (HIO) or 2 (RAAR)");
  DeviceTables tb;
  SPRING_TRY(device_tables(&tb));
  FftOp op;
  op.kind = fwd_only ? OP_ROW_SPLIT_FWD : OP_ROW_SPLIT;
  op.alg = alg;
  op.kclass = fwd_only ? SPRING_KC_OTHER : SPRING_KC_ROW_ITER;
  op.sa.w = w;
  op.sa.x = x;
  op.sa.Sb = Sb;
  op.sa.tw = tb.tw + tw_offset(n);
  op.sa.nsets = batch * (n / split_q_of(n));
  op.sa.beta = beta;
  op.sa.chi_on = chi < 1.0f;
  op.sa.cchi = (float)((chi == 0.5f) ? 0.0 : std::cos((double)chi * 3.14159265358979323846));
  op.bytes = fwd_only ? (double)batch * n * n * 16.0
                      : (double)batch * n * n * (8.0 + (alg ? 8.0 : 0.0) + 16.0 + 0.125);
  return dispatch(n, op, s);
}

spring_status launch_col_split(int n, float2* w, const float* Mp, int batch, cudaStream_t s, int m_group) {
  if (!split_side(n)) return invalid("the split passes cover sides 192, 384, 512, 768 and 1024");
  DeviceTables tb;
  SPRING_TRY(device_tables(&tb));
  FftOp op;
  op.kind = OP_COL_SPLIT;
  op.kclass = SPRING_KC_COL_PM;
  op.ca.data = w;
  op.ca.M = Mp;
  op.ca.tw = tb.tw + tw_offset(n / split_q_of(n));
  op.ca.batch = batch;
  op.ca.m_group = m_group;
  const double nm = m_group > 0 ? (double)((batch + m_group - 1) / m_group) : 1.0;
  op.bytes = (double)batch * n * n * 16.0 + nm * n * n * 4.0;
  return dispatch(n, op, s);
}

// k iterations (column pass, then row pass) in the split form; w must hold the chunked
// forward spectra of x (launch_row_split with fwd_only) on entry and holds them on exit
spring_status iterate_split(int n, int alg, float2* w, float2* x, const uint32_t* Sb, const float* Mp,
                            long long batch, int m_group, float beta, float chi, int k, cudaStream_t s) {
  if (batch > INT32_MAX) return invalid("batch too large");
  for (int it = 0; it < k; ++it) {
    SPRING_TRY(launch_col_split(n, w, Mp, (int)batch, s, m_group));
    SPRING_TRY(launch_row_split(n, alg, false, w, x, Sb, batch, beta, chi, s));
  }
  return SPRING_OK;
}

// Supports to one bit per pixel: thread k packs pixels 32k .. 32k + 31 (two 16-byte loads)
// into word k, pixel 32k + b at bit b.  npix is a multiple of 32 (every supported N^2 is).
template <bool ALIGNED>
__global__ void k_pack_support(const uint8_t* __restrict__ S, uint32_t* __restrict__ Sb, long long nwords) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < nwords;
       k += (long long)gridDim.x * blockDim.x) {
    uint32_t wbits = 0u;
    if constexpr (ALIGNED) {
      const uint4 lo = *reinterpret_cast<const uint4*>(S + 32 * k);
      const uint4 hi = *reinterpret_cast<const uint4*>(S + 32 * k + 16);
      const uint32_t q[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int b = 0; b < 4; ++b) wbits |= (((q[i] >> (8 * b)) & 0xffu) != 0u ? 1u : 0u) << (4 * i + b);
    } else {  // a support array that does not start on a 16-byte boundary
#pragma unroll 4
      for (int b = 0; b < 32; ++b) wbits |= (S[32 * k + b] != 0 ? 1u : 0u) << b;
    }
    Sb[k] = wbits;
  }
}

spring_status launch_pack_support(const uint8_t* S, uint32_t* Sb, long long npix, cudaStream_t s) {
  if (npix % 32) return invalid("support size must be a multiple of 32 pixels");
  const long long nw = npix / 32;
  if (nw < 1) return SPRING_OK;
  const long long blocks = div_up(nw, 256) < 16LL * sm_count() ? div_up(nw, 256) : 16LL * sm_count();
  launch_begin(SPRING_KC_OTHER, s);
  if ((reinterpret_cast<uintptr_t>(S) & 15u) == 0)
    k_pack_support<true><<<(int)blocks, 256, 0, s>>>(S, Sb, nw);
  else
    k_pack_support<false><<<(int)blocks, 256, 0, s>>>(S, Sb, nw);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, (double)npix * 1.125);
  return SPRING_OK;
}

__global__ void k_half_to_float(const __half2* __restrict__ xh, float2* __restrict__ x, long long total,
                                const float* __restrict__ s16) {
  const float isx = 1.0f / __ldg(s16);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 v = __half22float2(xh[i]);
    x[i] = make_float2(v.x * isx, v.y * isx);
  }
}

spring_status launch_half_to_float(const void* xh, float2* x, long long total, const float* s16, cudaStream_t s) {
  if (total < 1) return SPRING_OK;
  launch_begin(SPRING_KC_OTHER, s);
  k_half_to_float<<<div_up(total, 256) < 16 * sm_count() ? div_up(total, 256) : 16 * sm_count(), 256, 0, s>>>(
      static_cast<const __half2*>(xh), x, total, s16);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, (double)total * 12.0);
  return SPRING_OK;
}

// Raise the dynamic shared-memory limit of every transform kernel of side N once, before
// any launch (and so before any stream capture).
spring_status prepare_fft_kernels(int n) {
  if (side_index(n) < 0) return invalid("unsupported pattern side");
  FftOp op;
  const int last_kind = split_side(n) ? OP_COL_SPLIT : OP_ROW_INIT16;
  for (int kind = OP_ROW_ITER; kind <= last_kind; ++kind) {
    op.kind = kind;
    const int nv = kind == OP_ROW_ITER ? ROW_VARIANTS : kind == OP_COL_PM ? COL_VARIANTS : 1;
    const bool algs = kind == OP_ROW_ITER || kind == OP_ROW_ITER16 || kind == OP_ROW_SPLIT;
    for (int v = 0; v < nv; ++v)
      for (int alg = 0; alg < (algs ? 3 : 1); ++alg) {
        op.variant = v;
        op.alg = alg;
        SPRING_TRY(dispatch(n, op, nullptr, true));
      }
  }
  SPRING_TRY(prepare_cluster_kernels(n));
  SPRING_CHECK_LAUNCH();
  return SPRING_OK;
}

// once per device and side, before the first launch of that side
static std::atomic<unsigned> g_prepared[64];

static spring_status prepare_once(int n) {
  int dev = 0;
  SPRING_CUDA(cudaGetDevice(&dev));
  const int si = side_index(n);
  if (dev < 0 || dev >= 64 || si < 0) return invalid("device or side out of range");
  const unsigned bit = 1u << si;
  if (g_prepared[dev].load(std::memory_order_acquire) & bit) return SPRING_OK;
  SPRING_TRY(prepare_fft_kernels(n));
  g_prepared[dev].fetch_or(bit, std::memory_order_acq_rel);
  return SPRING_OK;
}

// ------------------------------------------------------------------ autotuner
__global__ void k_fill_state(float2* x, uint8_t* S, float* M, long long total, long long nn) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  uint32_t r[4];
  philox4x32_10((uint32_t)i, (uint32_t)(i >> 32), 0x7475u, 0u, 0x12345678u, 0x9abcdef0u, r);
  x[i] = make_float2((float)(int)r[0] * 4.6566e-10f, (float)(int)r[1] * 4.6566e-10f);
  S[i] = (r[2] & 3u) == 0u;
  if (i < nn) M[i] = (r[3] & 31u) == 0u ? -1.0f : 0.1f + (float)(r[3] >> 8) * 5.96e-8f;
}

static spring_status time_op(int n, const FftOp& op, cudaStream_t s, int reps, float* ms) {
  cudaEvent_t a, b;
  SPRING_CUDA(cudaEventCreate(&a));
  SPRING_CUDA(cudaEventCreate(&b));
  spring_status st = dispatch(n, op, s);  // warm-up
  if (st == SPRING_OK) {
    cudaEventRecord(a, s);
    for (int r = 0; r < reps && st == SPRING_OK; ++r) st = dispatch(n, op, s);
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    cudaEventElapsedTime(ms, a, b);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return st;
}

// Time every variant of the two per-iteration passes on `batch` images of side n (scratch
// state, RAAR) and keep the fastest.  Call outside stream capture.
spring_status autotune_n(int n, int batch, cudaStream_t s) {
  const int si = side_index(n);
  if (si < 0) return invalid("unsupported pattern side");
  if (batch < 1) return invalid("batch must be >= 1");
  SPRING_TRY(prepare_fft_kernels(n));
  DeviceTables tb;
  SPRING_TRY(device_tables(&tb));
  const long long nn = (long long)n * n, total = nn * batch;
  Scratch buf;
  SPRING_TRY(buf.alloc(total * (2 * sizeof(float2) + 1) + nn * sizeof(float) + 1024, s));
  float2* x = buf.as<float2>();
  float2* w = x + total;
  float* M = reinterpret_cast<float*>(w + total);
  uint8_t* S = reinterpret_cast<uint8_t*>(M + nn);
  k_fill_state<<<div_up(total, 256), 256, 0, s>>>(x, S, M, total, nn);
  SPRING_CHECK_LAUNCH();
  Scratch bits;
  SPRING_TRY(bits.alloc(sizeof(uint32_t) * (size_t)(total / 32 + 1), s));
  SPRING_TRY(launch_pack_support(S, bits.as<uint32_t>(), total, s));
  SPRING_CUDA(cudaMemcpyAsync(w, x, sizeof(float2) * total, cudaMemcpyDeviceToDevice, s));
  FftOp op;
  op.kind = OP_ROW_ITER;
  op.alg = 2;
  op.ra.in = w;
  op.ra.out = w;
  op.ra.x = x;
  op.ra.Sb = bits.as<uint32_t>();
  op.ra.tw = tb.tw + tw_offset(n);
  op.ra.nrows = (long long)batch * n;
  op.ra.beta = 0.9f;
  op.ra.chi_on = 1;
  op.ra.cchi = 0.f;
  op.ra.zout = 1;
  const int reps = 4;
  int best_r = 0;
  float best_ms = 1e30f;
  for (int v = 0; v < ROW_VARIANTS; ++v) {
    op.variant = v;
    float ms = 0.f;
    SPRING_TRY(time_op(n, op, s, reps, &ms));
    if (ms < best_ms) {
      best_ms = ms;
      best_r = v;
    }
  }
  FftOp cop;
  cop.kind = OP_COL_PM;
  cop.ca.data = w;
  cop.ca.M = M;
  cop.ca.tw = tb.tw + tw_offset(n);
  cop.ca.batch = batch;
  int best_c = 0;
  best_ms = 1e30f;
  for (int v = 0; v < COL_VARIANTS; ++v) {
    cop.variant = v;
    float ms = 0.f;
    SPRING_TRY(time_op(n, cop, s, reps, &ms));
    if (ms < best_ms) {
      best_ms = ms;
      best_c = v;
    }
  }
  // the on-chip path against the two passes with the chosen variants, over one block of
  // 20 iterations
  int path = 0;
  bool fused_ok = false;
  SPRING_TRY(cluster_supported(n, &fused_ok));
  if (fused_ok) {
    constexpr int K = 20;
    op.variant = best_r;
    cop.variant = best_c;
    cudaEvent_t e0, e1, e2;
    SPRING_CUDA(cudaEventCreate(&e0));
    SPRING_CUDA(cudaEventCreate(&e1));
    SPRING_CUDA(cudaEventCreate(&e2));
    spring_status st = launch_cluster_iter(n, 2, x, S, M, batch, 0.9f, 0.5f, K, s);  // warm-up
    if (st == SPRING_OK) st = dispatch(n, cop, s);
    if (st == SPRING_OK) st = dispatch(n, op, s);
    cudaEventRecord(e0, s);
    for (int k = 0; k < K && st == SPRING_OK; ++k) {
      st = dispatch(n, cop, s);
      if (st == SPRING_OK) st = dispatch(n, op, s);
    }
    cudaEventRecord(e1, s);
    if (st == SPRING_OK) st = launch_cluster_iter(n, 2, x, S, M, batch, 0.9f, 0.5f, K, s);
    cudaEventRecord(e2, s);
    cudaEventSynchronize(e2);
    float two = 0.f, one = 0.f;
    cudaEventElapsedTime(&two, e0, e1);
    cudaEventElapsedTime(&one, e1, e2);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    SPRING_TRY(st);
    path = one < two ? 1 : 0;
  }
  // the split passes (N = 192-1024) against the two passes with the chosen variants over a
  // block of 20 iterations
  if (split_side(n)) {
    constexpr int K = 20;
    op.variant = best_r;
    cop.variant = best_c;
    Scratch mp;
    SPRING_TRY(mp.alloc(sizeof(float) * nn, s));
    SPRING_TRY(launch_split_modulus(n, M, mp.as<float>(), 1, s));
    cudaEvent_t e0, e1, e2;
    SPRING_CUDA(cudaEventCreate(&e0));
    SPRING_CUDA(cudaEventCreate(&e1));
    SPRING_CUDA(cudaEventCreate(&e2));
    spring_status st = dispatch(n, cop, s);  // warm-up of both forms
    if (st == SPRING_OK) st = dispatch(n, op, s);
    if (st == SPRING_OK) st = launch_row_split(n, 2, true, w, x, nullptr, batch, 0.9f, 0.5f, s);
    if (st == SPRING_OK) st = iterate_split(n, 2, w, x, bits.as<uint32_t>(), mp.as<float>(), batch, 0, 0.9f, 0.5f, 1, s);
    cudaEventRecord(e0, s);
    for (int k = 0; k < K && st == SPRING_OK; ++k) {
      st = dispatch(n, cop, s);
      if (st == SPRING_OK) st = dispatch(n, op, s);
    }
    cudaEventRecord(e1, s);
    if (st == SPRING_OK) st = iterate_split(n, 2, w, x, bits.as<uint32_t>(), mp.as<float>(), batch, 0, 0.9f, 0.5f, K, s);
    cudaEventRecord(e2, s);
    cudaEventSynchronize(e2);
    float two = 0.f, split = 0.f;
    cudaEventElapsedTime(&two, e0, e1);
    cudaEventElapsedTime(&split, e1, e2);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    SPRING_TRY(st);
    if (split < two) path = 2;
  }
  std::lock_guard<std::mutex> lk(g_var_mu);
  g_row_var[si] = best_r;
  g_col_var[si] = best_c;
  g_path[si] = path;
  g_tuned[si] = true;
  return SPRING_OK;
}

static bool autotune_enabled() {
  const char* e = std::getenv("SPRING_AUTOTUNE");
  return !(e && e[0] == '0');
}

// once per side and process, unless disabled or set explicitly
spring_status ensure_tuned(int n, int batch, cudaStream_t s) {
  const int si = side_index(n);
  if (si < 0) return invalid("unsupported pattern side");
  {
    std::lock_guard<std::mutex> lk(g_var_mu);
    if (g_tuned[si] || !autotune_enabled()) return SPRING_OK;
  }
  return autotune_n(n, batch, s);
}

}  // namespace spring

using namespace spring;

extern "C" {

spring_status spring_set_kernel_variant(int n, int row_variant, int col_variant) {
  const int si = side_index(n);
  if (si < 0) return invalid("unsupported pattern side");
  if (row_variant >= ROW_VARIANTS || col_variant >= COL_VARIANTS) return invalid("no such variant");
  std::lock_guard<std::mutex> lk(g_var_mu);
  if (row_variant >= 0) g_row_var[si] = row_variant;
  if (col_variant >= 0) g_col_var[si] = col_variant;
  g_tuned[si] = true;  // an explicit choice is kept
  return SPRING_OK;
}

spring_status spring_get_kernel_variant(int n, int* row_variant, int* col_variant) {
  const int si = side_index(n);
  if (si < 0) return invalid("unsupported pattern side");
  std::lock_guard<std::mutex> lk(g_var_mu);
  if (row_variant) *row_variant = g_row_var[si];
  if (col_variant) *col_variant = g_col_var[si];
  return SPRING_OK;
}

spring_status spring_autotune(int n, int batch, void* stream) {
  return autotune_n(n, batch, reinterpret_cast<cudaStream_t>(stream));
}

spring_status spring_set_iteration_path(int n, int path) {
  const int si = side_index(n);
  if (si < 0) return invalid("unsupported pattern side");
  if (path < 0 || path > 2) return invalid("path must be 0 (two passes), 1 (on chip) or 2 (split passes)");
  if (path == 2 && !split_side(n)) return invalid("the split passes cover sides 192, 384, 512, 768 and 1024");
  if (path == 1) {
    bool ok = false;
    SPRING_TRY(cluster_supported(n, &ok));
    if (!ok) return invalid("the on-chip iteration kernel does not cover this side on this device");
  }
  std::lock_guard<std::mutex> lk(g_var_mu);
  g_path[si] = path;
  g_tuned[si] = true;  // an explicit choice is kept
  return SPRING_OK;
}

spring_status spring_get_iteration_path(int n, int* path) {
  const int si = side_index(n);
  if (si < 0) return invalid("unsupported pattern side");
  std::lock_guard<std::mutex> lk(g_var_mu);
  if (path) *path = g_path[si];
  return SPRING_OK;
}

}  // extern "C"
