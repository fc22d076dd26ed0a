// k_fft.cu -- the per-iteration passes of the hot path and the plain 2D transforms.
//
// One MPR iteration x_n -> x_{n+1} (Sec. "The phase problem and conventional
// approaches"; Eq. pm_full; App. "Real-space constraints") is two kernels over an
// intermediate image w kept in HBM between them:
//
//   row pass    (k_row<ROW_ITER>):  m = rowIFFT(w)            (= P_M x_n, see below)
//                                   x_{n+1} = U(x_n, m, S)    (ER / HIO / RAAR + chi)
//                                   w = rowFFT(x_{n+1})
//   column pass (k_col<COL_PM>):    X = colFFT(w) / N         (= F x_{n+1}, unitary)
//                                   Y = M X / |X| on Xi = 1, X elsewhere      (Eq. pm_full)
//                                   w = colIFFT(Y / N)
//
// so the next row pass's inverse row transform completes F^-1 and yields P_M x_{n+1}.
// Per iteration and pixel this moves 8 (w) + 8 (x_n) + 8 (x_{n+1}) + 8 (w) bytes in the
// row pass and 8 + 8 in the column pass, plus 1 support byte: 49 B (ER: 41 B, x_n unread).
#include "fft.cuh"
#include "internal.h"

namespace spring {

enum { ROW_ITER = 0, ROW_FWD = 1, ROW_INV = 2 };
enum { COL_PM = 0, COL_FWD = 1, COL_INV = 2, COL_ERR = 3 };

constexpr int ROW_THREADS = 256;
constexpr int COL_W = 16;  // columns per column-pass block (16 x 8 B = 128 B row segments)

struct RowArgs {
  const float2* in;   // ITER: w (column-pass output); FWD/INV: input rows
  float2* out;        // ITER: w (forward row FFT of x_{n+1}); FWD/INV: output rows
  float2* x;          // ITER: state x_n -> x_{n+1}
  const uint8_t* S;   // ITER: support; FWD: optional multiplier (S x); else unused
  const float2* tw;
  long long nrows;
  float beta, cchi, scale;
  int chi_on, zout;
};

template <int N>
__device__ __forceinline__ WarpSync row_sync() {
  constexpr int T = N / Plan<N>::E;
  static_assert(T <= 32, "one transform per lane group of a warp");
  const unsigned lane = threadIdx.x & 31u;
  return WarpSync{T == 32 ? 0xffffffffu : (((1u << T) - 1u) << (lane & ~(unsigned)(T - 1)))};
}

template <int N, int MODE, int ALG>
__global__ void __launch_bounds__(ROW_THREADS) k_row(RowArgs a) {
  using P = Plan<N>;
  constexpr int E = P::E, T = N / E, G = ROW_THREADS / T, SME = pad_elems<N>();
  extern __shared__ float2 smem[];
  const int grp = threadIdx.x / T, t = threadIdx.x % T;
  float2* sm = smem + grp * SME;
  const WarpSync sync = row_sync<N>();
  for (long long row = (long long)blockIdx.x * G + grp; row < a.nrows; row += (long long)gridDim.x * G) {
    const long long base = row * N + t;
    float2 v[E];
    if constexpr (MODE == ROW_ITER) {
      uint8_t s[E];
      float2 xo[E];
#pragma unroll
      for (int m = 0; m < E; ++m) {
        s[m] = a.S[base + m * T];
        if (ALG != 0) xo[m] = a.x[base + m * T];
        v[m] = a.in[base + m * T];
      }
      fft_regs<N, +1, true, 1>(v, sm, t, a.tw, sync);  // m = P_M x_n
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const float2 pm = v[m];
        bool in_c = s[m] != 0;
        if (a.chi_on) in_c = in_c && (pm.x >= a.cchi * sqrtf(pm.x * pm.x + pm.y * pm.y));
        float2 xn;
        if (in_c) {
          xn = pm;
        } else if (ALG == 0) {
          xn = make_float2(0.f, 0.f);
        } else if (ALG == 1) {
          xn = make_float2(xo[m].x - a.beta * pm.x, xo[m].y - a.beta * pm.y);
        } else {
          const float c = 1.f - 2.f * a.beta;
          xn = make_float2(a.beta * xo[m].x + c * pm.x, a.beta * xo[m].y + c * pm.y);
        }
        v[m] = xn;
        a.x[base + m * T] = xn;
      }
      if (a.zout) {
        fft_regs<N, -1, true, 1>(v, sm, t, a.tw, sync);
#pragma unroll
        for (int m = 0; m < E; ++m) a.out[base + m * T] = v[m];
      }
    } else {
#pragma unroll
      for (int m = 0; m < E; ++m) {
        float2 q = a.in[base + m * T];
        if (MODE == ROW_FWD && a.S && !a.S[base + m * T]) q = make_float2(0.f, 0.f);
        v[m] = q;
      }
      fft_regs<N, MODE == ROW_FWD ? -1 : +1, true, 1>(v, sm, t, a.tw, sync);
#pragma unroll
      for (int m = 0; m < E; ++m) a.out[base + m * T] = cscale(v[m], a.scale);
    }
  }
}

struct ColArgs {
  float2* data;       // batch images, transformed in place along columns
  const float* M;     // PM / ERR: modulus (negative = not measured), DFT order
  const float2* tw;
  int batch;
  float scale;        // FWD / INV output scale
  double* partials;   // ERR: [batch][N / COL_W][2] (sum Xi (|X| - M)^2, sum Xi M^2)
};

template <int N>
constexpr int col_threads() { return COL_W * (N / Plan<N>::E); }

template <int N, int MODE>
__global__ void __launch_bounds__(col_threads<N>()) k_col(ColArgs a) {
  using P = Plan<N>;
  constexpr int E = P::E, T = N / E, W = COL_W, STRIPS = N / W;
  extern __shared__ float2 smem[];
  const int c = threadIdx.x % W, t = threadIdx.x / W;
  const int img = blockIdx.x / STRIPS, strip = blockIdx.x % STRIPS;
  const int col = strip * W + c;
  float2* base = a.data + (size_t)img * N * N + col;
  const BlockSync sync;
  float2 v[E];
#pragma unroll
  for (int m = 0; m < E; ++m) v[m] = base[(size_t)(t + m * T) * N];
  if constexpr (MODE == COL_INV) {
    fft_regs<N, +1, false, W>(v, smem + c, t, a.tw, sync);
#pragma unroll
    for (int m = 0; m < E; ++m) base[(size_t)(t + m * T) * N] = cscale(v[m], a.scale);
    return;
  }
  fft_regs<N, -1, false, W>(v, smem + c, t, a.tw, sync);
  if constexpr (MODE == COL_FWD) {
#pragma unroll
    for (int m = 0; m < E; ++m) base[(size_t)(t + m * T) * N] = cscale(v[m], a.scale);
  } else if constexpr (MODE == COL_PM) {
    constexpr float inv_n = 1.0f / N;
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const float Mv = __ldg(&a.M[(size_t)(t + m * T) * N + col]);
      const float2 X = v[m];
      if (Mv >= 0.f) {
        const float a2 = X.x * X.x + X.y * X.y;
        v[m] = a2 > 0.f ? cscale(X, Mv * rsqrtf(a2) * inv_n) : make_float2(Mv * inv_n, 0.f);
      } else {
        v[m] = cscale(X, inv_n * inv_n);
      }
    }
    fft_regs<N, +1, false, W>(v, smem + c, t, a.tw, sync);
#pragma unroll
    for (int m = 0; m < E; ++m) base[(size_t)(t + m * T) * N] = v[m];
  } else {  // COL_ERR
    constexpr float inv_n = 1.0f / N;
    double num = 0.0, den = 0.0;
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const float Mv = __ldg(&a.M[(size_t)(t + m * T) * N + col]);
      if (Mv >= 0.f) {
        const float amp = sqrtf(v[m].x * v[m].x + v[m].y * v[m].y) * inv_n;
        const double d = (double)amp - (double)Mv;
        num += d * d;
        den += (double)Mv * (double)Mv;
      }
    }
    // fixed-order block reduction: warp tree, then warp 0 over the warp sums
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      num += __shfl_down_sync(0xffffffffu, num, o);
      den += __shfl_down_sync(0xffffffffu, den, o);
    }
    __shared__ double red[2][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();  // the transform's shared buffer is no longer read
    if (lane == 0) {
      red[0][warp] = num;
      red[1][warp] = den;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double sn = 0.0, sd = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        sn += red[0][w];
        sd += red[1][w];
      }
      a.partials[((size_t)img * STRIPS + strip) * 2 + 0] = sn;
      a.partials[((size_t)img * STRIPS + strip) * 2 + 1] = sd;
    }
  }
}

__global__ void k_err_finalize(const double* __restrict__ partials, int strips, int batch,
                               double* __restrict__ err, int* __restrict__ status) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  double sn = 0.0, sd = 0.0;
  for (int s = 0; s < strips; ++s) {
    sn += partials[((size_t)b * strips + s) * 2 + 0];
    sd += partials[((size_t)b * strips + s) * 2 + 1];
  }
  const double e = sd > 0.0 ? sqrt(sn / sd) : 0.0;
  if (!isfinite(e) && status) atomicOr(status, 1);
  err[b] = e;
}

// ------------------------------------------------------------------ launchers
template <class K>
static void allow_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int N, int MODE, int ALG>
static spring_status row_launch(const RowArgs& a, cudaStream_t s, int kclass, double bytes) {
  constexpr int T = N / Plan<N>::E, G = ROW_THREADS / T;
  const size_t smem = (size_t)G * pad_elems<N>() * sizeof(float2);
  static bool init = false;
  if (!init) {
    allow_smem(k_row<N, MODE, ALG>, smem);
    init = true;
  }
  long long blocks = (a.nrows + G - 1) / G;
  const long long cap = 64LL * sm_count();
  if (blocks > cap) blocks = cap;
  if (blocks < 1) return SPRING_OK;
  launch_begin(kclass, s);
  k_row<N, MODE, ALG><<<(int)blocks, ROW_THREADS, smem, s>>>(a);
  SPRING_CHECK_LAUNCH();
  launch_end(kclass, s, bytes);
  return SPRING_OK;
}

template <int N, int MODE>
static spring_status col_launch(const ColArgs& a, cudaStream_t s, int kclass, double bytes) {
  const size_t smem = (size_t)N * COL_W * sizeof(float2);
  static bool init = false;
  if (!init) {
    allow_smem(k_col<N, MODE>, smem);
    init = true;
  }
  if (a.batch < 1) return SPRING_OK;
  launch_begin(kclass, s);
  k_col<N, MODE><<<a.batch * (N / COL_W), col_threads<N>(), smem, s>>>(a);
  SPRING_CHECK_LAUNCH();
  launch_end(kclass, s, bytes);
  return SPRING_OK;
}

#define SPRING_DISPATCH_N(n, CALL)            \
  switch (n) {                                \
    case 64: { constexpr int NN = 64; return CALL; }     \
    case 128: { constexpr int NN = 128; return CALL; }   \
    case 192: { constexpr int NN = 192; return CALL; }   \
    case 256: { constexpr int NN = 256; return CALL; }   \
    case 512: { constexpr int NN = 512; return CALL; }   \
    case 1024: { constexpr int NN = 1024; return CALL; } \
    default: return invalid("unsupported pattern side");  \
  }

template <int N>
static spring_status row_iter_n(int alg, const RowArgs& a, cudaStream_t s, double bytes) {
  switch (alg) {
    case 0: return row_launch<N, ROW_ITER, 0>(a, s, SPRING_KC_ROW_ITER, bytes);
    case 1: return row_launch<N, ROW_ITER, 1>(a, s, SPRING_KC_ROW_ITER, bytes);
    case 2: return row_launch<N, ROW_ITER, 2>(a, s, SPRING_KC_ROW_ITER, bytes);
  }
  return invalid("algorithm must be 0 (ER), 1 (HIO) or 2 (RAAR)");
}

spring_status launch_row_iter(int n, int alg, float2* w, float2* x, const uint8_t* S, long long batch,
                              float beta, float chi, bool zout, cudaStream_t s) {
  DeviceTables tb;
  SPRING_TRY(device_tables(&tb));
  RowArgs a{};
  a.in = w;
  a.out = w;
  a.x = x;
  a.S = S;
  a.tw = tb.tw + tw_offset(n);
  a.nrows = batch * n;
  a.beta = beta;
  a.chi_on = chi < 1.0f;
  const double c = (chi == 0.5f) ? 0.0 : cos((double)chi * 3.14159265358979323846);
  a.cchi = (float)c;
  a.zout = zout ? 1 : 0;
  const double px = (double)batch * n * n;
  const double bytes = px * (8.0 + (alg ? 8.0 : 0.0) + 8.0 + (zout ? 8.0 : 0.0) + 1.0);
  SPRING_DISPATCH_N(n, row_iter_n<NN>(alg, a, s, bytes));
}

spring_status launch_row_fft(int n, int dir, const float2* in, float2* out, const uint8_t* Smul,
                             long long batch, float scale, cudaStream_t s) {
  DeviceTables tb;
  SPRING_TRY(device_tables(&tb));
  RowArgs a{};
  a.in = in;
  a.out = out;
  a.S = Smul;
  a.tw = tb.tw + tw_offset(n);
  a.nrows = batch * n;
  a.scale = scale;
  const double bytes = (double)batch * n * n * (16.0 + (Smul ? 1.0 : 0.0));
  if (dir < 0) {
    SPRING_DISPATCH_N(n, (row_launch<NN, ROW_FWD, 0>(a, s, SPRING_KC_OTHER, bytes)));
  } else {
    SPRING_DISPATCH_N(n, (row_launch<NN, ROW_INV, 0>(a, s, SPRING_KC_OTHER, bytes)));
  }
}

spring_status launch_col_pm(int n, float2* w, const float* M, int batch, cudaStream_t s) {
  DeviceTables tb;
  SPRING_TRY(device_tables(&tb));
  ColArgs a{};
  a.data = w;
  a.M = M;
  a.tw = tb.tw + tw_offset(n);
  a.batch = batch;
  const double bytes = (double)batch * n * n * 16.0 + (double)n * n * 4.0;
  SPRING_DISPATCH_N(n, (col_launch<NN, COL_PM>(a, s, SPRING_KC_COL_PM, bytes)));
}

spring_status launch_col_fft(int n, int dir, float2* data, int batch, float scale, cudaStream_t s) {
  DeviceTables tb;
  SPRING_TRY(device_tables(&tb));
  ColArgs a{};
  a.data = data;
  a.tw = tb.tw + tw_offset(n);
  a.batch = batch;
  a.scale = scale;
  const double bytes = (double)batch * n * n * 16.0;
  if (dir < 0) {
    SPRING_DISPATCH_N(n, (col_launch<NN, COL_FWD>(a, s, SPRING_KC_OTHER, bytes)));
  } else {
    SPRING_DISPATCH_N(n, (col_launch<NN, COL_INV>(a, s, SPRING_KC_OTHER, bytes)));
  }
}

int err_strips(int n) { return n / COL_W; }

spring_status launch_col_err(int n, float2* w, const float* M, int batch, double* partials,
                             cudaStream_t s) {
  DeviceTables tb;
  SPRING_TRY(device_tables(&tb));
  ColArgs a{};
  a.data = w;
  a.M = M;
  a.tw = tb.tw + tw_offset(n);
  a.batch = batch;
  a.partials = partials;
  const double bytes = (double)batch * n * n * 8.0 + (double)n * n * 4.0;
  SPRING_DISPATCH_N(n, (col_launch<NN, COL_ERR>(a, s, SPRING_KC_OTHER, bytes)));
}

spring_status launch_err_finalize(int n, const double* partials, int batch, double* err,
                                  int* status, cudaStream_t s) {
  if (batch < 1) return SPRING_OK;
  launch_begin(SPRING_KC_OTHER, s);
  k_err_finalize<<<div_up(batch, 128), 128, 0, s>>>(partials, n / COL_W, batch, err, status);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, 16.0 * batch * (n / COL_W));
  return SPRING_OK;
}

}  // namespace spring

namespace spring {

// Raise the dynamic shared-memory limit of every transform kernel of side N once, before
// any launch (and so before any stream capture).
template <int N>
static void prepare_n() {
  constexpr int T = N / Plan<N>::E, G = ROW_THREADS / T;
  const size_t rs = (size_t)G * pad_elems<N>() * sizeof(float2);
  const size_t cs = (size_t)N * COL_W * sizeof(float2);
  allow_smem(k_row<N, ROW_ITER, 0>, rs);
  allow_smem(k_row<N, ROW_ITER, 1>, rs);
  allow_smem(k_row<N, ROW_ITER, 2>, rs);
  allow_smem(k_row<N, ROW_FWD, 0>, rs);
  allow_smem(k_row<N, ROW_INV, 0>, rs);
  allow_smem(k_col<N, COL_PM>, cs);
  allow_smem(k_col<N, COL_FWD>, cs);
  allow_smem(k_col<N, COL_INV>, cs);
  allow_smem(k_col<N, COL_ERR>, cs);
}

spring_status prepare_fft_kernels(int n) {
  switch (n) {
    case 64: prepare_n<64>(); break;
    case 128: prepare_n<128>(); break;
    case 192: prepare_n<192>(); break;
    case 256: prepare_n<256>(); break;
    case 512: prepare_n<512>(); break;
    case 1024: prepare_n<1024>(); break;
    default: return invalid("unsupported pattern side");
  }
  SPRING_CHECK_LAUNCH();
  return SPRING_OK;
}

}  // namespace spring

namespace spring {

// Variants of the error-path launchers that take the twiddle table from the caller
// instead of the per-device table (used by the entry point that must not allocate).
spring_status launch_row_fft_tw(int n, int dir, const float2* in, float2* out, const uint8_t* Smul,
                                long long batch, float scale, const float2* tw_all, cudaStream_t s) {
  RowArgs a{};
  a.in = in;
  a.out = out;
  a.S = Smul;
  a.tw = tw_all + tw_offset(n);
  a.nrows = batch * n;
  a.scale = scale;
  const double bytes = (double)batch * n * n * (16.0 + (Smul ? 1.0 : 0.0));
  if (dir < 0) {
    SPRING_DISPATCH_N(n, (row_launch<NN, ROW_FWD, 0>(a, s, SPRING_KC_OTHER, bytes)));
  } else {
    SPRING_DISPATCH_N(n, (row_launch<NN, ROW_INV, 0>(a, s, SPRING_KC_OTHER, bytes)));
  }
}

spring_status launch_col_err_tw(int n, float2* w, const float* M, int batch, double* partials,
                                const float2* tw_all, cudaStream_t s) {
  ColArgs a{};
  a.data = w;
  a.M = M;
  a.tw = tw_all + tw_offset(n);
  a.batch = batch;
  a.partials = partials;
  const double bytes = (double)batch * n * n * 8.0 + (double)n * n * 4.0;
  SPRING_DISPATCH_N(n, (col_launch<NN, COL_ERR>(a, s, SPRING_KC_OTHER, bytes)));
}

}  // namespace spring
