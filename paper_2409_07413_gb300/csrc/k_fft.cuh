// k_fft.cuh -- the per-iteration passes of the hot path and the plain 2D transforms
// (kernel templates; instantiated per side N in k_fft_n*.cu).
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
// Per iteration and pixel this moves 8 (w) + 8 (x_n) + 1 (S) + 8 (x_{n+1}) + 8 (w) bytes
// in the row pass and 8 + 8 in the column pass: 49 B (ER: 41 B, x_n unread).
//
// Launch-shape variants (bit-identical results within a plan):
//   row:    0 = state loads before the inverse transform, 1 block/SM of registers;
//           1 / 2 = state loads after it, register budget for 2 / 3 blocks per SM
//   column: 0 = default plan, 16-column tiles; 1 = alternative plan (other radices:
//           results differ by rounding); 2 = 32-column tiles; 3 = 8-column tiles
#pragma once

#include "fft.cuh"
#include "internal.h"

namespace spring {

enum { ROW_ITER = 0, ROW_FWD = 1, ROW_INV = 2 };
enum { COL_PM = 0, COL_FWD = 1, COL_INV = 2, COL_ERR = 3 };
enum { OP_ROW_ITER = 0, OP_ROW_FWD, OP_ROW_INV, OP_COL_PM, OP_COL_FWD, OP_COL_INV, OP_COL_ERR };

constexpr int ROW_THREADS = 256;
constexpr int ROW_VARIANTS = 3;
constexpr int COL_VARIANTS = 4;
constexpr int ERR_W = 16;  // column tile of the error pass (layout of its partial sums)

// alternative column-pass plans
template <int N> struct AltPlan;
template <> struct AltPlan<64>   : PlanT<64, 16, 16, 4> {};
template <> struct AltPlan<128>  : PlanT<128, 16, 16, 8> {};
template <> struct AltPlan<192>  : PlanT<192, 24, 3, 8, 8> {};
template <> struct AltPlan<256>  : PlanT<256, 32, 32, 8> {};
template <> struct AltPlan<512>  : PlanT<512, 32, 32, 16> {};
template <> struct AltPlan<1024> : PlanT<1024, 16, 16, 8, 8> {};

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

struct ColArgs {
  float2* data;       // batch images, transformed in place along columns
  const float* M;     // PM / ERR: modulus (negative = not measured), DFT order
  const float2* tw;
  int batch;
  float scale;        // FWD / INV output scale
  double* partials;   // ERR: [batch][N / ERR_W][2] (sum Xi (|X| - M)^2, sum Xi M^2)
};

struct FftOp {
  int kind = 0, alg = 0, variant = 0, kclass = SPRING_KC_OTHER;
  double bytes = 0.0;
  RowArgs ra{};
  ColArgs ca{};
};

template <int T>
__device__ __forceinline__ WarpSync group_sync() {
  static_assert(T <= 32, "one transform per lane group of a warp");
  const unsigned lane = threadIdx.x & 31u;
  return WarpSync{T == 32 ? 0xffffffffu : (((1u << T) - 1u) << (lane & ~(unsigned)(T - 1)))};
}

__device__ __forceinline__ float2 update_pixel(int alg, float2 xo, float2 pm, bool in_c, float beta) {
  if (in_c) return pm;
  if (alg == 0) return make_float2(0.f, 0.f);
  if (alg == 1) return make_float2(xo.x - beta * pm.x, xo.y - beta * pm.y);
  const float c = 1.f - 2.f * beta;
  return make_float2(beta * xo.x + c * pm.x, beta * xo.y + c * pm.y);
}

template <class P, int MODE, int ALG, bool LATE, int MINB>
__global__ void __launch_bounds__(ROW_THREADS, MINB) k_row(RowArgs a) {
  constexpr int N = P::N, E = P::E, T = P::T, G = ROW_THREADS / T, SME = pad_elems_p<P>();
  extern __shared__ float2 smem[];
  const int grp = threadIdx.x / T, t = threadIdx.x % T;
  float2* sm = smem + grp * SME;
  const WarpSync sync = group_sync<T>();
  for (long long row = (long long)blockIdx.x * G + grp; row < a.nrows; row += (long long)gridDim.x * G) {
    const long long base = row * N + t;
    float2 v[E];
    if constexpr (MODE == ROW_ITER) {
      uint8_t s[E];
      float2 xo[E];
      if constexpr (!LATE) {
#pragma unroll
        for (int m = 0; m < E; ++m) {
          s[m] = a.S[base + m * T];
          if (ALG != 0) xo[m] = a.x[base + m * T];
        }
      }
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = a.in[base + m * T];
      fft_plan<P, +1, true, 1>(v, sm, t, a.tw, sync);  // m = P_M x_n
      if constexpr (LATE) {
#pragma unroll
        for (int m = 0; m < E; ++m) {
          s[m] = a.S[base + m * T];
          if (ALG != 0) xo[m] = a.x[base + m * T];
        }
      }
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const float2 pm = v[m];
        bool in_c = s[m] != 0;
        if (a.chi_on) in_c = in_c && (pm.x >= a.cchi * sqrtf(pm.x * pm.x + pm.y * pm.y));
        const float2 xn = update_pixel(ALG, ALG ? xo[m] : pm, pm, in_c, a.beta);
        v[m] = xn;
        a.x[base + m * T] = xn;
      }
      if (a.zout) {
        fft_plan<P, -1, true, 1>(v, sm, t, a.tw, sync);
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
      fft_plan<P, MODE == ROW_FWD ? -1 : +1, true, 1>(v, sm, t, a.tw, sync);
#pragma unroll
      for (int m = 0; m < E; ++m) a.out[base + m * T] = cscale(v[m], a.scale);
    }
  }
}

template <class P, int W, int MODE>
__global__ void __launch_bounds__(W * P::T) k_col(ColArgs a) {
  constexpr int N = P::N, E = P::E, T = P::T, STRIPS = N / W;
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
    fft_plan<P, +1, false, W>(v, smem + c, t, a.tw, sync);
#pragma unroll
    for (int m = 0; m < E; ++m) base[(size_t)(t + m * T) * N] = cscale(v[m], a.scale);
    return;
  }
  fft_plan<P, -1, false, W>(v, smem + c, t, a.tw, sync);
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
    fft_plan<P, +1, false, W>(v, smem + c, t, a.tw, sync);
#pragma unroll
    for (int m = 0; m < E; ++m) base[(size_t)(t + m * T) * N] = v[m];
  } else {  // COL_ERR: FP64 accumulation of the Fourier error (Eq. error_calc)
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
    // fixed-order block reduction: warp tree, then thread 0 over the warp sums
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      num += __shfl_down_sync(0xffffffffu, num, o);
      den += __shfl_down_sync(0xffffffffu, den, o);
    }
    __shared__ double red[2][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
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

// ------------------------------------------------------------------ launch helpers
template <class K>
inline void allow_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <class P, int MODE, int ALG, bool LATE, int MINB>
inline spring_status row_launch(const FftOp& op, cudaStream_t s, bool prepare_only) {
  constexpr int G = ROW_THREADS / P::T;
  const size_t smem = (size_t)G * pad_elems_p<P>() * sizeof(float2);
  if (prepare_only) {
    allow_smem(k_row<P, MODE, ALG, LATE, MINB>, smem);
    return SPRING_OK;
  }
  long long blocks = (op.ra.nrows + G - 1) / G;
  const long long cap = 64LL * sm_count();
  if (blocks > cap) blocks = cap;
  if (blocks < 1) return SPRING_OK;
  launch_begin(op.kclass, s);
  k_row<P, MODE, ALG, LATE, MINB><<<(int)blocks, ROW_THREADS, smem, s>>>(op.ra);
  SPRING_CHECK_LAUNCH();
  launch_end(op.kclass, s, op.bytes);
  return SPRING_OK;
}

template <int N, int W>
constexpr int fit_w() {  // keep the column tile within shared memory and 1024 threads
  return ((size_t)N * W * 8 > 200 * 1024 || W * Plan<N>::T > 1024) ? W / 2 : W;
}

template <class P, int W, int MODE>
inline spring_status col_launch(const FftOp& op, cudaStream_t s, bool prepare_only) {
  const size_t smem = (size_t)P::N * W * sizeof(float2);
  if (prepare_only) {
    allow_smem(k_col<P, W, MODE>, smem);
    return SPRING_OK;
  }
  if (op.ca.batch < 1) return SPRING_OK;
  launch_begin(op.kclass, s);
  k_col<P, W, MODE><<<op.ca.batch * (P::N / W), W * P::T, smem, s>>>(op.ca);
  SPRING_CHECK_LAUNCH();
  launch_end(op.kclass, s, op.bytes);
  return SPRING_OK;
}

template <int N, int ALG>
inline spring_status row_iter_variant(const FftOp& op, cudaStream_t s, bool prep) {
  switch (op.variant) {
    case 0: return row_launch<Plan<N>, ROW_ITER, ALG, false, 1>(op, s, prep);
    case 1: return row_launch<Plan<N>, ROW_ITER, ALG, true, 2>(op, s, prep);
    default: return row_launch<Plan<N>, ROW_ITER, ALG, true, 3>(op, s, prep);
  }
}

template <int N, int MODE>
inline spring_status col_variant(const FftOp& op, cudaStream_t s, bool prep) {
  switch (op.variant) {
    case 0: return col_launch<Plan<N>, 16, MODE>(op, s, prep);
    case 1: return col_launch<AltPlan<N>, 16, MODE>(op, s, prep);
    case 2: return col_launch<Plan<N>, fit_w<N, 32>(), MODE>(op, s, prep);
    default: return col_launch<Plan<N>, 8, MODE>(op, s, prep);
  }
}

// every operation on side N; prep = only raise the shared-memory limits
template <int N>
spring_status run_fft_op(const FftOp& op, cudaStream_t s, bool prep) {
  switch (op.kind) {
    case OP_ROW_ITER:
      if (op.alg == 0) return row_iter_variant<N, 0>(op, s, prep);
      if (op.alg == 1) return row_iter_variant<N, 1>(op, s, prep);
      return row_iter_variant<N, 2>(op, s, prep);
    case OP_ROW_FWD: return row_launch<Plan<N>, ROW_FWD, 0, false, 1>(op, s, prep);
    case OP_ROW_INV: return row_launch<Plan<N>, ROW_INV, 0, false, 1>(op, s, prep);
    case OP_COL_PM: return col_variant<N, COL_PM>(op, s, prep);
    case OP_COL_FWD: return col_launch<Plan<N>, 16, COL_FWD>(op, s, prep);
    case OP_COL_INV: return col_launch<Plan<N>, 16, COL_INV>(op, s, prep);
    case OP_COL_ERR: return col_launch<Plan<N>, ERR_W, COL_ERR>(op, s, prep);
  }
  return invalid("unknown transform operation");
}

}  // namespace spring
