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
// Per iteration and pixel this moves 8 (w) + 8 (x_n) + 1/8 (S, one bit per pixel, packed
// before each block of iterations) + 8 (x_{n+1}) + 8 (w) bytes in the row pass and 8 + 8
// in the column pass: 48.125 B (ER: 40.125 B, x_n unread).
//
// Launch-shape variants (bit-identical results within a plan):
//   row:    0 = state loads before the inverse transform, 1 block/SM of registers;
//           1 / 2 = state loads after it, register budget for 2 / 3 blocks per SM;
//           3 / 4 = x and S rows streamed into shared memory (cp.async) during the
//           inverse transform, register budget for 2 / 3 blocks per SM;
//           5 / 6 = alternative radix plan (results differ by rounding), loads after the
//           inverse transform, register budget for 2 / 4 blocks per SM
//   column: 0 = default plan, 16-column tiles; 1 = alternative plan (other radices:
//           results differ by rounding), 16-column tiles, 8 where two such blocks would
//           not fit an SM; 2 = 32-column tiles; 3 = 8-column tiles;
//           4 / 5 = persistent blocks fed by TMA: while a block transforms one tile, the
//           next tile is already being copied into a second shared buffer (16 / 8 columns);
//           6 / 7 = transposed tiles, one lane group per column (16 / 32 columns; 8 at
//           N >= 1024 / 512); 8 / 9 = two adjacent columns per thread (16-byte accesses
//           throughout), 16 / 32-column tiles, plans of at most 8 elements per thread
//           (16 at N = 1024); 10 = alternative plan, 512-thread blocks held to three per
//           SM (40 registers, 48 warps per SM), where such a tile divides the side
#pragma once

#include <cuda_fp16.h>

#include <type_traits>

#include "fft.cuh"
#include "internal.h"
#include "tma.cuh"

namespace spring {

enum { ROW_ITER = 0, ROW_FWD = 1, ROW_INV = 2, ROW_INIT16 = 3 };
enum { COL_PM = 0, COL_FWD = 1, COL_INV = 2, COL_ERR = 3 };
enum { OP_ROW_ITER = 0, OP_ROW_FWD, OP_ROW_INV, OP_COL_PM, OP_COL_FWD, OP_COL_INV, OP_COL_ERR,
       OP_ROW_ITER16, OP_COL_PM16, OP_ROW_INIT16, OP_ROW_SPLIT, OP_ROW_SPLIT_FWD, OP_COL_SPLIT };

constexpr int ROW_THREADS = 256;
constexpr int ROW_VARIANTS = 7;
constexpr int COL_VARIANTS = 11;
constexpr int ERR_W = 16;  // column tile of the error pass (layout of its partial sums)

// alternative column-pass plans
template <int N> struct AltPlan;
template <> struct AltPlan<64>   : PlanT<64, 16, 16, 4> {};
template <> struct AltPlan<96>   : PlanT<96, 24, 3, 8, 4> {};
template <> struct AltPlan<128>  : PlanT<128, 16, 16, 8> {};
template <> struct AltPlan<192>  : PlanT<192, 24, 3, 8, 8> {};
template <> struct AltPlan<256>  : PlanT<256, 32, 32, 8> {};
template <> struct AltPlan<384>  : PlanT<384, 24, 3, 8, 4, 4> {};
template <> struct AltPlan<512>  : PlanT<512, 8, 8, 8, 8> {};
template <> struct AltPlan<768>  : PlanT<768, 24, 3, 8, 8, 4> {};
template <> struct AltPlan<1024> : PlanT<1024, 16, 16, 8, 8> {};

// row and column plans of the FP16-storage iteration passes
template <int N> struct Row16Plan : Plan<N> {};
template <> struct Row16Plan<1024> : PlanT<1024, 16, 16, 8, 8> {};
template <int N> struct Col16Plan : Plan<N> {};
template <> struct Col16Plan<1024> : PlanT<1024, 16, 16, 8, 8> {};

// plans of the paired column pass (two columns per thread; the fewest elements per
// thread that the radices allow)
template <int N> struct Col2Plan;
template <> struct Col2Plan<64>   : PlanT<64, 8, 8, 8> {};
template <> struct Col2Plan<96>   : PlanT<96, 12, 4, 4, 2, 3> {};
template <> struct Col2Plan<128>  : PlanT<128, 8, 8, 4, 4> {};
template <> struct Col2Plan<192>  : PlanT<192, 12, 4, 4, 4, 3> {};
template <> struct Col2Plan<256>  : PlanT<256, 8, 8, 8, 4> {};
template <> struct Col2Plan<384>  : PlanT<384, 12, 4, 4, 4, 2, 3> {};
template <> struct Col2Plan<512>  : PlanT<512, 8, 8, 8, 8> {};
template <> struct Col2Plan<768>  : PlanT<768, 12, 4, 4, 4, 4, 3> {};
template <> struct Col2Plan<1024> : PlanT<1024, 16, 16, 8, 8> {};

// alternative row-pass plans (fewer elements per thread; T = 64 rows sync by named barrier)
template <int N> struct RowAltPlan : Plan<N> {};
template <> struct RowAltPlan<1024> : PlanT<1024, 16, 16, 8, 8> {};
template <> struct RowAltPlan<512> : PlanT<512, 8, 8, 8, 8> {};
template <> struct RowAltPlan<256> : PlanT<256, 32, 32, 8> {};
template <> struct RowAltPlan<128> : PlanT<128, 16, 16, 8> {};
template <> struct RowAltPlan<96> : PlanT<96, 12, 4, 4, 2, 3> {};
template <> struct RowAltPlan<192> : PlanT<192, 12, 4, 4, 4, 3> {};
template <> struct RowAltPlan<384> : PlanT<384, 12, 4, 4, 4, 2, 3> {};
template <> struct RowAltPlan<768> : PlanT<768, 12, 4, 4, 4, 4, 3> {};

// FP16 storage of the iteration buffers (precision 1): x as half2 scaled by the problem's
// power of two s16 (chosen from ||M||_2 so that every stored value stays well inside the
// FP16 range, see k_fp16_scale), w as half2 scaled by s16 times a power of two near
// 1/sqrt(N) that absorbs the growth of the unnormalised row transforms.  Power-of-two
// scales are exact, so only the FP16 rounding of each stored value remains.  All
// arithmetic stays FP32.
__host__ __device__ constexpr float w16_scale(int n) {
  return n >= 512 ? 1.0f / 32 : n >= 128 ? 1.0f / 16 : 1.0f / 8;
}
template <class ST>
__device__ __forceinline__ float2 ld_st(const ST* p, long long i, float inv) {
  if constexpr (std::is_same<ST, __half2>::value) {
    const float2 v = __half22float2(p[i]);
    return make_float2(v.x * inv, v.y * inv);
  } else {
    return p[i];
  }
}
template <class ST>
__device__ __forceinline__ void st_st(ST* p, long long i, float2 v, float sc) {
  if constexpr (std::is_same<ST, __half2>::value) {
    p[i] = __float22half2_rn(make_float2(v.x * sc, v.y * sc));
  } else {
    p[i] = v;
  }
}

struct RowArgs {
  const float2* in;   // ITER: w (column-pass output); FWD/INV: input rows
  float2* out;        // ITER: w (forward row FFT of x_{n+1}); FWD/INV: output rows
  float2* x;          // ITER: state x_n -> x_{n+1}
  const uint8_t* S;   // FWD: optional multiplier (S x); else unused
  const uint32_t* Sb; // ITER: support, one bit per pixel (pixel i: bit i & 31 of word i >> 5)
  const float2* tw;
  long long nrows;
  float beta, cchi, scale;
  int chi_on, zout;
  void* xh;           // INIT16: FP16 copy of x (out)
  const float* s16;   // FP16 storage: device scalar s16 (power of two)
};

struct ColArgs {
  float2* data;       // batch images, transformed in place along columns
  const float* M;     // PM / ERR: modulus (negative = not measured), DFT order
  const float2* tw;
  int batch;
  float scale;        // FWD / INV output scale
  double* partials;   // ERR: [batch][N / ERR_W][2] (sum Xi (|X| - M)^2, sum Xi M^2)
  const float* s16;   // FP16 storage: device scalar s16 (power of two)
  int m_group;        // > 0: M holds one N x N array per m_group consecutive images
  int img0;           // index of data's first image in the m_group numbering
  int skip_m2;        // ERR: leave out sum Xi M^2 (formed once per problem instead); 0 there
};

// the modulus array of image img
__device__ __forceinline__ const float* m_of(const ColArgs& a, int img, int n) {
  return a.m_group > 0 ? a.M + (size_t)((a.img0 + img) / a.m_group) * n * n : a.M;
}



// synchronisation of the T threads that own one row transform: a lane group inside a
// warp (T <= 32) or a named barrier over T / 32 whole warps (T = 64, 128)
template <int T, bool WIDE = (T > 32)>
struct GroupSync;
template <int T>
struct GroupSync<T, false> {
  static __device__ __forceinline__ WarpSync make() {
    const unsigned lane = threadIdx.x & 31u;
    return WarpSync{T == 32 ? 0xffffffffu : (((1u << T) - 1u) << (lane & ~(unsigned)(T - 1)))};
  }
};
template <int T>
struct GroupSync<T, true> {
  static_assert(T % 32 == 0 && T <= 128, "wide groups are whole warps");
  static __device__ __forceinline__ NamedSync make() { return NamedSync{1u + threadIdx.x / T, (unsigned)T}; }
};

// The modulus projection of one value X of the unnormalised column transform (|X| / N is
// the unitary modulus), Eq. pm_full with the upper bounds of Eq. pm_bounds, times the 1/N
// that completes the unitary inverse.  Encoding of M: M >= 0 measured (modulus -> M);
// M <= -2 missing with bound U = -2 - M (modulus -> min(|X| / N, U)); otherwise missing
// and free (X unchanged).
__device__ __forceinline__ float2 pm_value(float2 X, float Mv, float inv_n) {
  const float a2 = X.x * X.x + X.y * X.y;
  if (Mv >= 0.f) return a2 > 0.f ? cscale(X, Mv * rsqrtf(a2) * inv_n) : make_float2(Mv * inv_n, 0.f);
  if (Mv <= -2.f) {
    const float U = -2.f - Mv;
    if (a2 * (inv_n * inv_n) > U * U) return cscale(X, U * rsqrtf(a2) * inv_n);
  }
  return cscale(X, inv_n * inv_n);
}

__device__ __forceinline__ float2 update_pixel(int alg, float2 xo, float2 pm, bool in_c, float beta) {
  if (in_c) return pm;
  if (alg == 0) return make_float2(0.f, 0.f);
  if (alg == 1) return make_float2(xo.x - beta * pm.x, xo.y - beta * pm.y);
  const float c = 1.f - 2.f * beta;
  return make_float2(beta * xo.x + c * pm.x, beta * xo.y + c * pm.y);
}

// row-pass staging area of one lane group: the x row (N float2) and the row's support
// words (N / 32 words, rounded up to whole 16-byte units), so that every group's area
// starts on a 16-byte boundary (the x row arrives by 16-byte cp.async)
template <class P>
__host__ __device__ constexpr int stage_elems() { return P::N + 2 * ((P::N / 32 + 3) / 4); }

// support bit of column j of a row from the word that holds it (packed by
// launch_pack_support: rows of N pixels, N a multiple of 32, so column j of a row is bit
// j & 31 of the row's word j >> 5); the words are loaded apart from the test, so that the
// loads of a thread stay independent of one another
__device__ __forceinline__ bool support_bit(uint32_t word, int j) { return (word & (1u << (j & 31))) != 0u; }

// The row pass of the blocks blk, blk + nblk, ... (G rows each) of a launch of
// ROW_THREADS threads per block (k_row runs it over its grid).
template <class P, int MODE, int ALG, bool LATE, bool STAGE = false, class ST = float2>
__device__ __forceinline__ void row_pass(const RowArgs& a, long long blk, long long nblk) {
  constexpr int N = P::N, E = P::E, T = P::T, G = ROW_THREADS / T, SME = pad_elems_p<P>();
  extern __shared__ float2 smem[];
  const int grp = threadIdx.x / T, t = threadIdx.x % T;
  float2* sm = smem + grp * SME;
  float2* xs = smem + G * SME + grp * stage_elems<P>();  // STAGE: x row, then the support words
  uint32_t* sws = reinterpret_cast<uint32_t*>(xs + N);
  static_assert(!STAGE || ((G * SME) % 2 == 0 && stage_elems<P>() % 2 == 0 && N % 2 == 0),
                "staging rows on 16-byte boundaries (16-byte cp.async of x)");
  static_assert(!STAGE || 2 * (stage_elems<P>() - N) >= N / 32, "room for the row's support words");
  const auto sync = GroupSync<T>::make();
  for (long long row = blk * G + grp; row < a.nrows; row += nblk * G) {
    const long long base = row * N + t;
    float2 v[E];
    if constexpr (MODE == ROW_ITER && STAGE) {
      // x_n and the support words of this row stream into shared memory while the row is
      // transformed
      const float2* xr = a.x + row * N;
      const uint32_t* sr = a.Sb + row * (N / 32);
      if (ALG != 0)
        for (int k = t; k < N / 2; k += T) cp_async16(xs + 2 * k, xr + 2 * k);
      for (int k = t; k < N / 32; k += T) cp_async4(sws + k, sr + k);
      cp_async_commit();
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = a.in[base + m * T];
      fft_plan<P, +1, true, 1>(v, sm, t, a.tw, sync);  // m = P_M x_n
      cp_async_wait_all();
      sync();
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const float2 pm = v[m];
        bool in_c = support_bit(sws[(t + m * T) >> 5], t + m * T);
        if (a.chi_on) in_c = in_c && (pm.x >= a.cchi * sqrtf(pm.x * pm.x + pm.y * pm.y));
        const float2 xn = update_pixel(ALG, ALG ? xs[t + m * T] : pm, pm, in_c, a.beta);
        v[m] = xn;
        a.x[base + m * T] = xn;
      }
      sync();  // the staging area is reused by the next row
      if (a.zout) {
        fft_plan<P, -1, true, 1>(v, sm, t, a.tw, sync);
#pragma unroll
        for (int m = 0; m < E; ++m) a.out[base + m * T] = v[m];
      }
    } else if constexpr (MODE == ROW_ITER) {
      const ST* win = reinterpret_cast<const ST*>(a.in);
      ST* wout = reinterpret_cast<ST*>(a.out);
      ST* xs_ = reinterpret_cast<ST*>(a.x);
      constexpr bool H = std::is_same<ST, __half2>::value;
      const float sx = H ? __ldg(a.s16) : 1.0f, ws = H ? w16_scale(N) * sx : 1.0f;
      const float isx = 1.0f / sx, iws = 1.0f / ws;  // exact: powers of two
      uint32_t s[E];  // the support word of each element
      float2 xo[E];
      const uint32_t* srow = a.Sb + row * (N / 32);  // this row's support words
      if constexpr (!LATE) {
#pragma unroll
        for (int m = 0; m < E; ++m) {
          s[m] = srow[(t + m * T) >> 5];
          if (ALG != 0) xo[m] = ld_st(xs_, base + m * T, isx);
        }
      }
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = ld_st(win, base + m * T, iws);
      fft_plan<P, +1, true, 1>(v, sm, t, a.tw, sync);  // m = P_M x_n
      if constexpr (LATE) {
#pragma unroll
        for (int m = 0; m < E; ++m) {
          s[m] = srow[(t + m * T) >> 5];
          if (ALG != 0) xo[m] = ld_st(xs_, base + m * T, isx);
        }
      }
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const float2 pm = v[m];
        bool in_c = support_bit(s[m], t + m * T);
        if (a.chi_on) in_c = in_c && (pm.x >= a.cchi * sqrtf(pm.x * pm.x + pm.y * pm.y));
        const float2 xn = update_pixel(ALG, ALG ? xo[m] : pm, pm, in_c, a.beta);
        v[m] = xn;
        st_st(xs_, base + m * T, xn, sx);
      }
      if (a.zout) {
        fft_plan<P, -1, true, 1>(v, sm, t, a.tw, sync);
#pragma unroll
        for (int m = 0; m < E; ++m) st_st(wout, base + m * T, v[m], ws);
      }
    } else if constexpr (MODE == ROW_INIT16) {
      // FP16 copies of x (xh) and of its scaled forward row transform (out)
      __half2* xh = reinterpret_cast<__half2*>(a.xh);
      __half2* wout = reinterpret_cast<__half2*>(a.out);
      const float sx = __ldg(a.s16), isx = 1.0f / sx;
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const float2 q = a.in[base + m * T];
        xh[base + m * T] = __float22half2_rn(make_float2(q.x * sx, q.y * sx));
        v[m] = ld_st(xh, base + m * T, isx);  // transform exactly what is stored
      }
      fft_plan<P, -1, true, 1>(v, sm, t, a.tw, sync);
#pragma unroll
      for (int m = 0; m < E; ++m) st_st(wout, base + m * T, v[m], w16_scale(N) * sx);
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

template <class P, int MODE, int ALG, bool LATE, int MINB, bool STAGE = false, class ST = float2>
__global__ void __launch_bounds__(ROW_THREADS, MINB) k_row(RowArgs a) {
  row_pass<P, MODE, ALG, LATE, STAGE, ST>(a, blockIdx.x, gridDim.x);
}

// The column pass of tile `tile` (image tile / (N / W), strip of W columns) by a block of
// W * P::T threads (k_col runs one tile per block).
template <class P, int W, int MODE, class ST = float2>
__device__ __forceinline__ void col_pass(const ColArgs& a, int tile) {
  constexpr int N = P::N, E = P::E, T = P::T, STRIPS = N / W;
  constexpr bool H = std::is_same<ST, __half2>::value;
  const float ws = H ? w16_scale(N) * __ldg(a.s16) : 1.0f, iws = 1.0f / ws;
  extern __shared__ float2 smem[];
  const int c = threadIdx.x % W, t = threadIdx.x / W;
  const int img = tile / STRIPS, strip = tile % STRIPS;
  const int col = strip * W + c;
  ST* base = reinterpret_cast<ST*>(a.data) + (size_t)img * N * N + col;
  const BlockSync sync;
  // PM / ERR: the strip's modulus values (N x W floats) arrive in shared memory by
  // cp.async while the tile is read and transformed, so no global latency is exposed
  // between the forward and the inverse transform.  The transform's exchange area holds
  // the W columns interleaved (element i of column c at i W + c)
  float* Ms = reinterpret_cast<float*>(smem + (size_t)N * W);
  if constexpr (MODE == COL_PM || MODE == COL_ERR) {
    constexpr int CH = W / 4;  // 16-byte chunks per row
    for (int k = threadIdx.x; k < N * CH; k += blockDim.x) {
      const int row = k / CH, q = k % CH;
      cp_async16(Ms + row * W + 4 * q, m_of(a, img, N) + (size_t)row * N + strip * W + 4 * q);
    }
    cp_async_commit();
  }
  float2 v[E];
#pragma unroll
  for (int m = 0; m < E; ++m) v[m] = ld_st(base, (long long)(t + m * T) * N, iws);
  if constexpr (MODE == COL_INV) {
    fft_plan<P, +1, false, W, false>(v, smem + c, t, a.tw, sync);  // no shared-memory use after it
#pragma unroll
    for (int m = 0; m < E; ++m) base[(size_t)(t + m * T) * N] = cscale(v[m], a.scale);
    return;
  }
  // PM / ERR: the barrier after the strip's cp.async wait also ends the transform's reads
  fft_plan<P, -1, false, W, MODE == COL_FWD>(v, smem + c, t, a.tw, sync);
  if constexpr (MODE == COL_FWD) {
#pragma unroll
    for (int m = 0; m < E; ++m) base[(size_t)(t + m * T) * N] = cscale(v[m], a.scale);
  } else if constexpr (MODE == COL_PM) {
    constexpr float inv_n = 1.0f / N;
    cp_async_wait_all();
    sync();
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const float Mv = Ms[(t + m * T) * W + c];
      const float2 X = v[m];
      v[m] = pm_value(X, Mv, inv_n);
    }
    fft_plan<P, +1, false, W, false>(v, smem + c, t, a.tw, sync);  // no shared-memory use after it
#pragma unroll
    for (int m = 0; m < E; ++m) st_st(base, (long long)(t + m * T) * N, v[m], ws);
  } else {  // COL_ERR: FP64 accumulation of the Fourier error (Eq. error_calc)
    constexpr float inv_n = 1.0f / N;
    double num = 0.0, den = 0.0;
    cp_async_wait_all();
    sync();
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const float Mv = Ms[(t + m * T) * W + c];
      if (Mv >= 0.f) {
        const float amp = sqrtf(v[m].x * v[m].x + v[m].y * v[m].y) * inv_n;
        const double d = (double)amp - (double)Mv;
        num += d * d;
        if (!a.skip_m2) den += (double)Mv * (double)Mv;
      }
    }
    // fixed-order block reduction: warp tree, then thread 0 over the warp sums
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) num += __shfl_down_sync(0xffffffffu, num, o);
    if (!a.skip_m2) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) den += __shfl_down_sync(0xffffffffu, den, o);
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

template <class P, int W, int MODE, class ST = float2, int MINB = (W * P::T <= 512 ? 2 : 1)>
__global__ void __launch_bounds__(W * P::T, MINB) k_col(ColArgs a) {
  col_pass<P, W, MODE, ST>(a, blockIdx.x);
}

// ------------------------------------------------------------------ split passes
// The column transform of length N = Q L by decimation in frequency over the rows,
// n = n1 + L n2: its first radix-Q stage combines the Q rows n1, n1 + L, ..., n1 + (Q - 1) L,
// y[n1][k2] = W_N^{n1 k2} sum_{n2} x[n1 + L n2] W_Q^{n2 k2}, and the L-point transform of
// y[.][k2] over n1 gives the full transform at the rows Q k1 + k2.  So the row pass of an
// iteration, which transforms those rows anyway, also runs that first stage (and, on its
// way in, the inverse one), and the column pass transforms L-row chunks: chunk k2 holds
// y[n1][k2] at rows k2 L + n1 (the chunked layout of w), and its modulus values come from
// a copy of M permuted to the same layout (row k2 L + k1 of it holds row Q k1 + k2 of M).
// The arithmetic is the same unnormalised 2D transform pair as the two passes', in another
// order of summation.  The column pass, bound by issue rather than HBM, gets shorter
// transforms; the row pass, bound by HBM, takes the first stage.
// Q per side: 512 = 2 x 256 and 192 = 3 x 64, 384 = 3 x 128, 768 = 3 x 256 (the column pass
// runs power-of-two transforms of one exchange, the row pass a radix-2 or radix-3 butterfly
// per set of pixels in registers), 1024 = 8 x 128
__host__ __device__ constexpr int split_q_of(int n) {
  return n == 512 ? 2 : (n == 192 || n == 384 || n == 768) ? 3 : 8;
}
template <int N> __host__ __device__ constexpr int split_q() { return split_q_of(N); }

template <int N> struct SplitRowPlan : RowAltPlan<N> {};  // row transforms of a split row pass
// blocks per SM the register budget of the 8-row set kernel (Q = 8, at 1024) is sized for:
// one 512-thread block of 16-element transforms
template <int N> __host__ __device__ constexpr int split_row_minb() { return 1; }
constexpr bool split_side(int n) { return n == 192 || n == 384 || n == 512 || n == 768 || n == 1024; }
// columns per tile of the split column pass: 16 for 256-point chunks, 32 for shorter
template <int L> __host__ __device__ constexpr int split_col_w() { return L >= 256 ? 16 : 32; }

struct SplitArgs {
  float2* w;           // chunked spectra of the batch (N x N per image)
  float2* x;           // ITER: state x_n -> x_{n+1}; FWD: input
  const uint32_t* Sb;  // ITER: support bits (pixel i: bit i & 31 of word i >> 5)
  const float2* tw;    // e^{-2 pi i k / N}
  long long nsets;     // batch x L sets of Q rows
  float beta, cchi;
  int chi_on;
};

struct FftOp {
  int kind = 0, alg = 0, variant = 0, kclass = SPRING_KC_OTHER;
  double bytes = 0.0;
  RowArgs ra{};
  ColArgs ca{};
  SplitArgs sa{};
};

// shared-memory float2 elements of a split row pass block: the Q rows' exchange areas and,
// staged, the next set's Q spectra rows, the set's Q x rows and its Q rows of support words
template <class P, bool STAGE>
__host__ __device__ constexpr size_t split_row_elems() {
  constexpr int Q = split_q<P::N>();
  return (size_t)Q * pad_elems_p<P>() + (STAGE ? (size_t)2 * Q * P::N + Q * P::N / 64 : 0);
}

// A block of Q T threads per set of Q rows n1 + L n2: lane group n2 transforms row
// n1 + L n2.  MODE ROW_ITER: inverse first stage (chunked w -> rows), inverse row
// transforms (P_M x_n), update, forward row transforms, forward first stage (-> chunked w).
// MODE ROW_FWD: from x, forward row transforms and first stage only.  STAGE (ROW_ITER):
// blocks are persistent and their loads asynchronous 16-byte copies into shared memory --
// the next set's spectra rows are in flight while a set is transformed, and a set's x rows
// and support words while its inverse row transforms run -- so no load waits in line with
// the arithmetic.
template <class P, int MODE, int ALG, bool STAGE>
__global__ void __launch_bounds__(split_q<P::N>() * P::T, split_row_minb<P::N>()) k_row_split(SplitArgs a) {
  constexpr int N = P::N, E = P::E, T = P::T, Q = split_q<N>(), L = N / Q, TH = Q * T, RS = pad_elems_p<P>();
  constexpr int CPT = N / TH;  // columns per thread in the first stages
  static_assert(N % TH == 0 && RS >= N, "a column per thread group, rows fit their exchange areas");
  static_assert(!STAGE || MODE == ROW_ITER, "staging serves the iteration");
  static_assert(!STAGE || ((Q * RS) % 2 == 0 && N % 128 == 0 && (Q * N / 2) % TH == 0),
                "16-byte aligned staging areas, whole copies per thread");
  extern __shared__ __align__(16) float2 smem[];
  float2* R = smem;                 // Q rows of RS: the set's rows, and each row's exchange area
  float2* Ws = smem + Q * RS;       // STAGE: spectra rows k2 L + n1 of the set, k2 = 0..Q-1
  float2* Xs = Ws + Q * N;          // STAGE: the set's x rows, one per lane group
  uint32_t* Bs = reinterpret_cast<uint32_t*>(Xs + Q * N);  // STAGE: their support words
  const int tid = threadIdx.x, grp = tid / T, t = tid % T;
  const auto gsync = GroupSync<T>::make();
  // STAGE: the Q spectra rows of set `set` into Ws (an empty group past the last set)
  auto stage_w = [&](long long set) {
    if (set < a.nsets) {
      const float2* src = a.w + (set / L) * N * N + (set % L) * N;
#pragma unroll
      for (int i = 0; i < Q * N / 2 / TH; ++i) {
        const int k = tid + i * TH, k2 = k / (N / 2), q = k % (N / 2);
        cp_async16(Ws + k2 * N + 2 * q, src + (long long)k2 * L * N + 2 * q);
      }
    }
    cp_async_commit();
  };
  if constexpr (STAGE) {
    stage_w(blockIdx.x);
    cp_async_wait_all();
    __syncthreads();
  }
  for (long long set = blockIdx.x; set < a.nsets; set += gridDim.x) {
    const long long img = set / L;
    const int n1 = (int)(set % L);
    float2* wi = a.w + img * N * N;
    float2* xi = a.x + img * N * N;
    const long long xrow = (long long)(n1 + L * grp) * N;  // the row this lane group owns
    float2 v[E];
    if constexpr (MODE == ROW_ITER) {
      const uint32_t* srow = a.Sb + (img * N * N + xrow) / 32;
#pragma unroll
      for (int j = 0; j < CPT; ++j) {  // inverse first stage of column c
        const int c = tid + j * TH;
        float2 z[Q];
#pragma unroll
        for (int k2 = 0; k2 < Q; ++k2) z[k2] = STAGE ? Ws[k2 * N + c] : wi[(long long)(k2 * L + n1) * N + c];
#pragma unroll
        for (int k2 = 1; k2 < Q; ++k2) z[k2] = cmul(z[k2], cconj(__ldg(&a.tw[n1 * k2])));
        DFT<Q, +1>::run(z);
#pragma unroll
        for (int n2 = 0; n2 < Q; ++n2) R[n2 * RS + c] = z[n2];
      }
      __syncthreads();
      if constexpr (STAGE) {  // the group's own x row and support words, then the next set's spectra
        if constexpr (ALG != 0) {
#pragma unroll
          for (int i = 0; i < N / 2 / T; ++i) cp_async16(Xs + grp * N + 2 * (t + i * T), xi + xrow + 2 * (t + i * T));
        }
        if (t < N / 128) cp_async16(Bs + grp * (N / 32) + 4 * t, srow + 4 * t);
        cp_async_commit();
        stage_w(set + gridDim.x);
      }
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = R[grp * RS + t + m * T];
      gsync();                                                    // before the exchange writes
      fft_plan<P, +1, true, 1>(v, R + grp * RS, t, a.tw, gsync);  // m = P_M x_n
      if constexpr (STAGE) {  // this set's group of copies (the next set's may still fly)
        cp_async_wait_group<1>();
        gsync();
      }
      uint32_t sw[E];
      float2 xo[E];
#pragma unroll
      for (int m = 0; m < E; ++m) {
        sw[m] = STAGE ? Bs[grp * (N / 32) + ((t + m * T) >> 5)] : srow[(t + m * T) >> 5];
        if (ALG != 0) xo[m] = STAGE ? Xs[grp * N + t + m * T] : xi[xrow + t + m * T];
      }
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const float2 pm = v[m];
        bool in_c = support_bit(sw[m], t + m * T);
        if (a.chi_on) in_c = in_c && (pm.x >= a.cchi * sqrtf(pm.x * pm.x + pm.y * pm.y));
        const float2 xn = update_pixel(ALG, ALG ? xo[m] : pm, pm, in_c, a.beta);
        v[m] = xn;
        xi[xrow + t + m * T] = xn;
      }
    } else {
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = xi[xrow + t + m * T];
    }
    fft_plan<P, -1, true, 1>(v, R + grp * RS, t, a.tw, gsync);  // ends with the group's barrier
#pragma unroll
    for (int m = 0; m < E; ++m) R[grp * RS + t + m * T] = v[m];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < CPT; ++j) {  // forward first stage of column c
      const int c = tid + j * TH;
      float2 y[Q];
#pragma unroll
      for (int n2 = 0; n2 < Q; ++n2) y[n2] = R[n2 * RS + c];
      DFT<Q, -1>::run(y);
#pragma unroll
      for (int k2 = 1; k2 < Q; ++k2) y[k2] = cmul(y[k2], __ldg(&a.tw[n1 * k2]));
#pragma unroll
      for (int k2 = 0; k2 < Q; ++k2) wi[(long long)(k2 * L + n1) * N + c] = y[k2];
    }
    if constexpr (STAGE) cp_async_wait_all();  // the next set's spectra rows
    __syncthreads();  // R (and Ws, Xs, Bs) are written again for the next set
  }
}

// The split row pass for Q = 2 or 3 with all rows of a set in one lane group: rows
// n1 + L n2 (L = N / Q) are read at the same columns, so the column transform's first
// radix-Q stage and its inverse run in registers, and the Q row transforms follow one
// another through the group's exchange area.  No shared-memory transposes and no block
// barriers: one set per lane group.  Each thread parks its own elements of the rows that
// wait in shared memory (slot j: row j + 1's input, then row j's result), which needs no
// barrier and keeps one row in registers at a time.  The arithmetic is that of k_row_split
// with the same Q (the twiddles W_N^{n1 k2}, then a radix-Q DFT).
template <class P, int MODE, int ALG, int BT, int MINB>
__global__ void __launch_bounds__(BT, MINB) k_row_group(SplitArgs a) {
  constexpr int N = P::N, E = P::E, T = P::T, G = BT / T, Q = split_q<N>(), L = N / Q, SME = pad_elems_p<P>();
  static_assert((Q == 2 || Q == 3) && E * T == N && G * T == BT && L * Q == N, "Q rows per lane group");
  extern __shared__ float2 smem[];
  const int grp = threadIdx.x / T, t = threadIdx.x % T;
  float2* sm = smem + grp * SME;
  float2* hold = smem + G * SME + grp * (Q - 1) * N;  // Q - 1 parking slots of N
  const auto sync = GroupSync<T>::make();
  for (long long set = (long long)blockIdx.x * G + grp; set < a.nsets; set += (long long)gridDim.x * G) {
    const long long img = set / L;
    const int n1 = (int)(set % L);
    float2* wi = a.w + img * N * N;
    float2* xi = a.x + img * N * N;
    // rows n1 + L n2 of x are the chunk rows k2 L + n1 of w (the same row indices)
    auto row = [&](int q) { return (long long)(n1 + L * q) * N; };
    float2 v[E];
    if constexpr (MODE == ROW_ITER) {
#pragma unroll
      for (int m = 0; m < E; ++m) {  // inverse first stage
        float2 z[Q];
#pragma unroll
        for (int k2 = 0; k2 < Q; ++k2) z[k2] = wi[row(k2) + t + m * T];
#pragma unroll
        for (int k2 = 1; k2 < Q; ++k2) z[k2] = cmul(z[k2], cconj(__ldg(&a.tw[n1 * k2])));
        DFT<Q, +1>::run(z);
        v[m] = z[0];
#pragma unroll
        for (int q = 1; q < Q; ++q) hold[(q - 1) * N + t + m * T] = z[q];
      }
      // row r of x: inverse transform (m = P_M x_n), update, forward transform
      auto iterate_row = [&](long long r) {
        fft_plan<P, +1, true, 1>(v, sm, t, a.tw, sync);
        const uint32_t* srow = a.Sb + (img * N * N + r) / 32;
        uint32_t sw[E];
        float2 xo[E];
#pragma unroll
        for (int m = 0; m < E; ++m) {
          sw[m] = srow[(t + m * T) >> 5];
          if (ALG != 0) xo[m] = xi[r + t + m * T];
        }
#pragma unroll
        for (int m = 0; m < E; ++m) {
          const float2 pm = v[m];
          bool in_c = support_bit(sw[m], t + m * T);
          if (a.chi_on) in_c = in_c && (pm.x >= a.cchi * sqrtf(pm.x * pm.x + pm.y * pm.y));
          const float2 xn = update_pixel(ALG, ALG ? xo[m] : pm, pm, in_c, a.beta);
          v[m] = xn;
          xi[r + t + m * T] = xn;
        }
        fft_plan<P, -1, true, 1>(v, sm, t, a.tw, sync);  // ends with the group's barrier
      };
      iterate_row(row(0));
#pragma unroll 1
      for (int q = 1; q < Q; ++q) {
#pragma unroll
        for (int m = 0; m < E; ++m) {  // slot q - 1: row q's input out, row q - 1's result in
          const float2 nxt = hold[(q - 1) * N + t + m * T];
          hold[(q - 1) * N + t + m * T] = v[m];
          v[m] = nxt;
        }
        iterate_row(row(q));
      }
    } else {  // ROW_FWD: the forward row transforms of x
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        if (q > 0) {
#pragma unroll
          for (int m = 0; m < E; ++m) hold[(q - 1) * N + t + m * T] = v[m];
        }
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = xi[row(q) + t + m * T];
        fft_plan<P, -1, true, 1>(v, sm, t, a.tw, sync);
      }
    }
#pragma unroll
    for (int m = 0; m < E; ++m) {  // forward first stage, into the chunks
      float2 y[Q];
#pragma unroll
      for (int q = 0; q < Q - 1; ++q) y[q] = hold[q * N + t + m * T];
      y[Q - 1] = v[m];
      DFT<Q, -1>::run(y);
#pragma unroll
      for (int k2 = 1; k2 < Q; ++k2) y[k2] = cmul(y[k2], __ldg(&a.tw[n1 * k2]));
#pragma unroll
      for (int k2 = 0; k2 < Q; ++k2) wi[row(k2) + t + m * T] = y[k2];
    }
  }
}

// Split column pass: L-point transforms of the chunks (plan PL of side L), P_M against the
// permuted modulus (a.M in the chunked layout; its unnormalised scale is the full N-point
// transform's), inverse L-point transforms.  Tile = (image, chunk k2, strip of W columns).
template <class PL, int N, int W>
__global__ void __launch_bounds__(W * PL::T, 2) k_col_split(ColArgs a) {
  constexpr int L = PL::N, E = PL::E, T = PL::T, Q = N / L, STRIPS = N / W, CH = W / 4;
  static_assert(Q == split_q<N>() && W % 4 == 0 && N % W == 0, "split column tile");
  extern __shared__ float2 smem[];
  float* Ms = reinterpret_cast<float*>(smem + (size_t)L * W);
  const int c = threadIdx.x % W, t = threadIdx.x / W;
  const int img = blockIdx.x / (Q * STRIPS), rem = blockIdx.x % (Q * STRIPS);
  const int k2 = rem / STRIPS, strip = rem % STRIPS;
  float2* base = a.data + (size_t)img * N * N + (size_t)k2 * L * N + strip * W + c;
  const float* Mb = m_of(a, img, N) + (size_t)k2 * L * N + strip * W;
  for (int k = threadIdx.x; k < L * CH; k += blockDim.x) {
    const int row = k / CH, q = k % CH;
    cp_async16(Ms + row * W + 4 * q, Mb + (size_t)row * N + 4 * q);
  }
  cp_async_commit();
  const BlockSync sync;
  float2 v[E];
#pragma unroll
  for (int m = 0; m < E; ++m) v[m] = base[(size_t)(t + m * T) * N];
  fft_plan<PL, -1, false, W, false>(v, smem + c, t, a.tw, sync);
  cp_async_wait_all();
  sync();  // also ends the transform's shared-memory reads
  constexpr float inv_n = 1.0f / N;
#pragma unroll
  for (int m = 0; m < E; ++m) v[m] = pm_value(v[m], Ms[(t + m * T) * W + c], inv_n);
  fft_plan<PL, +1, false, W, false>(v, smem + c, t, a.tw, sync);  // no shared-memory use after it
#pragma unroll
  for (int m = 0; m < E; ++m) base[(size_t)(t + m * T) * N] = v[m];
}

// Column pass (COL_PM) with transposed tiles.  The block's W columns are read with
// coalesced row segments and written transposed into shared memory (one region per
// column, odd stride: conflict-free); each lane group of T threads then transforms one
// whole column with only warp-level synchronisation, exactly like a row, applies P_M with
// the transposed modulus strip, and the result leaves through the same regions with
// coalesced stores.  Two block barriers per tile.
template <class P>
__host__ __device__ constexpr int colt_stride() { return pad_elems_p<P>() | 1; }

// Column pass with two adjacent columns per thread: the column loads and stores, the
// modulus reads and every shared-memory exchange move 16 bytes at a time, and the two
// columns' transforms run on packed pairs (cpk), one two-lane instruction per step of both;
// per column the operations are those of k_col's transform for the same plan, rounded the
// same way lane by lane, except that products with the radix-8 constants are fused into
// the butterfly's additions.
template <class P, int W>
__global__ void __launch_bounds__((W / 2) * P::T, ((W / 2) * P::T <= 512 ? 2 : 1)) k_col2(ColArgs a) {
  constexpr int N = P::N, E = P::E, T = P::T, WP = W / 2, STRIPS = N / W;
  extern __shared__ __align__(16) float2 smem2[];
  cpk* tile = reinterpret_cast<cpk*>(smem2);
  float* Ms = reinterpret_cast<float*>(smem2 + (size_t)N * W);
  const int cp = threadIdx.x % WP, t = threadIdx.x / WP;
  const int img = blockIdx.x / STRIPS, strip = blockIdx.x % STRIPS;
  cpair* base = reinterpret_cast<cpair*>(a.data + (size_t)img * N * N + strip * W) + cp;
  const BlockSync sync;
  {
    constexpr int CH = W / 4;  // 16-byte chunks per row of the strip
    for (int k = threadIdx.x; k < N * CH; k += blockDim.x) {
      const int row = k / CH, q = k % CH;
      cp_async16(Ms + row * W + 4 * q, m_of(a, img, N) + (size_t)row * N + strip * W + 4 * q);
    }
    cp_async_commit();
  }
  cpk v[E];
#pragma unroll
  for (int m = 0; m < E; ++m) v[m] = pack_pair(base[(size_t)(t + m * T) * (N / 2)]);
  fft_plan<P, -1, false, WP, false>(v, tile + cp, t, a.tw, sync);
  cp_async_wait_all();
  sync();  // also ends the transform's shared-memory reads
  constexpr float inv_n = 1.0f / N;
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const float2 mv = *reinterpret_cast<const float2*>(Ms + (t + m * T) * W + 2 * cp);
    cpair q = unpack_pair(v[m]);
    q.a = pm_value(q.a, mv.x, inv_n);
    q.b = pm_value(q.b, mv.y, inv_n);
    v[m] = pack_pair(q);
  }
  fft_plan<P, +1, false, WP, false>(v, tile + cp, t, a.tw, sync);
#pragma unroll
  for (int m = 0; m < E; ++m) base[(size_t)(t + m * T) * (N / 2)] = unpack_pair(v[m]);
}

template <class P, int W>
__global__ void __launch_bounds__(W * P::T, (W * P::T <= 512 ? 2 : 1)) k_colT(ColArgs a) {
  constexpr int N = P::N, E = P::E, T = P::T, STRIPS = N / W, RS = colt_stride<P>(), MS = N + 1;
  extern __shared__ float2 smem[];
  float2* reg = smem;                                           // W regions of RS
  float* MsT = reinterpret_cast<float*>(smem + (size_t)W * RS);  // W x MS
  const int img = blockIdx.x / STRIPS, strip = blockIdx.x % STRIPS;
  float2* base = a.data + (size_t)img * N * N + strip * W;
  const float* Mb = m_of(a, img, N) + strip * W;
  // phase A: coalesced loads (lanes along the columns), transposed writes
  {
    const int ca = threadIdx.x % W, ra = threadIdx.x / W;
#pragma unroll
    for (int k = 0; k < E; ++k) {
      const int row = ra + k * T;
      reg[ca * RS + row] = base[(size_t)row * N + ca];
      MsT[ca * MS + row] = __ldg(&Mb[(size_t)row * N + ca]);
    }
  }
  __syncthreads();
  // phase B: one lane group per column
  {
    const int cb = threadIdx.x / T, t = threadIdx.x % T;
    float2* col = reg + cb * RS;
    const float* mc = MsT + cb * MS;
    const auto sync = GroupSync<T>::make();
    float2 v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = col[t + m * T];
    sync();
    fft_plan<P, -1, true, 1>(v, col, t, a.tw, sync);
    constexpr float inv_n = 1.0f / N;
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const float Mv = mc[t + m * T];
      const float2 X = v[m];
      v[m] = pm_value(X, Mv, inv_n);
    }
    fft_plan<P, +1, true, 1>(v, col, t, a.tw, sync);
#pragma unroll
    for (int m = 0; m < E; ++m) col[t + m * T] = v[m];
  }
  __syncthreads();
  // phase C: coalesced stores
  {
    const int ca = threadIdx.x % W, ra = threadIdx.x / W;
#pragma unroll
    for (int k = 0; k < E; ++k) {
      const int row = ra + k * T;
      base[(size_t)row * N + ca] = reg[ca * RS + row];
    }
  }
}

template <class P, int W>
inline spring_status colT_launch(const FftOp& op, cudaStream_t s, bool prepare_only) {
  constexpr int N = P::N;
  const size_t smem = (size_t)W * colt_stride<P>() * sizeof(float2) + (size_t)W * (N + 1) * sizeof(float);
  if (prepare_only) return allow_smem(k_colT<P, W>, smem);
  if (op.ca.batch < 1) return SPRING_OK;
  launch_begin(op.kclass, s);
  k_colT<P, W><<<op.ca.batch * (N / W), W * P::T, smem, s>>>(op.ca);
  SPRING_CHECK_LAUNCH();
  launch_end(op.kclass, s, op.bytes);
  return SPRING_OK;
}

// rows of one TMA box of the column pass: the largest divisor of N of at most 256 (a box
// dimension is limited to 256 elements)
__host__ __device__ constexpr int tma_box_rows(int n) {
  int r = n < 256 ? n : 256;
  while (n % r) --r;
  return r;
}

// Persistent column pass (COL_PM) fed by TMA.  Tiles (image, 16- or 8-column strip) are
// taken in a grid-stride sequence; the next tile's bulk tensor copy into the second
// shared buffer is issued before the current tile is transformed, so HBM reads overlap the
// transforms.  The tile buffer is also the transform's exchange area.  Waits are bounded;
// a timeout sets bit 2 of *status and the block returns.
template <class P, int W>
__global__ void __launch_bounds__(W * P::T, (W * P::T <= 256 ? 2 : 1))
    k_col_pm_tma(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap mmap,
                 ColArgs a, int ntiles, int* status) {
  constexpr int N = P::N, E = P::E, T = P::T, STRIPS = N / W;
  constexpr int BOXR = tma_box_rows(N), NBOX = N / BOXR;
  constexpr uint32_t TILE_BYTES = (uint32_t)N * W * 8 + (uint32_t)N * W * 4;  // w tile + M strip
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // TMA destinations 1024-byte aligned (the launch reserves the slack)
  float2* const buf0 = reinterpret_cast<float2*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  float2* const buf1 = buf0 + N * W;
  float* const mb0 = reinterpret_cast<float*>(buf1 + N * W);
  float* const mb1 = mb0 + N * W;
  __shared__ __align__(8) uint64_t mbar[2];
  const int c = threadIdx.x % W, t = threadIdx.x / W;
  if (threadIdx.x == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  auto issue = [&](int tile, int b) {
    const int img = tile / STRIPS, strip = tile % STRIPS;
    float2* dst = b ? buf1 : buf0;
    float* mdst = b ? mb1 : mb0;
    mbar_arrive_expect_tx(&mbar[b], TILE_BYTES);
#pragma unroll
    for (int k = 0; k < NBOX; ++k) {
      tma_load_3d(dst + k * BOXR * W, &tmap, strip * 2 * W, k * BOXR, img, &mbar[b]);
      tma_load_3d(mdst + k * BOXR * W, &mmap, strip * W, k * BOXR, a.m_group > 0 ? (a.img0 + img) / a.m_group : 0,
                  &mbar[b]);
    }
  };
  int tile = blockIdx.x;
  if (threadIdx.x == 0 && tile < ntiles) issue(tile, 0);
  const BlockSync sync;
  constexpr float inv_n = 1.0f / N;
  for (int it = 0; tile < ntiles; tile += gridDim.x, ++it) {
    const int b = it & 1;
    const int nxt = tile + gridDim.x;
    if (threadIdx.x == 0 && nxt < ntiles) {
      fence_proxy_async_smem();  // the other buffer's last generic accesses precede the copy
      issue(nxt, b ^ 1);
    }
    const bool ok = __syncthreads_and(mbar_wait_bounded(&mbar[b], (uint32_t)(it >> 1) & 1u));
    if (!ok) {
      if (threadIdx.x == 0) {
        atomicOr(status, 2);
        if (nxt < ntiles) mbar_wait_bounded(&mbar[b ^ 1], (uint32_t)((it + 1) >> 1) & 1u);
      }
      return;
    }
    float2* cur = b ? buf1 : buf0;
    const float* Mcur = b ? mb1 : mb0;
    float2 v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = cur[(t + m * T) * W + c];
    sync();  // every thread has its inputs before the exchange overwrites the tile
    fft_plan<P, -1, false, W>(v, cur + c, t, a.tw, sync);
    const int img = tile / STRIPS, col = (tile % STRIPS) * W + c;
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const float Mv = Mcur[(t + m * T) * W + c];
      const float2 X = v[m];
      v[m] = pm_value(X, Mv, inv_n);
    }
    fft_plan<P, +1, false, W>(v, cur + c, t, a.tw, sync);
    float2* base = a.data + (size_t)img * N * N + col;
#pragma unroll
    for (int m = 0; m < E; ++m) base[(size_t)(t + m * T) * N] = v[m];
    sync();  // this buffer is free for the copy issued in the next iteration
  }
}

// ------------------------------------------------------------------ launch helpers
// raise the kernel's dynamic shared-memory limit to `bytes` (always: static shared
// memory counts against the default 48 KB limit too)
template <class K>
inline spring_status allow_smem(K kernel, size_t bytes) {
  SPRING_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return SPRING_OK;
}

template <class P, int MODE, int ALG, bool LATE, int MINB, bool STAGE = false, class ST = float2>
inline spring_status row_launch(const FftOp& op, cudaStream_t s, bool prepare_only) {
  constexpr int G = ROW_THREADS / P::T;
  const size_t smem = (size_t)G * (pad_elems_p<P>() + (STAGE ? stage_elems<P>() : 0)) * sizeof(float2);
  if (prepare_only) return allow_smem(k_row<P, MODE, ALG, LATE, MINB, STAGE, ST>, smem);
  if (STAGE && (reinterpret_cast<uintptr_t>(op.ra.x) & 15u))
    return invalid("the staged row pass copies x in 16-byte pieces: x must be 16-byte aligned");
  long long blocks = (op.ra.nrows + G - 1) / G;
  const long long cap = 64LL * sm_count();
  if (blocks > cap) blocks = cap;
  if (blocks < 1) return SPRING_OK;
  launch_begin(op.kclass, s);
  k_row<P, MODE, ALG, LATE, MINB, STAGE, ST><<<(int)blocks, ROW_THREADS, smem, s>>>(op.ra);
  SPRING_CHECK_LAUNCH();
  launch_end(op.kclass, s, op.bytes);
  return SPRING_OK;
}

// shared memory of a column tile of W columns with its modulus strip
template <class P>
__host__ __device__ constexpr size_t col_tile_bytes(int w) {
  return (size_t)P::N * w * (sizeof(float2) + sizeof(float));
}

// columns per tile for a block of `threads` threads on plan P, if that tile is usable (whole
// 16-byte chunks of the modulus strip, whole tiles per image, within shared memory); else 0
template <class P>
constexpr int col_w_for(int threads) {
  const int w = threads / P::T;
  return (w >= 4 && w % 4 == 0 && P::N % w == 0 && col_tile_bytes<P>(w) <= 216 * 1024) ? w : 0;
}

template <int N, int W>
constexpr int fit_w() {  // keep the column tile and its modulus strip within shared memory and 1024 threads
  return (col_tile_bytes<Plan<N>>(W) > 216 * 1024 || W * Plan<N>::T > 1024) ? W / 2 : W;
}

template <int N>
constexpr int fit_w_pair() {  // 16-column tiles while two blocks (tile + modulus strip) fit an SM
  return col_tile_bytes<AltPlan<N>>(16) > 108 * 1024 ? 8 : 16;
}

template <int N>
constexpr int tma_w() {  // the TMA pass holds two tiles and two modulus strips
  return (size_t)2 * N * 16 * 12 + 1024 > 220 * 1024 ? 8 : 16;
}

template <int N, int W>
constexpr int fit_w2() {  // paired tile: shared memory and at most 1024 threads
  return (col_tile_bytes<Col2Plan<N>>(W) > 216 * 1024 || (W / 2) * Col2Plan<N>::T > 1024) ? W / 2 : W;
}

template <class P, int W>
inline spring_status col2_launch(const FftOp& op, cudaStream_t s, bool prepare_only) {
  const size_t smem = col_tile_bytes<P>(W);
  if (prepare_only) return allow_smem(k_col2<P, W>, smem);
  if (op.ca.batch < 1) return SPRING_OK;
  launch_begin(op.kclass, s);
  k_col2<P, W><<<op.ca.batch * (P::N / W), (W / 2) * P::T, smem, s>>>(op.ca);
  SPRING_CHECK_LAUNCH();
  launch_end(op.kclass, s, op.bytes);
  return SPRING_OK;
}

template <class P, int W, int MODE, class ST = float2, int MINB = (W * P::T <= 512 ? 2 : 1)>
inline spring_status col_launch(const FftOp& op, cudaStream_t s, bool prepare_only) {
  const size_t smem = (size_t)P::N * W * sizeof(float2) +
                      ((MODE == COL_PM || MODE == COL_ERR) ? (size_t)P::N * W * sizeof(float) : 0);
  auto kern = k_col<P, W, MODE, ST, MINB>;
  if (prepare_only) return allow_smem(kern, smem);
  if (op.ca.batch < 1) return SPRING_OK;
  launch_begin(op.kclass, s);
  kern<<<op.ca.batch * (P::N / W), W * P::T, smem, s>>>(op.ca);
  SPRING_CHECK_LAUNCH();
  launch_end(op.kclass, s, op.bytes);
  return SPRING_OK;
}

// the TMA column pass: tensor map of the batch (floats: 2N x N x batch), box 2W x min(N,256)
template <class P, int W>
inline spring_status col_pm_tma_launch(const FftOp& op, cudaStream_t s, bool prepare_only) {
  constexpr int N = P::N, BOXR = tma_box_rows(N);
  const size_t smem = (size_t)2 * N * W * (sizeof(float2) + sizeof(float)) + 1024;
  if (prepare_only) return allow_smem(k_col_pm_tma<P, W>, smem);
  if (op.ca.batch < 1) return SPRING_OK;
  CUtensorMap map, mmap;
  SPRING_TRY(encode_tmap_f32_3d(&map, op.ca.data, 2 * N, N, op.ca.batch, 2 * W, BOXR));
  const int nm = op.ca.m_group > 0 ? (op.ca.batch + op.ca.m_group - 1) / op.ca.m_group : 1;
  SPRING_TRY(encode_tmap_f32_3d(&mmap, op.ca.M, N, N, nm, W, BOXR));
  static int per_sm = 0;
  if (!per_sm) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_col_pm_tma<P, W>, W * P::T, smem);
    if (per_sm < 1) per_sm = 1;
  }
  const int ntiles = op.ca.batch * (N / W);
  const int blocks = ntiles < per_sm * sm_count() ? ntiles : per_sm * sm_count();
  DeviceTables tb;
  SPRING_TRY(device_tables(&tb));
  launch_begin(op.kclass, s);
  k_col_pm_tma<P, W><<<blocks, W * P::T, smem, s>>>(map, mmap, op.ca, ntiles, tb.status);
  SPRING_CHECK_LAUNCH();
  launch_end(op.kclass, s, op.bytes);
  return SPRING_OK;
}

// blocks of the row-group kernel: 256 threads at Q = 2 (registers allow four per SM), 128 at
// Q = 3 (the parking slots of two more rows per group make shared memory the limit)
template <int N> constexpr int row_group_threads() { return split_q<N>() == 2 ? ROW_THREADS : 128; }
template <int N, int MODE> constexpr int row_group_minb() {
  return split_q<N>() == 2 ? (MODE == ROW_ITER ? 4 : 3) : 4;
}

template <int N, int MODE, int ALG>
inline spring_status row_group_launch(const FftOp& op, cudaStream_t s, bool prep) {
  using P = SplitRowPlan<N>;
  constexpr int BT = row_group_threads<N>(), G = BT / P::T, Q = split_q<N>();
  const size_t smem = (size_t)G * (pad_elems_p<P>() + (Q - 1) * P::N) * sizeof(float2);
  auto kern = k_row_group<P, MODE, ALG, BT, row_group_minb<N, MODE>()>;
  if (prep) return allow_smem(kern, smem);
  long long blocks = (op.sa.nsets + G - 1) / G;
  const long long cap = 64LL * sm_count();
  if (blocks > cap) blocks = cap;
  if (blocks < 1) return SPRING_OK;
  launch_begin(op.kclass, s);
  kern<<<(int)blocks, BT, smem, s>>>(op.sa);
  SPRING_CHECK_LAUNCH();
  launch_end(op.kclass, s, op.bytes);
  return SPRING_OK;
}

template <int N, int MODE, int ALG>
inline spring_status row_split_launch(const FftOp& op, cudaStream_t s, bool prep) {
  if constexpr (split_q<N>() <= 3) {  // all rows of a set in one lane group
    return row_group_launch<N, MODE, ALG>(op, s, prep);
  } else {
    using P = SplitRowPlan<N>;
    constexpr bool STAGE = MODE == ROW_ITER;
    const size_t smem = split_row_elems<P, STAGE>() * sizeof(float2);
    auto kern = k_row_split<P, MODE, ALG, STAGE>;
    if (prep) return allow_smem(kern, smem);
    const long long sets = op.sa.nsets;
    if (sets < 1) return SPRING_OK;
    if (STAGE && ((reinterpret_cast<uintptr_t>(op.sa.w) | reinterpret_cast<uintptr_t>(op.sa.x) |
                   reinterpret_cast<uintptr_t>(op.sa.Sb)) & 15u))
      return invalid("the split row pass stages from 16-byte aligned w, x and support bits");
    int per_sm = 0;
    SPRING_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, split_q<N>() * P::T, smem));
    if (per_sm < 1) return invalid("split row pass does not fit an SM");
    const long long cap = (long long)per_sm * sm_count() * (STAGE ? 1 : 4);  // staged: persistent
    const int blocks = (int)(sets < cap ? sets : cap);
    launch_begin(op.kclass, s);
    kern<<<blocks, split_q<N>() * P::T, smem, s>>>(op.sa);
    SPRING_CHECK_LAUNCH();
    launch_end(op.kclass, s, op.bytes);
    return SPRING_OK;
  }
}

template <int N>
inline spring_status col_split_launch(const FftOp& op, cudaStream_t s, bool prep) {
  using PL = Plan<N / split_q<N>()>;
  constexpr int W = split_col_w<PL::N>();
  const size_t smem = (size_t)PL::N * W * (sizeof(float2) + sizeof(float));
  auto kern = k_col_split<PL, N, W>;
  if (prep) return allow_smem(kern, smem);
  if (op.ca.batch < 1) return SPRING_OK;
  launch_begin(op.kclass, s);
  kern<<<op.ca.batch * split_q<N>() * (N / W), W * PL::T, smem, s>>>(op.ca);
  SPRING_CHECK_LAUNCH();
  launch_end(op.kclass, s, op.bytes);
  return SPRING_OK;
}

template <int N, int ALG>
inline spring_status row_iter_variant(const FftOp& op, cudaStream_t s, bool prep) {
  switch (op.variant) {
    case 0: return row_launch<Plan<N>, ROW_ITER, ALG, false, 1>(op, s, prep);
    case 1: return row_launch<Plan<N>, ROW_ITER, ALG, true, 2>(op, s, prep);
    case 2: return row_launch<Plan<N>, ROW_ITER, ALG, true, 3>(op, s, prep);
    case 3: return row_launch<Plan<N>, ROW_ITER, ALG, true, 2, true>(op, s, prep);
    case 4: return row_launch<Plan<N>, ROW_ITER, ALG, true, 3, true>(op, s, prep);
    case 5: return row_launch<RowAltPlan<N>, ROW_ITER, ALG, true, 2>(op, s, prep);
    default: return row_launch<RowAltPlan<N>, ROW_ITER, ALG, true, 4>(op, s, prep);
  }
}

template <int N, int MODE>
inline spring_status col_variant(const FftOp& op, cudaStream_t s, bool prep) {
  switch (op.variant) {
    case 0: return col_launch<Plan<N>, 16, MODE>(op, s, prep);
    case 1: return col_launch<AltPlan<N>, fit_w_pair<N>(), MODE>(op, s, prep);
    case 2: return col_launch<Plan<N>, fit_w<N, 32>(), MODE>(op, s, prep);
    case 3: return col_launch<Plan<N>, 8, MODE>(op, s, prep);
    case 4:
      if constexpr (MODE == COL_PM) return col_pm_tma_launch<Plan<N>, tma_w<N>()>(op, s, prep);
      return col_launch<Plan<N>, 16, MODE>(op, s, prep);
    case 5:
      if constexpr (MODE == COL_PM) return col_pm_tma_launch<Plan<N>, 8>(op, s, prep);
      return col_launch<Plan<N>, 8, MODE>(op, s, prep);
    case 6:
      if constexpr (MODE == COL_PM) return colT_launch<Plan<N>, (N >= 1024 ? 8 : 16)>(op, s, prep);
      return col_launch<Plan<N>, 16, MODE>(op, s, prep);
    case 7:
      if constexpr (MODE == COL_PM) return colT_launch<Plan<N>, (N >= 512 ? 8 : 32)>(op, s, prep);
      return col_launch<Plan<N>, 16, MODE>(op, s, prep);
    case 8:
      if constexpr (MODE == COL_PM) return col2_launch<Col2Plan<N>, 16>(op, s, prep);
      return col_launch<Plan<N>, 16, MODE>(op, s, prep);
    case 9:
      if constexpr (MODE == COL_PM) return col2_launch<Col2Plan<N>, fit_w2<N, 32>()>(op, s, prep);
      return col_launch<Plan<N>, 16, MODE>(op, s, prep);
    default:  // the alternative plan in 512-thread blocks held to 3 per SM (48 warps: 40 registers)
      if constexpr (MODE == COL_PM) {
        constexpr int W = col_w_for<AltPlan<N>>(512);
        if constexpr (W > 0) return col_launch<AltPlan<N>, W, MODE, float2, 3>(op, s, prep);
      }
      return col_launch<Plan<N>, 16, MODE>(op, s, prep);
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
    case OP_ROW_ITER16:
      // the FP32 path's fastest shapes at 1024: 16 elements per thread, 8-column tiles
      if (op.alg == 0) return row_launch<Row16Plan<N>, ROW_ITER, 0, true, 2, false, __half2>(op, s, prep);
      if (op.alg == 1) return row_launch<Row16Plan<N>, ROW_ITER, 1, true, 2, false, __half2>(op, s, prep);
      return row_launch<Row16Plan<N>, ROW_ITER, 2, true, 2, false, __half2>(op, s, prep);
    case OP_COL_PM16: return col_launch<Col16Plan<N>, (N >= 1024 ? 8 : 16), COL_PM, __half2>(op, s, prep);
    case OP_ROW_INIT16: return row_launch<Plan<N>, ROW_INIT16, 0, false, 1>(op, s, prep);
    case OP_ROW_SPLIT:
    case OP_ROW_SPLIT_FWD:
    case OP_COL_SPLIT:
      if constexpr (split_side(N)) {
        if (op.kind == OP_COL_SPLIT) return col_split_launch<N>(op, s, prep);
        if (op.kind == OP_ROW_SPLIT_FWD) return row_split_launch<N, ROW_FWD, 0>(op, s, prep);
        if (op.alg == 0) return row_split_launch<N, ROW_ITER, 0>(op, s, prep);
        if (op.alg == 1) return row_split_launch<N, ROW_ITER, 1>(op, s, prep);
        return row_split_launch<N, ROW_ITER, 2>(op, s, prep);
      }
      return invalid("the split passes cover sides 192, 384, 512, 768 and 1024");
  }
  return invalid("unknown transform operation");
}

}  // namespace spring
