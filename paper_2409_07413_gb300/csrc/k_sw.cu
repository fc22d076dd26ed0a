// k_sw.cu -- shrink-wrap support updates (Sec. "The phase problem and conventional
// approaches", Eq. shrinkwrap; App. "The modified Shrink-wrap").
//
//   rho_sigma = G_sigma (*) |x|            separable, periodic, taps d = -r..r, r = ceil(4 sigma)
//   UpdateSupport:      S = [rho_sigma >= tau max rho_sigma]   (threshold compared in FP64)
//   UpdateSupportSize:  S = the alpha largest rho_sigma, equal values by lower linear index
//                       (radix select on the float bit patterns: exact, deterministic)
#include <cmath>
#include <vector>

#include "internal.h"

namespace spring {

struct Taps {
  float w[2 * SW_MAX_RADIUS + 1];
  int r;
};

// pass 1: |x| along rows -> tmp.  One block per row: |x| is computed once per pixel into
// a shared row extended by a periodic halo of r pixels on each side, so each tap is a
// plain shared-memory read.
constexpr int SW_ROW_THREADS = 256;

__global__ void __launch_bounds__(SW_ROW_THREADS) k_smooth_rows(const float2* __restrict__ x,
                                                                float* __restrict__ tmp, int n,
                                                                const Taps taps) {
  extern __shared__ float ext[];  // n + 2 r
  const long long row0 = (long long)blockIdx.x * n;
  const int r = taps.r, len = n + 2 * r;
  for (int k = threadIdx.x; k < len; k += blockDim.x) {
    int c = k - r;
    c %= n;
    if (c < 0) c += n;
    const float2 v = __ldg(&x[row0 + c]);
    ext[k] = sqrtf(v.x * v.x + v.y * v.y);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    float acc = 0.f;
    for (int d = 0; d <= 2 * r; ++d) acc = fmaf(taps.w[d], ext[c + d], acc);
    tmp[row0 + c] = acc;
  }
}

// pass 2: along columns -> out, and the per-image maximum.  A block smooths a tile of
// 32 columns x SW_TILE_ROWS rows from a shared copy of those columns with r halo rows
// above and below (periodic).  Non-negative floats compare like their bit patterns, so an
// integer atomicMax gives the exact maximum in any order.
constexpr int SW_TILE_ROWS = 64;

__global__ void __launch_bounds__(256) k_smooth_cols(const float* __restrict__ tmp, float* __restrict__ out,
                                                     int n, const Taps taps, unsigned* __restrict__ img_max) {
  extern __shared__ float tile[];  // (SW_TILE_ROWS + 2 r) x 32
  const int r = taps.r;
  const int tiles_x = n / 32, tiles_y = (n + SW_TILE_ROWS - 1) / SW_TILE_ROWS;
  const int img = blockIdx.x / (tiles_x * tiles_y);
  const int rem = blockIdx.x % (tiles_x * tiles_y);
  const int c0 = (rem % tiles_x) * 32, r0 = (rem / tiles_x) * SW_TILE_ROWS;
  const int rows_out = min(SW_TILE_ROWS, n - r0), rows_in = rows_out + 2 * r;
  const long long base = (long long)img * n * n;
  const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;  // 32 x 8 threads
  for (int k = ly; k < rows_in; k += 8) {
    int rr = r0 - r + k;
    rr %= n;
    if (rr < 0) rr += n;
    tile[k * 32 + lx] = __ldg(&tmp[base + (long long)rr * n + c0 + lx]);
  }
  __syncthreads();
  unsigned vmax = 0u;
  for (int k = ly; k < rows_out; k += 8) {
    float acc = 0.f;
    for (int d = 0; d <= 2 * r; ++d) acc = fmaf(taps.w[d], tile[(k + d) * 32 + lx], acc);
    out[base + (long long)(r0 + k) * n + c0 + lx] = acc;
    vmax = max(vmax, __float_as_uint(fmaxf(acc, 0.f)));
  }
  if (img_max) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) vmax = max(vmax, __shfl_down_sync(0xffffffffu, vmax, o));
    if (lx == 0) atomicMax(&img_max[img], vmax);
  }
}

// Radius-specialised passes (r = R <= 8, i.e. sigma <= 2): taps in registers and a sliding
// window, so each output costs 2R+1 FMAs and about one shared-memory read.  The sum of each
// output runs over d = 0..2R in the same order as in the general kernels (same bits).
constexpr int SW_RK = 4;  // row outputs per thread

template <int R>
__global__ void __launch_bounds__(256) k_smooth_rows_r(const float2* __restrict__ x, float* __restrict__ tmp,
                                                       int n, long long nrows, const Taps taps) {
  extern __shared__ float ext_r[];  // rows_per_block x (n + 2R)
  const int tpr = n / SW_RK;                   // threads per row
  const int rpb = blockDim.x / tpr;            // rows per block
  const int lr = threadIdx.x / tpr, lt = threadIdx.x % tpr;
  const long long row = (long long)blockIdx.x * rpb + lr;
  const int len = n + 2 * R;
  float* ext = ext_r + lr * len;
  float w[2 * R + 1];
#pragma unroll
  for (int d = 0; d <= 2 * R; ++d) w[d] = taps.w[d];
  if (row < nrows) {
    const long long row0 = row * n;
    for (int k = lt; k < len; k += tpr) {
      int c = k - R;
      c %= n;
      if (c < 0) c += n;
      const float2 v = __ldg(&x[row0 + c]);
      ext[k] = sqrtf(v.x * v.x + v.y * v.y);
    }
  }
  __syncthreads();
  if (row >= nrows || lr >= rpb) return;
  const int c0 = lt * SW_RK;
  float win[SW_RK + 2 * R];
#pragma unroll
  for (int k = 0; k < SW_RK + 2 * R; ++k) win[k] = ext[c0 + k];
  float4 o;
  float* op = &o.x;
#pragma unroll
  for (int j = 0; j < SW_RK; ++j) {
    float acc = 0.f;
#pragma unroll
    for (int d = 0; d <= 2 * R; ++d) acc = fmaf(w[d], win[j + d], acc);
    op[j] = acc;
  }
  *reinterpret_cast<float4*>(&tmp[row * n + c0]) = o;
}

constexpr int SW_CK = 8;  // column outputs per thread

template <int R>
__global__ void __launch_bounds__(256) k_smooth_cols_r(const float* __restrict__ tmp, float* __restrict__ out,
                                                       int n, const Taps taps, unsigned* __restrict__ img_max) {
  extern __shared__ float tile_r[];  // (SW_TILE_ROWS + 2R) x 32
  const int tiles_x = n / 32, tiles_y = (n + SW_TILE_ROWS - 1) / SW_TILE_ROWS;
  const int img = blockIdx.x / (tiles_x * tiles_y);
  const int rem = blockIdx.x % (tiles_x * tiles_y);
  const int c0 = (rem % tiles_x) * 32, r0 = (rem / tiles_x) * SW_TILE_ROWS;
  const int rows_out = min(SW_TILE_ROWS, n - r0), rows_in = rows_out + 2 * R;
  const long long base = (long long)img * n * n;
  const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;  // 32 x 8 threads
  for (int k = ly; k < rows_in; k += 8) {
    int rr = r0 - R + k;
    rr %= n;
    if (rr < 0) rr += n;
    tile_r[k * 32 + lx] = __ldg(&tmp[base + (long long)rr * n + c0 + lx]);
  }
  float w[2 * R + 1];
#pragma unroll
  for (int d = 0; d <= 2 * R; ++d) w[d] = taps.w[d];
  __syncthreads();
  unsigned vmax = 0u;
  const int k0 = ly * SW_CK;  // 8 consecutive output rows per thread
  if (k0 < rows_out) {
    float win[SW_CK + 2 * R];
#pragma unroll
    for (int k = 0; k < SW_CK + 2 * R; ++k) win[k] = (k0 + k < rows_in) ? tile_r[(k0 + k) * 32 + lx] : 0.f;
#pragma unroll
    for (int j = 0; j < SW_CK; ++j) {
      if (k0 + j < rows_out) {
        float acc = 0.f;
#pragma unroll
        for (int d = 0; d <= 2 * R; ++d) acc = fmaf(w[d], win[j + d], acc);
        out[base + (long long)(r0 + k0 + j) * n + c0 + lx] = acc;
        vmax = max(vmax, __float_as_uint(fmaxf(acc, 0.f)));
      }
    }
  }
  if (img_max) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) vmax = max(vmax, __shfl_down_sync(0xffffffffu, vmax, o));
    if (lx == 0) atomicMax(&img_max[img], vmax);
  }
}

template <int R>
static spring_status smooth_r(int n, const float2* x, float* tmp, float* out, int batch, const Taps& taps,
                              unsigned* img_max, cudaStream_t s) {
  const long long total = (long long)batch * n * n, nrows = (long long)batch * n;
  const int tpr = n / SW_RK, rpb = 256 / tpr > 0 ? 256 / tpr : 1;
  const size_t row_smem = sizeof(float) * rpb * (n + 2 * R);
  const size_t col_smem = sizeof(float) * 32 * (SW_TILE_ROWS + 2 * R);
  launch_begin(SPRING_KC_OTHER, s);
  k_smooth_rows_r<R><<<(int)((nrows + rpb - 1) / rpb), rpb * tpr, row_smem, s>>>(x, tmp, n, nrows, taps);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, total * 12.0);
  const int tiles = (n / 32) * ((n + SW_TILE_ROWS - 1) / SW_TILE_ROWS);
  launch_begin(SPRING_KC_OTHER, s);
  k_smooth_cols_r<R><<<batch * tiles, 256, col_smem, s>>>(tmp, out, n, taps, img_max);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, total * 8.0);
  return SPRING_OK;
}

// S = [rho_sigma >= tau max].  The comparison is decided exactly as in FP64: with
// t = tau * max in double, (double)v >= t holds for a float v iff v >= f, f the smallest
// float not below t; f is formed once per block.
constexpr int SW_THR_PER_BLOCK = 1024;

__global__ void k_threshold(const float* __restrict__ sm, const unsigned* __restrict__ img_max,
                            double tau, uint8_t* __restrict__ S, long long nn) {
  __shared__ float f_s;
  const long long first = (long long)blockIdx.x * SW_THR_PER_BLOCK;  // blocks never straddle images
  if (threadIdx.x == 0) {
    const double t = tau * (double)__uint_as_float(img_max[first / nn]);
    float f = (float)t;
    if ((double)f < t) f = nextafterf(f, INFINITY);
    f_s = f;
  }
  __syncthreads();
  const float f = f_s;
  for (int k = threadIdx.x; k < SW_THR_PER_BLOCK; k += blockDim.x) S[first + k] = sm[first + k] >= f ? 1 : 0;
}

static Taps make_taps(float sigma) {
  Taps t{};
  if (!(sigma > 0.f)) {
    t.r = 0;
    t.w[0] = 1.f;
    return t;
  }
  const double sg = sigma;
  int r = (int)std::ceil(4.0 * sg);
  if (r > SW_MAX_RADIUS) r = SW_MAX_RADIUS;
  std::vector<double> w(2 * r + 1);
  double s = 0.0;
  for (int d = -r; d <= r; ++d) s += (w[d + r] = std::exp(-(double)d * d / (2.0 * sg * sg)));
  for (int d = -r; d <= r; ++d) t.w[d + r] = (float)(w[d + r] / s);
  t.r = r;
  return t;
}

spring_status launch_smooth(int n, const float2* x, float* tmp, float* out, int batch, float sigma,
                            unsigned* img_max, cudaStream_t s) {
  if (!(sigma >= 0.f) || sigma > 64.f) return invalid("shrink-wrap sigma must be in [0, 64]");
  const Taps taps = make_taps(sigma);
  const long long total = (long long)batch * n * n;
  if (total == 0) return SPRING_OK;
  if (img_max) SPRING_CUDA(cudaMemsetAsync(img_max, 0, sizeof(unsigned) * batch, s));
  switch (taps.r) {
    case 1: return smooth_r<1>(n, x, tmp, out, batch, taps, img_max, s);
    case 2: return smooth_r<2>(n, x, tmp, out, batch, taps, img_max, s);
    case 3: return smooth_r<3>(n, x, tmp, out, batch, taps, img_max, s);
    case 4: return smooth_r<4>(n, x, tmp, out, batch, taps, img_max, s);
    case 5: return smooth_r<5>(n, x, tmp, out, batch, taps, img_max, s);
    case 6: return smooth_r<6>(n, x, tmp, out, batch, taps, img_max, s);
    case 7: return smooth_r<7>(n, x, tmp, out, batch, taps, img_max, s);
    case 8: return smooth_r<8>(n, x, tmp, out, batch, taps, img_max, s);
    default: break;
  }
  const size_t row_smem = sizeof(float) * (n + 2 * taps.r);
  const size_t col_smem = sizeof(float) * 32 * (SW_TILE_ROWS + 2 * taps.r);
  SPRING_CUDA(cudaFuncSetAttribute(k_smooth_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)col_smem));
  launch_begin(SPRING_KC_OTHER, s);
  k_smooth_rows<<<(int)((long long)batch * n), SW_ROW_THREADS, row_smem, s>>>(x, tmp, n, taps);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, total * 12.0);
  const int tiles = (n / 32) * ((n + SW_TILE_ROWS - 1) / SW_TILE_ROWS);
  launch_begin(SPRING_KC_OTHER, s);
  k_smooth_cols<<<batch * tiles, 256, col_smem, s>>>(tmp, out, n, taps, img_max);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, total * 8.0);
  return SPRING_OK;
}

spring_status launch_threshold(int n, const float* sm, const unsigned* img_max, float tau,
                               uint8_t* S, int batch, cudaStream_t s) {
  const long long nn = (long long)n * n, total = nn * batch;
  if (total == 0) return SPRING_OK;
  launch_begin(SPRING_KC_OTHER, s);
  k_threshold<<<(int)(total / SW_THR_PER_BLOCK), 256, 0, s>>>(sm, img_max, (double)tau, S, nn);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, total * 5.0);
  return SPRING_OK;
}

// ------------------------------------------------------------------ exact-area select
// One block per image.  The alpha-th largest bit pattern is found digit by digit
// (11, 11, 10 bits) from shared-memory histograms; pixels above it are selected, and of
// the pixels equal to it the first (alpha - #above) in linear order.
constexpr int SEL_THREADS = 1024;

__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned* warp_tot, unsigned* total) {
  // exclusive scan over the block in thread order
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    unsigned t = lane < nw ? warp_tot[lane] : 0u;
    unsigned it = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned u = __shfl_up_sync(0xffffffffu, it, o);
      if (lane >= o) it += u;
    }
    if (lane < nw) warp_tot[lane] = it - t;  // exclusive warp offsets
    if (lane == nw - 1) *total = it;
  }
  __syncthreads();
  const unsigned r = warp_tot[warp] + inc - v;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(SEL_THREADS) k_select_area(const float* __restrict__ sm,
                                                             const int64_t* __restrict__ alpha,
                                                             int alpha_stride, int alpha_group,
                                                             uint8_t* __restrict__ S, int n) {
  __shared__ unsigned hist[2048];
  __shared__ unsigned warp_tot[32];
  __shared__ unsigned total;
  __shared__ unsigned sel_digit, sel_above;
  const long long nn = (long long)n * n;
  const unsigned* v = reinterpret_cast<const unsigned*>(sm) + (long long)blockIdx.x * nn;
  uint8_t* out = S + (long long)blockIdx.x * nn;
  long long a = alpha[(long long)(blockIdx.x / alpha_group) * alpha_stride];
  if (a <= 0 || a >= nn) {
    const uint8_t fill = a <= 0 ? 0 : 1;
    for (long long i = threadIdx.x; i < nn; i += blockDim.x) out[i] = fill;
    return;
  }
  unsigned prefix = 0, pmask = 0;
  unsigned k = (unsigned)a;  // rank still to place within the current prefix
  const int shifts[3] = {21, 10, 0};
  const int widths[3] = {11, 11, 10};
  for (int pass = 0; pass < 3; ++pass) {
    const int sh = shifts[pass], nb = 1 << widths[pass];
    for (int b = threadIdx.x; b < 2048; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    for (long long i = threadIdx.x; i < nn; i += blockDim.x) {
      const unsigned u = v[i];
      if ((u & pmask) == prefix) atomicAdd(&hist[(u >> sh) & (nb - 1)], 1u);
    }
    __syncthreads();
    // counts above each digit: scan over digits in decreasing order (two per thread)
    const int d0 = nb - 1 - 2 * threadIdx.x, d1 = d0 - 1;
    const unsigned c0 = (d0 >= 0) ? hist[d0] : 0u, c1 = (d1 >= 0) ? hist[d1] : 0u;
    const unsigned above0 = block_excl_scan(c0 + c1, warp_tot, &total);
    const unsigned above1 = above0 + c0;
    if (d0 >= 0 && above0 < k && k <= above0 + c0) {
      sel_digit = (unsigned)d0;
      sel_above = above0;
    }
    if (d1 >= 0 && above1 < k && k <= above1 + c1) {
      sel_digit = (unsigned)d1;
      sel_above = above1;
    }
    __syncthreads();
    prefix |= sel_digit << sh;
    pmask |= (unsigned)(nb - 1) << sh;
    k -= sel_above;
    __syncthreads();
  }
  // prefix is the alpha-th largest pattern; k pixels equal to it are still to be taken
  unsigned eq_before = 0;
  for (long long i0 = 0; i0 < nn; i0 += blockDim.x) {
    const long long i = i0 + threadIdx.x;
    const unsigned u = (i < nn) ? v[i] : 0u;
    const bool eq = (i < nn) && (u == prefix);
    const int any_eq = __syncthreads_count(eq);
    unsigned rank = 0;
    if (any_eq) rank = block_excl_scan(eq ? 1u : 0u, warp_tot, &total);
    if (i < nn) out[i] = (u > prefix || (eq && eq_before + rank < k)) ? 1 : 0;
    eq_before += (unsigned)any_eq;
  }
}

spring_status launch_select_area(int n, const float* sm, const int64_t* alpha, int alpha_stride,
                                 uint8_t* S, int batch, cudaStream_t s, int alpha_group) {
  if (batch < 1) return SPRING_OK;
  if (alpha_group < 1) return invalid("alpha_group must be >= 1");
  launch_begin(SPRING_KC_OTHER, s);
  k_select_area<<<batch, SEL_THREADS, 0, s>>>(sm, alpha, alpha_stride, alpha_group, S, n);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, (double)batch * n * n * 13.0);
  return SPRING_OK;
}

}  // namespace spring
