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

constexpr int SW_CK = 8;  // column outputs per thread

// Radius-specialised smoothing (r = R <= 8, i.e. sigma <= 2), both passes in one kernel: taps
// in registers, and a block produces a tile of SW_TILE_ROWS rows x 32 columns.  |x| of the
// tile and its periodic halo (R rows above and below, R columns left and right) is read once
// into shared memory, the row sums are formed for every row of the halo'd tile, then the
// column sums from them.  A row sum thread forms four adjacent outputs from a window of
// 2R + 4 values that it reads as 16-byte words (one shared-memory load per output instead of
// 2R + 1).  Each output is summed over d = 0..2R in the same order as in the general
// two-pass kernels above (same bits); the row-smoothed image never goes through HBM.
template <int R>
__global__ void __launch_bounds__(256) k_smooth2d_r(const float2* __restrict__ x, float* __restrict__ out,
                                                    int n, const Taps taps, unsigned* __restrict__ img_max) {
  constexpr int TW = 32, IW = TW + 2 * R, IH = SW_TILE_ROWS + 2 * R;
  constexpr int IWP = (IW + 3) & ~3, NQ = (2 * R + 4 + 3) / 4;  // row pitch; 16-byte words per window
  static_assert(4 * (TW / 4 - 1) + 4 * NQ <= IWP, "every window inside its row");
  __shared__ __align__(16) float a[IH * IWP];  // |x| with halo
  __shared__ __align__(16) float b[IH * TW];   // row sums
  const int tiles_x = n / TW, tiles_y = (n + SW_TILE_ROWS - 1) / SW_TILE_ROWS;
  const int img = blockIdx.x / (tiles_x * tiles_y);
  const int rem = blockIdx.x % (tiles_x * tiles_y);
  const int c0 = (rem % tiles_x) * TW, r0 = (rem / tiles_x) * SW_TILE_ROWS;
  const int rows_out = min(SW_TILE_ROWS, n - r0), rows_in = rows_out + 2 * R;
  const long long base = (long long)img * n * n;
  const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;  // 32 x 8 threads
  // |x| of rows r0 - R .. r0 + rows_out + R - 1 and columns c0 - R .. c0 + TW + R - 1: every
  // load of the warp's rows is issued before the first is used (IW - 32 = 2R < 32 extra
  // columns: two loads per row at most)
  constexpr int KPW = (IH + 7) / 8;  // rows per warp
  int c_a = c0 - R + lx, c_b = c0 - R + 32 + lx;
  c_a = c_a < 0 ? c_a + n : (c_a >= n ? c_a - n : c_a);  // R < n
  c_b = c_b >= n ? c_b - n : c_b;
  const bool has_b = lx < IW - 32;
  float2 va[KPW], vb[KPW];
#pragma unroll
  for (int q = 0; q < KPW; ++q) {
    const int k = ly + 8 * q;
    if (k < rows_in) {
      int rr = r0 - R + k;
      rr = rr < 0 ? rr + n : (rr >= n ? rr - n : rr);
      const float2* row = x + base + (long long)rr * n;
      va[q] = __ldg(&row[c_a]);
      if (has_b) vb[q] = __ldg(&row[c_b]);
    }
  }
#pragma unroll
  for (int q = 0; q < KPW; ++q) {
    const int k = ly + 8 * q;
    if (k < rows_in) {
      a[k * IWP + lx] = sqrtf(va[q].x * va[q].x + va[q].y * va[q].y);
      if (has_b) a[k * IWP + 32 + lx] = sqrtf(vb[q].x * vb[q].x + vb[q].y * vb[q].y);
    }
  }
  float w[2 * R + 1];
#pragma unroll
  for (int d = 0; d <= 2 * R; ++d) w[d] = taps.w[d];
  __syncthreads();
  for (int item = threadIdx.x; item < rows_in * (TW / 4); item += blockDim.x) {
    const int k = item / (TW / 4), j = item % (TW / 4);  // row k, outputs 4 j .. 4 j + 3
    const float4* src = reinterpret_cast<const float4*>(a + k * IWP + 4 * j);
    float win[4 * NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const float4 v = src[q];
      win[4 * q] = v.x;
      win[4 * q + 1] = v.y;
      win[4 * q + 2] = v.z;
      win[4 * q + 3] = v.w;
    }
    float acc[4];
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      acc[o] = 0.f;
#pragma unroll
      for (int d = 0; d <= 2 * R; ++d) acc[o] = fmaf(w[d], win[o + d], acc[o]);
    }
    *reinterpret_cast<float4*>(b + k * TW + 4 * j) = make_float4(acc[0], acc[1], acc[2], acc[3]);
  }
  __syncthreads();
  unsigned vmax = 0u;
  const int k0 = ly * SW_CK;  // 8 consecutive output rows per thread
  if (k0 < rows_out) {
    float win[SW_CK + 2 * R];
#pragma unroll
    for (int k = 0; k < SW_CK + 2 * R; ++k) win[k] = (k0 + k < rows_in) ? b[(k0 + k) * TW + lx] : 0.f;
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
static spring_status smooth_r(int n, const float2* x, float* out, int batch, const Taps& taps,
                              unsigned* img_max, cudaStream_t s) {
  static_assert(SW_TILE_ROWS == 8 * SW_CK, "eight warps of SW_CK output rows cover a tile");
  const long long total = (long long)batch * n * n;
  const int tiles = (n / 32) * ((n + SW_TILE_ROWS - 1) / SW_TILE_ROWS);
  launch_begin(SPRING_KC_OTHER, s);
  k_smooth2d_r<R><<<batch * tiles, 256, 0, s>>>(x, out, n, taps, img_max);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, total * 12.0);
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
  static_assert(SW_THR_PER_BLOCK == 4 * 256, "256 threads x 4 pixels");
  // the thread's 4 consecutive pixels are loaded before the threshold is known
  const float4 v = *reinterpret_cast<const float4*>(sm + first + 4 * threadIdx.x);
  if (threadIdx.x == 0) {
    const double t = tau * (double)__uint_as_float(img_max[first / nn]);
    float f = (float)t;
    if ((double)f < t) f = nextafterf(f, INFINITY);
    f_s = f;
  }
  __syncthreads();
  const float f = f_s;
  uchar4 o;
  o.x = v.x >= f ? 1 : 0;
  o.y = v.y >= f ? 1 : 0;
  o.z = v.z >= f ? 1 : 0;
  o.w = v.w >= f ? 1 : 0;
  *reinterpret_cast<uchar4*>(S + first + 4 * threadIdx.x) = o;
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
    case 1: return smooth_r<1>(n, x, out, batch, taps, img_max, s);
    case 2: return smooth_r<2>(n, x, out, batch, taps, img_max, s);
    case 3: return smooth_r<3>(n, x, out, batch, taps, img_max, s);
    case 4: return smooth_r<4>(n, x, out, batch, taps, img_max, s);
    case 5: return smooth_r<5>(n, x, out, batch, taps, img_max, s);
    case 6: return smooth_r<6>(n, x, out, batch, taps, img_max, s);
    case 7: return smooth_r<7>(n, x, out, batch, taps, img_max, s);
    case 8: return smooth_r<8>(n, x, out, batch, taps, img_max, s);
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
constexpr int SEL_THREADS = 1024;  // digit pick: two digits per thread

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

// The alpha-th largest bit pattern of an image (sm >= 0, so the order of the float values
// is that of their bit patterns) is found digit by digit, 11, 11 and 10 bits, from the
// top.  Each pass histograms the digit over the pixels whose higher digits match the
// prefix found so far: the image is split into chunks of SEL_CHUNK pixels, one block per
// chunk, with block histograms in shared memory (equal bins of a warp merged first) added
// into one global histogram per image; one block per image then picks the digit.  A final
// pair of launches counts, per chunk, the pixels equal to the found pattern and writes S:
// pixels above it are selected, and of those equal to it the first k in linear order.
constexpr int SEL_CHUNK = 16384;
constexpr int SEL_T = 512;
constexpr int SEL_BINS = 2048;

__host__ __device__ constexpr int sel_shift(int pass) { return pass == 0 ? 21 : pass == 1 ? 10 : 0; }
__host__ __device__ constexpr int sel_width(int pass) { return pass == 2 ? 10 : 11; }

struct SelScratch {
  unsigned* ghist;  // [batch][SEL_BINS]
  unsigned* state;  // [batch][4]: prefix, prefix mask, rank still to place, fill (0 none, 1 all 0, 2 all 1)
  unsigned* eqcnt;  // [batch][chunks]
};

static int sel_chunks(long long nn) { return (int)((nn + SEL_CHUNK - 1) / SEL_CHUNK); }

size_t select_area_scratch_bytes(int n, int batch) {
  const long long nn = (long long)n * n;
  return sizeof(unsigned) * (size_t)batch * (SEL_BINS + 4 + sel_chunks(nn));
}

template <int PASS>
__global__ void __launch_bounds__(SEL_T) k_sel_hist(const float* __restrict__ sm, const int64_t* __restrict__ alpha,
                                                    int alpha_stride, int alpha_group, SelScratch sc, long long nn,
                                                    int chunks) {
  __shared__ unsigned hist[SEL_BINS];
  constexpr int sh = sel_shift(PASS), nb = 1 << sel_width(PASS);
  const int img = blockIdx.x / chunks, ch = blockIdx.x % chunks;
  unsigned prefix = 0, pmask = 0;
  if (PASS == 0) {
    const long long a = alpha[(long long)(img / alpha_group) * alpha_stride];
    if (a <= 0 || a >= nn) return;  // filled by the write pass
  } else {
    if (sc.state[4 * img + 3]) return;
    prefix = sc.state[4 * img + 0];
    pmask = sc.state[4 * img + 1];
  }
  for (int b = threadIdx.x; b < nb; b += blockDim.x) hist[b] = 0;
  __syncthreads();
  const unsigned* v = reinterpret_cast<const unsigned*>(sm) + (long long)img * nn;
  const long long lo = (long long)ch * SEL_CHUNK, hi = min(nn, lo + SEL_CHUNK);  // multiples of 4
  const int lane = threadIdx.x & 31;
  // four consecutive pixels per thread (one 16-byte load); every lane takes the same trips
  for (long long b0 = lo; b0 < hi; b0 += 4LL * blockDim.x) {
    const long long i = b0 + 4LL * threadIdx.x;
    const uint4 q = i < hi ? *reinterpret_cast<const uint4*>(v + i) : make_uint4(0u, 0u, 0u, 0u);
    const unsigned us[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const unsigned u = us[e];
      const bool take = i < hi && (u & pmask) == prefix;
      if (PASS > 0 && !__any_sync(0xffffffffu, take)) continue;  // later passes: few pixels match
      const unsigned key = take ? (u >> sh) & (nb - 1) : 0xffffffffu;
      const unsigned same = __match_any_sync(0xffffffffu, key);
      if (take && lane == __ffs(same) - 1) atomicAdd(&hist[key], (unsigned)__popc(same));
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
    if (hist[b]) atomicAdd(&sc.ghist[(long long)img * SEL_BINS + b], hist[b]);
}

template <int PASS>
__global__ void __launch_bounds__(SEL_THREADS) k_sel_digit(const int64_t* __restrict__ alpha, int alpha_stride,
                                                          int alpha_group, SelScratch sc, long long nn) {
  __shared__ unsigned warp_tot[32];
  __shared__ unsigned total;
  __shared__ unsigned sel_digit, sel_above;
  constexpr int sh = sel_shift(PASS), nb = 1 << sel_width(PASS);
  const int img = blockIdx.x;
  unsigned* st = sc.state + 4 * img;
  unsigned* gh = sc.ghist + (long long)img * SEL_BINS;
  unsigned prefix = 0, pmask = 0, k = 0;
  if (PASS == 0) {
    const long long a = alpha[(long long)(img / alpha_group) * alpha_stride];
    if (a <= 0 || a >= nn) {
      if (threadIdx.x == 0) st[3] = a <= 0 ? 1u : 2u;
      return;
    }
    k = (unsigned)a;
  } else {
    if (st[3]) return;
    prefix = st[0];
    pmask = st[1];
    k = st[2];
  }
  // counts above each digit: scan over digits in decreasing order (two per thread)
  const int d0 = nb - 1 - 2 * threadIdx.x, d1 = d0 - 1;
  const unsigned c0 = (d0 >= 0) ? gh[d0] : 0u, c1 = (d1 >= 0) ? gh[d1] : 0u;
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
  if (threadIdx.x == 0) {
    st[0] = prefix | (sel_digit << sh);
    st[1] = pmask | ((unsigned)(nb - 1) << sh);
    st[2] = k - sel_above;
    st[3] = 0u;
  }
  for (int b = threadIdx.x; b < SEL_BINS; b += blockDim.x) gh[b] = 0u;  // clean for the next pass
}

// pixels equal to the found pattern, per chunk
__global__ void __launch_bounds__(SEL_T) k_sel_eqcount(const float* __restrict__ sm, SelScratch sc, long long nn,
                                                       int chunks) {
  __shared__ unsigned cnt;
  const int img = blockIdx.x / chunks, ch = blockIdx.x % chunks;
  if (sc.state[4 * img + 3]) return;
  const unsigned prefix = sc.state[4 * img + 0];
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  const unsigned* v = reinterpret_cast<const unsigned*>(sm) + (long long)img * nn;
  const long long lo = (long long)ch * SEL_CHUNK, hi = min(nn, lo + SEL_CHUNK);
  unsigned c = 0;
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) c += v[i] == prefix ? 1u : 0u;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(&cnt, c);
  __syncthreads();
  if (threadIdx.x == 0) sc.eqcnt[(long long)img * chunks + ch] = cnt;
}

__global__ void __launch_bounds__(SEL_T) k_sel_write(const float* __restrict__ sm, SelScratch sc,
                                                     uint8_t* __restrict__ S, long long nn, int chunks) {
  __shared__ unsigned warp_tot[32];
  __shared__ unsigned total;
  const int img = blockIdx.x / chunks, ch = blockIdx.x % chunks;
  const long long lo = (long long)ch * SEL_CHUNK, hi = min(nn, lo + SEL_CHUNK);
  uint8_t* out = S + (long long)img * nn;
  const unsigned fill = sc.state[4 * img + 3];
  if (fill) {
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) out[i] = fill == 2u ? 1 : 0;
    return;
  }
  const unsigned prefix = sc.state[4 * img + 0], k = sc.state[4 * img + 2];
  unsigned eq_before = 0;
  for (int c = 0; c < ch; ++c) eq_before += sc.eqcnt[(long long)img * chunks + c];
  const unsigned* v = reinterpret_cast<const unsigned*>(sm) + (long long)img * nn;
  // four consecutive pixels per thread; the rank of an equal pixel among the equal pixels
  // of this step is the block's exclusive scan of the per-thread counts plus the equal
  // pixels before it in the thread's four
  for (long long b0 = lo; b0 < hi; b0 += 4LL * blockDim.x) {
    const long long i = b0 + 4LL * threadIdx.x;
    const bool in = i < hi;
    const uint4 q = in ? *reinterpret_cast<const uint4*>(v + i) : make_uint4(0u, 0u, 0u, 0u);
    const unsigned e0 = in && q.x == prefix, e1 = in && q.y == prefix, e2 = in && q.z == prefix,
                   e3 = in && q.w == prefix;
    const unsigned c = e0 + e1 + e2 + e3;
    const int any_eq = __syncthreads_count(c > 0);
    unsigned r = 0, step_total = 0;
    if (any_eq) {
      r = block_excl_scan(c, warp_tot, &total);
      step_total = total;
    }
    const unsigned b = eq_before + r;
    uchar4 o;
    o.x = (q.x > prefix || (e0 && b < k)) ? 1 : 0;
    o.y = (q.y > prefix || (e1 && b + e0 < k)) ? 1 : 0;
    o.z = (q.z > prefix || (e2 && b + e0 + e1 < k)) ? 1 : 0;
    o.w = (q.w > prefix || (e3 && b + e0 + e1 + e2 < k)) ? 1 : 0;
    if (in) *reinterpret_cast<uchar4*>(out + i) = o;
    eq_before += step_total;
  }
}

spring_status launch_select_area(int n, const float* sm, const int64_t* alpha, int alpha_stride,
                                 uint8_t* S, int batch, cudaStream_t s, int alpha_group, void* scratch) {
  if (batch < 1) return SPRING_OK;
  if (alpha_group < 1) return invalid("alpha_group must be >= 1");
  if (!scratch) return invalid("select scratch missing");
  const long long nn = (long long)n * n;
  const int chunks = sel_chunks(nn);
  SelScratch sc;
  sc.ghist = static_cast<unsigned*>(scratch);
  sc.state = sc.ghist + (size_t)batch * SEL_BINS;
  sc.eqcnt = sc.state + (size_t)batch * 4;
  SPRING_CUDA(cudaMemsetAsync(sc.ghist, 0, sizeof(unsigned) * (size_t)batch * SEL_BINS, s));
  const int blocks = batch * chunks;
  launch_begin(SPRING_KC_OTHER, s);
  k_sel_hist<0><<<blocks, SEL_T, 0, s>>>(sm, alpha, alpha_stride, alpha_group, sc, nn, chunks);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, (double)nn * batch * 4.0);
  launch_begin(SPRING_KC_OTHER, s);
  k_sel_digit<0><<<batch, SEL_THREADS, 0, s>>>(alpha, alpha_stride, alpha_group, sc, nn);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, 0.0);
  launch_begin(SPRING_KC_OTHER, s);
  k_sel_hist<1><<<blocks, SEL_T, 0, s>>>(sm, alpha, alpha_stride, alpha_group, sc, nn, chunks);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, (double)nn * batch * 4.0);
  launch_begin(SPRING_KC_OTHER, s);
  k_sel_digit<1><<<batch, SEL_THREADS, 0, s>>>(alpha, alpha_stride, alpha_group, sc, nn);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, 0.0);
  launch_begin(SPRING_KC_OTHER, s);
  k_sel_hist<2><<<blocks, SEL_T, 0, s>>>(sm, alpha, alpha_stride, alpha_group, sc, nn, chunks);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, (double)nn * batch * 4.0);
  launch_begin(SPRING_KC_OTHER, s);
  k_sel_digit<2><<<batch, SEL_THREADS, 0, s>>>(alpha, alpha_stride, alpha_group, sc, nn);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, 0.0);
  launch_begin(SPRING_KC_OTHER, s);
  k_sel_eqcount<<<blocks, SEL_T, 0, s>>>(sm, sc, nn, chunks);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, (double)nn * batch * 4.0);
  launch_begin(SPRING_KC_OTHER, s);
  k_sel_write<<<blocks, SEL_T, 0, s>>>(sm, sc, S, nn, chunks);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, (double)nn * batch * 5.0);
  return SPRING_OK;
}

}  // namespace spring
