// k_ga.cu -- once-per-generation kernels of MPR: the genetic operators (App. "Crossover",
// App. "The Selection step"), alignment (App. "Aligning the reconstructions"), averaging
// (Eq. avgrec), area bookkeeping (Alg. improve), initialisation (App. "Initialization of
// the starting densities") and the monitors (Sec. "Monitoring the reconstruction process").
//
// Every integer decision (parents, crossover tiles, selection, argmax/argmin ties, areas)
// is computed with integer arithmetic or exact comparisons, so it is reproducible given
// the same inputs; every floating-point reduction runs in a fixed order.
#include <cmath>

#include "internal.h"

namespace spring {

// ------------------------------------------------------------------ RandomChoice
__global__ void k_random_choice(uint64_t seed, int g, int P, int32_t* __restrict__ abc) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  uint32_t u[4];
  draw(seed, (uint32_t)g, (uint32_t)p, 1u, 0u, 0u, u);
  int taken[4] = {p, 0, 0, 0};
  int nt = 1;
  for (int k = 0; k < 3; ++k) {
    int v = (int)uniform_below(u[k], (uint32_t)(P - 1 - k));
    int ex[4];
    for (int i = 0; i < nt; ++i) ex[i] = taken[i];
    for (int i = 1; i < nt; ++i)  // insertion sort of the excluded indices
      for (int j = i; j > 0 && ex[j - 1] > ex[j]; --j) {
        int t = ex[j];
        ex[j] = ex[j - 1];
        ex[j - 1] = t;
      }
    for (int i = 0; i < nt; ++i)
      if (v >= ex[i]) ++v;
    abc[3 * p + k] = v;
    taken[nt++] = v;
  }
}

spring_status launch_random_choice(uint64_t seed, int g, int P, int32_t* abc, cudaStream_t s) {
  if (P < 4) return invalid("population must be >= 4");
  launch_begin(SPRING_KC_OTHER, s);
  k_random_choice<<<div_up(P, 128), 128, 0, s>>>(seed, g, P, abc);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, 12.0 * P);
  return SPRING_OK;
}

// ------------------------------------------------------------------ CrossoverMap
struct MapCfg {
  uint64_t seed;
  uint64_t thr;  // elected iff draw < floor(C_p 2^32)
  int g, tmin, tmax, n;
};

static MapCfg make_map_cfg(uint64_t seed, int g, int n, int tmin, int tmax, float cp) {
  MapCfg c{};
  c.seed = seed;
  double t = std::floor((double)cp * 4294967296.0);
  if (t > 4294967296.0) t = 4294967296.0;
  if (t < 0.0) t = 0.0;
  c.thr = (uint64_t)t;
  c.g = g;
  c.tmin = tmin;
  c.tmax = tmax <= 0 ? n / 8 : tmax;
  if (c.tmax < c.tmin) c.tmax = c.tmin;
  c.n = n;
  return c;
}

struct MapGeom {
  int tx, ty, ox, oy, k;
};

__device__ __forceinline__ MapGeom map_geometry(const MapCfg& c, int p) {
  uint32_t u[4], v[4];
  draw(c.seed, (uint32_t)c.g, (uint32_t)p, 2u, 0u, 0u, u);
  draw(c.seed, (uint32_t)c.g, (uint32_t)p, 2u, 0u, 1u, v);
  const uint32_t span = (uint32_t)(c.tmax - c.tmin + 1);
  MapGeom m;
  m.tx = c.tmin + (int)uniform_below(u[0], span);
  m.ty = c.tmin + (int)uniform_below(u[1], span);
  m.ox = (int)uniform_below(u[2], (uint32_t)m.tx);
  m.oy = (int)uniform_below(v[0], (uint32_t)m.ty);
  m.k = (int)uniform_below(v[1], 1024u);
  return m;
}

__device__ __forceinline__ long long floor_div(long long a, long long b) {
  long long q = a / b;
  if ((a % b != 0) && (a < 0)) --q;
  return q;
}

// tile election at DFT-order pixel (i, j) for individual p
__device__ __forceinline__ bool map_elected(const MapCfg& c, int p, const MapGeom& m, long long ck,
                                            long long sk, int i, int j) {
  const int n = c.n;
  const long long v = ((i + n / 2) % n) - n / 2;  // centred row frequency
  const long long u = ((j + n / 2) % n) - n / 2;  // centred column frequency
  const long long ONE = 1LL << 30;
  const long long U = ck * u + sk * v + (long long)m.ox * ONE;
  const long long V = -sk * u + ck * v + (long long)m.oy * ONE;
  const long long tix = floor_div(U, (long long)m.tx * ONE);
  const long long tiy = floor_div(V, (long long)m.ty * ONE);
  uint32_t r[4];
  draw(c.seed, (uint32_t)c.g, (uint32_t)p, 3u, (uint32_t)(tix + 32768), (uint32_t)(tiy + 32768), r);
  return (uint64_t)r[0] < c.thr;
}

__global__ void k_crossover_map(MapCfg c, int p, const long long* __restrict__ rc,
                                const long long* __restrict__ rs, uint8_t* __restrict__ map) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = c.n;
  if (idx >= n * n) return;
  const MapGeom m = map_geometry(c, p);
  map[idx] = map_elected(c, p, m, rc[m.k], rs[m.k], idx / n, idx % n) ? 1 : 0;
}

spring_status launch_crossover_map(uint64_t seed, int g, int p, int n, int tmin, int tmax, float cp,
                                   uint8_t* map, cudaStream_t s) {
  DeviceTables tb;
  SPRING_TRY(device_tables(&tb));
  if (tmin < 1) return invalid("tile_min must be >= 1");
  const MapCfg c = make_map_cfg(seed, g, n, tmin, tmax, cp);
  launch_begin(SPRING_KC_OTHER, s);
  k_crossover_map<<<div_up((long long)n * n, 256), 256, 0, s>>>(c, p, tb.rot_cos, tb.rot_sin, map);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, (double)n * n);
  return SPRING_OK;
}

// ------------------------------------------------------------------ Reshift
// Cross-correlation spectra (Eq. crosscorr) of pairs q: A[q] = Xi conj(X_x) X_ref (for
// x onto ref), B[q] = Xi X_x X_ref (its twin conj(x(-r)) onto ref).
__global__ void k_xcorr_spectra(const float2* __restrict__ X, const int32_t* __restrict__ ix,
                                const int32_t* __restrict__ ir, const float* __restrict__ M,
                                float2* __restrict__ A, float2* __restrict__ B, long long nn) {
  const int q = blockIdx.y;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  const float2 a = X[(long long)ix[q] * nn + i];
  const float2 r = X[(long long)ir[q] * nn + i];
  const bool xi = __ldg(&M[i]) >= 0.f;
  A[(long long)q * nn + i] = xi ? cmul(cconj(a), r) : make_float2(0.f, 0.f);
  B[(long long)q * nn + i] = xi ? cmul(a, r) : make_float2(0.f, 0.f);
}

spring_status launch_xcorr_spectra(int n, const float2* X, const int32_t* ix, const int32_t* ir,
                                   int npairs, const float* M, float2* A, float2* B, cudaStream_t s) {
  if (npairs < 1) return SPRING_OK;
  const long long nn = (long long)n * n;
  dim3 grid(div_up(nn, 256), npairs);
  launch_begin(SPRING_KC_OTHER, s);
  k_xcorr_spectra<<<grid, 256, 0, s>>>(X, ix, ir, M, A, B, nn);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, (double)npairs * nn * 32.0);
  return SPRING_OK;
}

// Peak search: per image the largest |c|^2 with the lowest linear index on ties.
struct Peak {
  float v;
  int i;
};
__device__ __forceinline__ Peak better(Peak a, Peak b) {
  return (b.v > a.v || (b.v == a.v && b.i < a.i)) ? b : a;
}

constexpr int PEAK_THREADS = 256;
constexpr int PEAK_BLOCKS = 16;  // partial results per image

__global__ void k_peak_partial(const float2* __restrict__ A, const float2* __restrict__ B,
                               long long nn, Peak* __restrict__ part) {
  const int img = blockIdx.y;  // 2q: A[q], 2q + 1: B[q]
  const float2* c = ((img & 1) ? B : A) + (long long)(img >> 1) * nn;
  Peak b{-1.f, 0x7fffffff};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nn;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 z = c[i];
    b = better(b, Peak{z.x * z.x + z.y * z.y, (int)i});
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Peak t;
    t.v = __shfl_down_sync(0xffffffffu, b.v, o);
    t.i = __shfl_down_sync(0xffffffffu, b.i, o);
    b = better(b, t);
  }
  __shared__ Peak w[PEAK_THREADS / 32];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = b;
  __syncthreads();
  if (threadIdx.x == 0) {
    Peak r = w[0];
    for (int k = 1; k < PEAK_THREADS / 32; ++k) r = better(r, w[k]);
    part[(long long)img * gridDim.x + blockIdx.x] = r;
  }
}

__global__ void k_peak_final(const float2* __restrict__ A, const float2* __restrict__ B, long long nn, int n,
                             const Peak* __restrict__ part, int nparts, int npairs,
                             int32_t* __restrict__ info, float2* __restrict__ phasor) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= npairs) return;
  Peak pk[2];
  for (int t = 0; t < 2; ++t) {
    Peak r = part[(long long)(2 * q + t) * nparts];
    for (int k = 1; k < nparts; ++k) r = better(r, part[(long long)(2 * q + t) * nparts + k]);
    pk[t] = r;
  }
  const int twin = pk[1].v > pk[0].v ? 1 : 0;
  const int idx = pk[twin].i;
  const float2 z = (twin ? B : A)[(long long)q * nn + idx];
  const float a = sqrtf(z.x * z.x + z.y * z.y);
  info[3 * q + 0] = idx / n;
  info[3 * q + 1] = idx % n;
  info[3 * q + 2] = twin;
  phasor[q] = a > 0.f ? make_float2(z.x / a, z.y / a) : make_float2(1.f, 0.f);
}

size_t peaks_scratch_bytes(int, int npairs) { return sizeof(Peak) * (size_t)PEAK_BLOCKS * 2 * npairs; }

spring_status launch_peaks(int n, const float2* A, const float2* B, int npairs, int32_t* info,
                           float2* phasor, void* scratch, cudaStream_t s) {
  if (npairs < 1) return SPRING_OK;
  const long long nn = (long long)n * n;
  Peak* part = reinterpret_cast<Peak*>(scratch);
  launch_begin(SPRING_KC_OTHER, s);
  k_peak_partial<<<dim3(PEAK_BLOCKS, 2 * npairs), PEAK_THREADS, 0, s>>>(A, B, nn, part);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, (double)npairs * nn * 16.0);
  launch_begin(SPRING_KC_OTHER, s);
  k_peak_final<<<div_up(npairs, 128), 128, 0, s>>>(A, B, nn, n, part, PEAK_BLOCKS, npairs, info, phasor);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, (double)npairs * 64.0);
  return SPRING_OK;
}

// source pixel of the aligned image at (r, c): x'(r) = x(r - s) or conj(x(s - r))
__device__ __forceinline__ long long shift_src(int n, int r, int c, int sy, int sx, int twin) {
  int yr, xc;
  if (twin) {
    yr = sy - r;
    xc = sx - c;
  } else {
    yr = r - sy;
    xc = c - sx;
  }
  yr = ((yr % n) + n) % n;
  xc = ((xc % n) + n) % n;
  return (long long)yr * n + xc;
}

__global__ void k_apply_shift(const float2* __restrict__ x, const uint8_t* __restrict__ S,
                              const int32_t* __restrict__ ix, const int32_t* __restrict__ info,
                              const float2* __restrict__ phasor, float2* __restrict__ xo,
                              uint8_t* __restrict__ So, int n) {
  const int q = blockIdx.y;
  const long long nn = (long long)n * n;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  const int sy = info[3 * q], sx = info[3 * q + 1], tw = info[3 * q + 2];
  const long long src = shift_src(n, (int)(i / n), (int)(i % n), sy, sx, tw) + (long long)ix[q] * nn;
  if (xo) {
    float2 v = x[src];
    if (tw) v = cconj(v);
    xo[(long long)q * nn + i] = cmul(phasor[q], v);
  }
  if (So) So[(long long)q * nn + i] = S ? S[src] : 0;
}

spring_status launch_apply_shift(int n, const float2* x, const uint8_t* S, const int32_t* ix,
                                 int npairs, const int32_t* info, const float2* phasor,
                                 float2* x_out, uint8_t* S_out, cudaStream_t s) {
  if (npairs < 1 || (!x_out && !S_out)) return SPRING_OK;
  const long long nn = (long long)n * n;
  launch_begin(SPRING_KC_OTHER, s);
  k_apply_shift<<<dim3(div_up(nn, 256), npairs), 256, 0, s>>>(x, S, ix, info, phasor, x_out, S_out, n);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, (double)npairs * nn * 18.0);
  return SPRING_OK;
}

// ------------------------------------------------------------------ Crossover
// In Fourier space the aligned parent is e^{i phi} e^{-2 pi i (k . s) / N} X(k) (or the
// same with conj X(k) for the twin), the shift theorem applied to x(r - s).
__device__ __forceinline__ float2 aligned_spectrum(const float2* __restrict__ X, long long nn, int n,
                                                   int par, const int32_t* inf, float2 ph,
                                                   const float2* __restrict__ tw, int kr, int kc,
                                                   long long i) {
  float2 v = X[(long long)par * nn + i];
  if (inf[2]) v = cconj(v);
  const int idx = (int)(((long long)kr * inf[0] + (long long)kc * inf[1]) % n);
  return cmul(cmul(ph, __ldg(&tw[idx])), v);
}

__global__ void k_crossover_mix(const float2* __restrict__ X, const int32_t* __restrict__ abc,
                                const int32_t* __restrict__ info, const float2* __restrict__ phasor,
                                MapCfg c, float cw, const long long* __restrict__ rc,
                                const long long* __restrict__ rs, const float2* __restrict__ tw,
                                float ca, const float* __restrict__ mavg, float2* __restrict__ Xnew) {
  const int p = blockIdx.y, n = c.n;
  const long long nn = (long long)n * n;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  const int kr = (int)(i / n), kc = (int)(i % n);
  const MapGeom m = map_geometry(c, p);
  float2 out;
  if (map_elected(c, p, m, rc[m.k], rs[m.k], kr, kc)) {
    float2 A = aligned_spectrum(X, nn, n, abc[3 * p + 0], info + 9 * p + 0, phasor[3 * p + 0], tw, kr, kc, i);
    if (ca > 0.f) {  // Eq. crossavg: moduli towards the average ones, phases kept
      const float a = sqrtf(A.x * A.x + A.y * A.y);
      const float m = ca * mavg[i] + (1.f - ca) * a;
      A = a > 0.f ? make_float2(A.x * (m / a), A.y * (m / a)) : make_float2(m, 0.f);
    }
    const float2 B = aligned_spectrum(X, nn, n, abc[3 * p + 1], info + 9 * p + 3, phasor[3 * p + 1], tw, kr, kc, i);
    const float2 Cc = aligned_spectrum(X, nn, n, abc[3 * p + 2], info + 9 * p + 6, phasor[3 * p + 2], tw, kr, kc, i);
    out = make_float2(A.x + cw * (B.x - Cc.x), A.y + cw * (B.y - Cc.y));
  } else {
    out = X[(long long)p * nn + i];
  }
  Xnew[(long long)p * nn + i] = out;
}

spring_status launch_crossover_mix(int n, const float2* Xpop, const int32_t* abc,
                                   const int32_t* info, const float2* phasor, int P, uint64_t seed,
                                   int g, float cw, float cp, int tmin, int tmax, float ca,
                                   const float* mavg, float2* Xnew, cudaStream_t s) {
  if (ca > 0.f && !mavg) return invalid("crossover averaging needs the average moduli");
  DeviceTables tb;
  SPRING_TRY(device_tables(&tb));
  if (tmin < 1) return invalid("tile_min must be >= 1");
  const MapCfg c = make_map_cfg(seed, g, n, tmin, tmax, cp);
  const long long nn = (long long)n * n;
  launch_begin(SPRING_KC_OTHER, s);
  k_crossover_mix<<<dim3(div_up(nn, 256), P), 256, 0, s>>>(Xpop, abc, info, phasor, c, cw, tb.rot_cos,
                                                           tb.rot_sin, tb.tw + tw_offset(n), ca, mavg,
                                                           Xnew);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, (double)P * nn * 40.0);
  return SPRING_OK;
}

// per pixel: (|avg_spec| + mean_p |Xpop_p|) / 2, the sum over p in increasing order in FP32
__global__ void k_average_moduli(const float2* __restrict__ X, const float2* __restrict__ avg, int P,
                                 long long nn, float* __restrict__ mavg) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nn;
       i += (long long)gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int p = 0; p < P; ++p) {
      const float2 v = X[(long long)p * nn + i];
      acc += sqrtf(v.x * v.x + v.y * v.y);
    }
    const float2 a = avg[i];
    mavg[i] = 0.5f * (sqrtf(a.x * a.x + a.y * a.y) + acc / (float)P);
  }
}

spring_status launch_average_moduli(int n, const float2* Xpop, const float2* avg_spec, int P, float* mavg,
                                    cudaStream_t s) {
  const long long nn = (long long)n * n;
  launch_begin(SPRING_KC_OTHER, s);
  k_average_moduli<<<(int)std::min<long long>(div_up(nn, 256), 8LL * sm_count()), 256, 0, s>>>(
      Xpop, avg_spec, P, nn, mavg);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, (double)nn * (8.0 * P + 12.0));
  return SPRING_OK;
}

__global__ void k_crossover_support(const uint8_t* __restrict__ S, const int32_t* __restrict__ abc,
                                    const int32_t* __restrict__ info, int n, uint8_t* __restrict__ Snew) {
  const int p = blockIdx.y;
  const long long nn = (long long)n * n;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  const int r = (int)(i / n), c = (int)(i % n);
  uint8_t s3[3];
  for (int k = 0; k < 3; ++k) {
    const int32_t* in = info + 9 * p + 3 * k;
    s3[k] = S[(long long)abc[3 * p + k] * nn + shift_src(n, r, c, in[0], in[1], in[2])];
  }
  Snew[(long long)p * nn + i] = (s3[0] | (s3[1] & s3[2] & S[(long long)p * nn + i])) ? 1 : 0;
}

spring_status launch_crossover_support(int n, const uint8_t* Spop, const int32_t* abc,
                                       const int32_t* info, int P, uint8_t* Snew, cudaStream_t s) {
  const long long nn = (long long)n * n;
  launch_begin(SPRING_KC_OTHER, s);
  k_crossover_support<<<dim3(div_up(nn, 256), P), 256, 0, s>>>(Spop, abc, info, n, Snew);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, (double)P * nn * 5.0);
  return SPRING_OK;
}

__global__ void k_pairs_crossover(int P, const int32_t* __restrict__ abc, int32_t* ix, int32_t* ir) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= 3 * P) return;
  ix[q] = abc[q];
  ir[q] = q / 3;
}

spring_status launch_pairs_crossover(int P, const int32_t* abc, int32_t* ix, int32_t* ir,
                                     cudaStream_t s) {
  launch_begin(SPRING_KC_OTHER, s);
  k_pairs_crossover<<<div_up(3 * P, 128), 128, 0, s>>>(P, abc, ix, ir);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, 12.0 * P);
  return SPRING_OK;
}

// ------------------------------------------------------------------ Select
__global__ void k_select_copy(float2* __restrict__ px, uint8_t* __restrict__ pS,
                              const double* __restrict__ pe, const float2* __restrict__ nx,
                              const uint8_t* __restrict__ nS, const double* __restrict__ ne,
                              long long nn) {
  const int p = blockIdx.y;
  if (!(ne[p] < pe[p])) return;  // strict: ties keep the parent
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nn;
       i += (long long)gridDim.x * blockDim.x) {
    px[(long long)p * nn + i] = nx[(long long)p * nn + i];
    pS[(long long)p * nn + i] = nS[(long long)p * nn + i];
  }
}

__global__ void k_select_err(double* __restrict__ pe, const double* __restrict__ ne, int P,
                             uint8_t* __restrict__ replaced) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const bool r = ne[p] < pe[p];
  if (r) pe[p] = ne[p];
  if (replaced) replaced[p] = r ? 1 : 0;
}

spring_status launch_select(int n, float2* pop_x, uint8_t* pop_S, double* pop_err,
                            const float2* new_x, const uint8_t* new_S, const double* new_err,
                            int P, uint8_t* replaced, cudaStream_t s) {
  const long long nn = (long long)n * n;
  launch_begin(SPRING_KC_OTHER, s);
  k_select_copy<<<dim3(64, P), 256, 0, s>>>(pop_x, pop_S, pop_err, new_x, new_S, new_err, nn);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, (double)P * nn * 9.0);
  launch_begin(SPRING_KC_OTHER, s);
  k_select_err<<<div_up(P, 128), 128, 0, s>>>(pop_err, new_err, P, replaced);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, 17.0 * P);
  return SPRING_OK;
}

// ------------------------------------------------------------------ argmin / pairs
__global__ void k_argmin(const double* __restrict__ err, int P, int32_t* __restrict__ best) {
  if (threadIdx.x != 0) return;
  int b = 0;
  if (err)
    for (int p = 1; p < P; ++p)
      if (err[p] < err[b]) b = p;
  *best = b;
}

spring_status launch_argmin(const double* err, int P, int32_t* best, cudaStream_t s) {
  launch_begin(SPRING_KC_OTHER, s);
  k_argmin<<<1, 32, 0, s>>>(err, P, best);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, 8.0 * P);
  return SPRING_OK;
}

__global__ void k_pairs_onto_best(int P, const int32_t* __restrict__ best, int32_t* ix, int32_t* ir) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= P) return;
  ix[q] = q;
  ir[q] = *best;
}

spring_status launch_pairs_onto_best(int P, const int32_t* best, int32_t* ix, int32_t* ir,
                                     cudaStream_t s) {
  launch_begin(SPRING_KC_OTHER, s);
  k_pairs_onto_best<<<div_up(P, 128), 128, 0, s>>>(P, best, ix, ir);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, 8.0 * P);
  return SPRING_OK;
}

// ------------------------------------------------------------------ Average
__global__ void k_average(const float2* __restrict__ x, const uint8_t* __restrict__ S,
                          const int32_t* __restrict__ info, const float2* __restrict__ phasor,
                          const int32_t* __restrict__ bestp, int P, int n, float2* __restrict__ avg,
                          uint8_t* __restrict__ Savg) {
  const long long nn = (long long)n * n;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  const int best = *bestp, r = (int)(i / n), c = (int)(i % n);
  float2 acc = make_float2(0.f, 0.f);
  uint8_t u = 0;
  for (int p = 0; p < P; ++p) {
    float2 v;
    uint8_t sv;
    if (p == best) {
      v = x[(long long)p * nn + i];
      sv = S[(long long)p * nn + i];
    } else {
      const long long src = shift_src(n, r, c, info[3 * p], info[3 * p + 1], info[3 * p + 2]) + (long long)p * nn;
      v = x[src];
      if (info[3 * p + 2]) v = cconj(v);
      v = cmul(phasor[p], v);
      sv = S[src];
    }
    acc = cadd(acc, v);
    u |= sv;
  }
  avg[i] = cscale(acc, 1.0f / (float)P);
  Savg[i] = u ? 1 : 0;
}

spring_status launch_average(int n, const float2* x, const uint8_t* S, const int32_t* info,
                             const float2* phasor, const int32_t* best, int P, float2* avg,
                             uint8_t* S_avg, cudaStream_t s) {
  const long long nn = (long long)n * n;
  launch_begin(SPRING_KC_OTHER, s);
  k_average<<<div_up(nn, 256), 256, 0, s>>>(x, S, info, phasor, best, P, n, avg, S_avg);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, (double)P * nn * 9.0 + nn * 9.0);
  return SPRING_OK;
}

// ------------------------------------------------------------------ areas (Alg. improve)
__global__ void k_area_count(const uint8_t* __restrict__ S, const int32_t* __restrict__ bestp,
                             int P, long long nn, unsigned long long* __restrict__ cnt) {
  unsigned long long a_best = 0, a_all = 0;
  const int best = bestp ? *bestp : 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nn;
       i += (long long)gridDim.x * blockDim.x) {
    uint8_t u = 0;
    for (int p = 0; p < P; ++p) u |= S[(long long)p * nn + i];
    a_all += u ? 1 : 0;
    a_best += S[(long long)best * nn + i] ? 1 : 0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a_best += __shfl_down_sync(0xffffffffu, a_best, o);
    a_all += __shfl_down_sync(0xffffffffu, a_all, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&cnt[0], a_best);
    atomicAdd(&cnt[1], a_all);
  }
}

__global__ void k_area_finalize(int g, int G, int64_t* out) {
  // alpha_eval = (g/G) alpha_best + (1 - g/G) alpha_all, rounded half up, exactly
  const long long ab = out[0], aa = out[1];
  out[2] = (2LL * ((long long)g * ab + (long long)(G - g) * aa) + G) / (2LL * G);
}

spring_status launch_area_stats(int n, const uint8_t* S, const int32_t* best, int P, int g, int G,
                                int64_t* out3, cudaStream_t s) {
  if (G < 1 || g < 0 || g > G) return invalid("need 0 <= g <= G, G >= 1");
  const long long nn = (long long)n * n;
  SPRING_CUDA(cudaMemsetAsync(out3, 0, 2 * sizeof(int64_t), s));
  launch_begin(SPRING_KC_OTHER, s);
  k_area_count<<<div_up(nn, 256 * 8), 256, 0, s>>>(S, best, P, nn, reinterpret_cast<unsigned long long*>(out3));
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, (double)(P + 1) * nn);
  launch_begin(SPRING_KC_OTHER, s);
  k_area_finalize<<<1, 1, 0, s>>>(g, G, out3);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, 24.0);
  return SPRING_OK;
}

// ------------------------------------------------------------------ Initialize
__global__ void k_bbox_init(int* bbox, int n) {
  bbox[0] = n;
  bbox[1] = -1;
  bbox[2] = n;
  bbox[3] = -1;
}

__global__ void k_bbox(const uint8_t* __restrict__ S0, int n, int* bbox) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)n * n || !S0[i]) return;
  const int r = (int)(i / n), c = (int)(i % n);
  atomicMin(&bbox[0], r);
  atomicMax(&bbox[1], r);
  atomicMin(&bbox[2], c);
  atomicMax(&bbox[3], c);
}

struct Sphere {
  double R, cy, cx, ec, es;
};

__device__ __forceinline__ double unit24(uint32_t u) { return (double)(u >> 8) * (1.0 / 16777216.0); }

__global__ void k_init_params(uint64_t seed, int P, int ns, double phi_max, const int* __restrict__ bbox,
                              Sphere* __restrict__ sp) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= P * ns) return;
  const int p = q / ns, k = q % ns;
  Sphere o{0.0, 0.0, 0.0, 1.0, 0.0};
  if (bbox[1] >= 0) {
    const double h = bbox[1] - bbox[0] + 1, w = bbox[3] - bbox[2] + 1;
    const double side = h > w ? h : w;
    const double y0 = bbox[0] + (h - side) / 2.0, x0 = bbox[2] + (w - side) / 2.0;
    uint32_t u[4];
    draw(seed, 0u, (uint32_t)p, 4u, (uint32_t)k, 0u, u);
    const double D = side * (0.2 + 0.7 * unit24(u[0]));
    o.R = D / 2.0;
    o.cy = y0 + o.R + unit24(u[1]) * (side - D);
    o.cx = x0 + o.R + unit24(u[2]) * (side - D);
    const double phi = phi_max * (2.0 * unit24(u[3]) - 1.0);
    o.ec = cos(phi);
    o.es = sin(phi);
  }
  sp[q] = o;
}

__global__ void k_init_fill(const Sphere* __restrict__ sp, int ns, const uint8_t* __restrict__ S0,
                            int n, double gamma, float2* __restrict__ x) {
  const int p = blockIdx.y;
  const long long nn = (long long)n * n;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  const int r = (int)(i / n), c = (int)(i % n);
  double re = 0.0, im = 0.0;
  for (int k = 0; k < ns; ++k) {
    const Sphere o = sp[p * ns + k];
    const double d2 = (r - o.cy) * (r - o.cy) + (c - o.cx) * (c - o.cx);
    if (d2 < o.R * o.R) {
      const double t = 2.0 * sqrt(o.R * o.R - d2);
      re += o.ec * t;
      im += o.es * t;
    }
  }
  const double a = sqrt(re * re + im * im);
  if (a > 0.0 && gamma != 1.0) {
    const double f = pow(a, gamma) / a;
    re *= f;
    im *= f;
  }
  if (!S0[i]) re = im = 0.0;
  x[(long long)p * nn + i] = make_float2((float)re, (float)im);
}

spring_status launch_init_spheres(int n, uint64_t seed, const uint8_t* S0, int P, int n_spheres,
                                  float gamma, float phi_max, float2* x, void* scratch,
                                  cudaStream_t s) {
  if (n_spheres < 1) return invalid("init_n_spheres must be >= 1");
  int* bbox = reinterpret_cast<int*>(scratch);
  Sphere* sp = reinterpret_cast<Sphere*>(reinterpret_cast<char*>(scratch) + 64);
  const long long nn = (long long)n * n;
  launch_begin(SPRING_KC_OTHER, s);
  k_bbox_init<<<1, 1, 0, s>>>(bbox, n);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, 16.0);
  launch_begin(SPRING_KC_OTHER, s);
  k_bbox<<<div_up(nn, 256), 256, 0, s>>>(S0, n, bbox);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, (double)nn);
  launch_begin(SPRING_KC_OTHER, s);
  k_init_params<<<div_up(P * n_spheres, 128), 128, 0, s>>>(seed, P, n_spheres, (double)phi_max, bbox, sp);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, 40.0 * P * n_spheres);
  launch_begin(SPRING_KC_OTHER, s);
  k_init_fill<<<dim3(div_up(nn, 256), P), 256, 0, s>>>(sp, n_spheres, S0, n, (double)gamma, x);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, (double)P * nn * 9.0);
  return SPRING_OK;
}

size_t init_scratch_bytes(int P, int n_spheres) { return 64 + sizeof(Sphere) * (size_t)P * n_spheres; }

// nu (Eq. norm): per individual, sum_Xi M^2 / sum_Xi |X|^2, in a fixed-order FP64 reduction
constexpr int NORM_BLOCKS = 32;

__global__ void k_masked_power(const float2* __restrict__ X, const float* __restrict__ M, long long nn,
                               double* __restrict__ part) {
  const int p = blockIdx.y;
  double num = 0.0, den = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nn;
       i += (long long)gridDim.x * blockDim.x) {
    const float Mv = M[i];
    if (Mv >= 0.f) {
      const float2 v = X[(long long)p * nn + i];
      num += (double)Mv * (double)Mv;
      den += (double)v.x * v.x + (double)v.y * v.y;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_down_sync(0xffffffffu, num, o);
    den += __shfl_down_sync(0xffffffffu, den, o);
  }
  __shared__ double red[2][8];
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = num;
    red[1][threadIdx.x >> 5] = den;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    part[((long long)p * gridDim.x + blockIdx.x) * 2 + 0] = a;
    part[((long long)p * gridDim.x + blockIdx.x) * 2 + 1] = b;
  }
}

__global__ void k_scale_by_nu(float2* __restrict__ x, const double* __restrict__ part, int nparts,
                              long long nn) {
  const int p = blockIdx.y;
  double a = 0.0, b = 0.0;
  for (int k = 0; k < nparts; ++k) {
    a += part[((long long)p * nparts + k) * 2 + 0];
    b += part[((long long)p * nparts + k) * 2 + 1];
  }
  const float sc = b > 0.0 ? (float)sqrt(a / b) : 1.0f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nn;
       i += (long long)gridDim.x * blockDim.x)
    x[(long long)p * nn + i] = cscale(x[(long long)p * nn + i], sc);
}

size_t normalise_scratch_bytes(int P) { return sizeof(double) * 2 * NORM_BLOCKS * (size_t)P; }

spring_status launch_normalise(int n, const float2* X, const float* M, int P, float2* x,
                               double* partials, cudaStream_t s) {
  const long long nn = (long long)n * n;
  launch_begin(SPRING_KC_OTHER, s);
  k_masked_power<<<dim3(NORM_BLOCKS, P), 256, 0, s>>>(X, M, nn, partials);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, (double)P * nn * 12.0);
  launch_begin(SPRING_KC_OTHER, s);
  k_scale_by_nu<<<dim3(64, P), 256, 0, s>>>(x, partials, NORM_BLOCKS, nn);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, (double)P * nn * 16.0);
  return SPRING_OK;
}

// ------------------------------------------------------------------ monitors
constexpr int DENS_BLOCKS = 64;

__global__ void k_density_partial(const float2* __restrict__ x, long long nn, double* __restrict__ part) {
  // monitors only: per-thread FP32 sums (a few hundred terms), FP64 across threads
  const int p = blockIdx.y;
  float fr = 0.f, fi = 0.f, fa = 0.f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nn;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 v = x[(long long)p * nn + i];
    fr += v.x;
    fi += v.y;
    fa += sqrtf(v.x * v.x + v.y * v.y);
  }
  double sr = fr, si = fi, sa = fa;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_down_sync(0xffffffffu, sr, o);
    si += __shfl_down_sync(0xffffffffu, si, o);
    sa += __shfl_down_sync(0xffffffffu, sa, o);
  }
  __shared__ double red[3][8];
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = sr;
    red[1][threadIdx.x >> 5] = si;
    red[2][threadIdx.x >> 5] = sa;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0, c = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += red[0][w];
      b += red[1][w];
      c += red[2][w];
    }
    double* o = part + ((long long)p * gridDim.x + blockIdx.x) * 3;
    o[0] = a;
    o[1] = b;
    o[2] = c;
  }
}

__global__ void k_density_final(const double* __restrict__ part, int nparts, int P, double* __restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  double a = 0, b = 0, c = 0;
  for (int k = 0; k < nparts; ++k) {
    const double* o = part + ((long long)p * nparts + k) * 3;
    a += o[0];
    b += o[1];
    c += o[2];
  }
  out[2 * p] = sqrt(a * a + b * b);
  out[2 * p + 1] = c;
}

spring_status launch_density_sums(int n, const float2* x, int P, double* partials, double* out,
                                  cudaStream_t s) {
  const long long nn = (long long)n * n;
  launch_begin(SPRING_KC_OTHER, s);
  k_density_partial<<<dim3(DENS_BLOCKS, P), 256, 0, s>>>(x, nn, partials);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, (double)P * nn * 8.0);
  launch_begin(SPRING_KC_OTHER, s);
  k_density_final<<<div_up(P, 128), 128, 0, s>>>(partials, DENS_BLOCKS, P, out);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, 16.0 * P);
  return SPRING_OK;
}

size_t density_scratch_bytes(int P) { return sizeof(double) * 3 * DENS_BLOCKS * (size_t)P; }

__global__ void k_gen_stats(const double* __restrict__ err, const uint8_t* __restrict__ S,
                            const uint8_t* __restrict__ replaced, const double* __restrict__ dens,
                            int P, long long nn, double* __restrict__ row) {
  __shared__ int best_s;
  __shared__ unsigned long long area;
  if (threadIdx.x == 0) {
    int b = 0;
    for (int p = 1; p < P; ++p)
      if (err[p] < err[b]) b = p;
    best_s = b;
    area = 0;
  }
  __syncthreads();
  unsigned long long a = 0;
  for (long long i = threadIdx.x; i < nn; i += blockDim.x) a += S[(long long)best_s * nn + i] ? 1 : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(&area, a);
  __syncthreads();
  if (threadIdx.x == 0) {
    double mn = 0.0, mx = err[0], gam = 0.0, sm = 0.0;
    int rep = 0;
    for (int p = 0; p < P; ++p) {
      mn += err[p];
      mx = err[p] > mx ? err[p] : mx;
      rep += replaced ? replaced[p] : 0;
      const double s_abs = dens[2 * p], a_sum = dens[2 * p + 1];
      gam += a_sum > 0.0 ? 1.0 - s_abs / a_sum : 0.0;
      sm += s_abs;
    }
    row[0] = err[best_s];
    row[1] = mn / P;
    row[2] = mx;
    row[3] = __longlong_as_double(0x7ff8000000000000LL);  // NaN: E(avg) only at the end
    row[4] = (double)nn / (double)(area > 0 ? area : 1);
    row[5] = (double)rep / P;
    row[6] = gam / P;
    row[7] = sm / P;
    // spread of the density sums over the population: population standard deviation
    // relative to their mean (Sec. "Crossover averaging" tracks it in % of the mean)
    const double mean_s = sm / P;
    double var = 0.0;
    for (int p = 0; p < P; ++p) {
      const double d = dens[2 * p] - mean_s;
      var += d * d;
    }
    row[8] = mean_s > 0.0 ? sqrt(var / P) / mean_s : 0.0;
  }
}

spring_status launch_gen_stats(int n, const double* err, const uint8_t* S, const uint8_t* replaced,
                               const double* dens, int P, double* row, cudaStream_t s) {
  launch_begin(SPRING_KC_OTHER, s);
  k_gen_stats<<<1, 1024, 0, s>>>(err, S, replaced, dens, P, (long long)n * n, row);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, (double)n * n);
  return SPRING_OK;
}

// ------------------------------------------------------------------ problem set-up
__global__ void k_make_modulus(const float* __restrict__ I, const uint8_t* __restrict__ mask, int n,
                               float* __restrict__ M) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)n * n) return;
  const int r = (int)(i / n), c = (int)(i % n), h = n / 2;
  // DFT-order (r, c) holds the detector-centred value at ((r + N/2) mod N, (c + N/2) mod N)
  const long long src = (long long)((r + h) % n) * n + (c + h) % n;
  M[i] = mask[src] ? sqrtf(fmaxf(I[src], 0.f)) : -1.f;
}

spring_status launch_make_modulus(int n, const float* I_centred, const uint8_t* mask_centred,
                                  float* M, cudaStream_t s) {
  const long long nn = (long long)n * n;
  launch_begin(SPRING_KC_OTHER, s);
  k_make_modulus<<<div_up(nn, 256), 256, 0, s>>>(I_centred, mask_centred, n, M);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, nn * 9.0);
  return SPRING_OK;
}

__global__ void k_broadcast(const uint8_t* __restrict__ S0, long long nn, uint8_t* __restrict__ S) {
  const int p = blockIdx.y;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nn;
       i += (long long)gridDim.x * blockDim.x)
    S[(long long)p * nn + i] = S0[i];
}

spring_status launch_broadcast_support(int n, const uint8_t* S0, int P, uint8_t* S, cudaStream_t s) {
  const long long nn = (long long)n * n;
  launch_begin(SPRING_KC_OTHER, s);
  k_broadcast<<<dim3(32, P), 256, 0, s>>>(S0, nn, S);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, (double)P * nn + nn);
  return SPRING_OK;
}

}  // namespace spring
