// k_bounds.cu -- the modulus array M of a pattern, with optional upper bounds for the
// missing intensities (App. "Constraining intensities at large scattering angles":
// Eqs. avgint, stdint, upperbound; enforced by Eq. pm_bounds in the column pass).
//
// Encoding of M (float, DFT order), read by every modulus projection of the library:
//   M >= 0       measured pixel (Xi = 1), modulus M
//   M <= -2      missing pixel with an upper bound on its modulus: U = -2 - M
//   -2 < M < 0   missing pixel without a bound (the library writes -1)
// For 2 <= -M < 2^25 the FP32 subtraction -2 - M is exact, so U is read back exactly as
// encoded (the encoding itself rounds -2 - U to FP32 once).
//
// Rings: pixels are grouped by their distance q from the detector centre (pixel (N/2, N/2)
// of the centred array) rounded to the nearest integer, i.e. ring r holds the offsets with
// r(r - 1) < dy^2 + dx^2 <= r(r + 1) (r = 0: the centre only); the rule is exact in
// integers.  One thread per ring visits its pixels row by row and, inside a row, in
// increasing column, so each ring's FP64 sums are taken in plain row-major order.
#include <cmath>

#include "internal.h"

namespace spring {

__device__ __forceinline__ long long isqrt_ll(long long v) {  // floor(sqrt(v)), v >= 0
  long long s = (long long)sqrt((double)v);
  while (s * s > v) --s;
  while ((s + 1) * (s + 1) <= v) ++s;
  return s;
}

// visit the pixels of ring r in row-major order: f(k) with k the centred linear index
template <class F>
__device__ void for_ring(int n, int r, F f) {
  const int h = n / 2;
  const long long lo = (long long)r * (r - 1), hi = (long long)r * (r + 1);  // lo < d2 <= hi
  const int dy0 = max(-h, -(r + 1)), dy1 = min(h - 1, r + 1);
  for (int dy = dy0; dy <= dy1; ++dy) {
    const long long d2y = (long long)dy * dy;
    const long long rem_hi = hi - d2y;
    if (rem_hi < 0) continue;
    const long long b = isqrt_ll(rem_hi);
    const long long a = (r == 0 || lo - d2y < 0) ? 0 : isqrt_ll(lo - d2y) + 1;
    if (a > b) continue;
    const long long row = (long long)(dy + h) * n + h;
    for (long long dx = max((long long)-h, -b); dx <= -a; ++dx) f(row + dx);
    for (long long dx = max(a, 1LL); dx <= min(b, (long long)h - 1); ++dx) f(row + dx);
  }
}

// per ring: the amplitude bound sqrt(mu + eta sigma), or -1 where the ring takes none
__global__ void k_ring_bounds(const float* __restrict__ I, const uint8_t* __restrict__ mask,
                              const uint8_t* __restrict__ sat, int n, int nrings, double eta,
                              double max_missing, double max_saturated, double* __restrict__ Ur) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrings) return;
  long long cnt = 0, meas = 0, nsat = 0;
  double s1 = 0.0;
  for_ring(n, r, [&](long long k) {
    ++cnt;
    if (sat && sat[k]) ++nsat;
    if (mask[k]) {
      ++meas;
      s1 += (double)I[k];
    }
  });
  double u = -1.0;
  if (cnt > 0 && meas > 0 && (double)(cnt - meas) <= max_missing * (double)cnt &&
      (double)nsat <= max_saturated * (double)cnt) {
    const double mu = s1 / (double)meas;
    double s2 = 0.0;  // Eq. stdint as the mean squared deviation (no cancellation)
    for_ring(n, r, [&](long long k) {
      if (mask[k]) {
        const double d = (double)I[k] - mu;
        s2 += d * d;
      }
    });
    u = sqrt(fmax(0.0, mu + eta * sqrt(s2 / (double)meas)));
  }
  Ur[r] = u;
}

__device__ __forceinline__ int ring_of(int dy, int dx) {
  const long long d2 = (long long)dy * dy + (long long)dx * dx;
  const long long s = isqrt_ll(d2);
  return (int)(d2 > s * (s + 1) ? s + 1 : s);
}

// M in DFT order from detector-centred I, mask (and saturation map and ring bounds)
__global__ void k_make_modulus_b(const float* __restrict__ I, const uint8_t* __restrict__ mask,
                                 const uint8_t* __restrict__ sat, const double* __restrict__ Ur, int n,
                                 float* __restrict__ M) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)n * n) return;
  const int r = (int)(i / n), c = (int)(i % n), h = n / 2;
  // DFT-order (r, c) holds the detector-centred value at ((r + N/2) mod N, (c + N/2) mod N)
  const int yc = (r + h) % n, xc = (c + h) % n;
  const long long src = (long long)yc * n + xc;
  float m = -1.f;
  if (mask[src]) {
    m = sqrtf(fmaxf(I[src], 0.f));
  } else if (Ur && !(sat && sat[src])) {
    const double u = Ur[ring_of(yc - h, xc - h)];
    if (u >= 0.0) m = (float)(-2.0 - u);
  }
  M[i] = m;
}

int ring_count(int n) {
  const int h = n / 2;
  return (int)std::llround(std::sqrt(2.0 * h * h)) + 1;
}

spring_status launch_modulus_encode(int n, const float* I_c, const uint8_t* mask_c, const uint8_t* sat_c,
                                    const spring_bounds* b, double* ring_scratch, float* M, cudaStream_t s) {
  const long long nn = (long long)n * n;
  const bool bounded = b && b->eta > 0.f;
  if (bounded) {
    const int nr = ring_count(n);
    launch_begin(SPRING_KC_OTHER, s);
    k_ring_bounds<<<div_up(nr, 64), 64, 0, s>>>(I_c, mask_c, sat_c, n, nr, (double)b->eta,
                                                (double)b->max_missing, (double)b->max_saturated,
                                                ring_scratch);
    SPRING_CHECK_LAUNCH();
    launch_end(SPRING_KC_OTHER, s, nn * 2.0 * 6.0);
  }
  launch_begin(SPRING_KC_OTHER, s);
  k_make_modulus_b<<<div_up(nn, 256), 256, 0, s>>>(I_c, mask_c, sat_c, bounded ? ring_scratch : nullptr, n, M);
  SPRING_CHECK_LAUNCH();
  launch_end(SPRING_KC_OTHER, s, nn * 10.0);
  return SPRING_OK;
}

}  // namespace spring
