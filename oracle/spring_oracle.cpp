// spring_oracle.cpp -- plain FP64 reference ("oracle") of Memetic Phase Retrieval (MPR).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls this file:
// only the test-suite, the smoke check and the CPU-baseline leg of the benchmark do.
// It shares no code, header, table or helper with the CUDA library; it is deliberately
// slow and written to be checked against the paper by eye.
//
// Paper: Colombo et al., "SPRING: an effective and reliable framework for image
// reconstruction in single-particle Coherent Diffraction Imaging" (arXiv 2409.07413).
// Citations below name the paper's sections, equations and algorithms.
//
// Conventions (where the paper is silent, the reading taken):
//  * Arrays are row-major N x N.  Fourier-space arrays (M, mask, spectra) are in DFT
//    order (zero frequency at index 0); the top-level run takes detector-centred input
//    and applies ifftshift once.  Real-space arrays are used as given.
//  * The 2D transform is unitary (1/N per 2D transform in each direction), so that
//    Parseval (App. "Initialization of the starting densities") holds literally.
//  * Complex arrays cross the C interface as interleaved (re, im) doubles.
//
// Parity of every function below is pinned by tests under tests/ (test_oracle_*.py)
// against brute force, numpy/scipy library routines, closed forms and invariants.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <thread>
#include <vector>

typedef std::complex<double> cd;
static const double PI = 3.14159265358979323846;

// ------------------------------------------------------------------------------------
// Threads: individuals of a population are independent (Sec. "Computational cost and
// performance": the reconstructions are run in parallel), so the oracle runs them on
// std::thread workers.  The thread count is settable for the CPU-baseline timing.
// ------------------------------------------------------------------------------------
static int g_threads = 0;

extern "C" void orc_set_threads(int n) { g_threads = n; }
extern "C" int orc_get_threads(void) {
  if (g_threads > 0) return g_threads;
  unsigned h = std::thread::hardware_concurrency();
  return h ? (int)h : 1;
}

template <class F>
static void parallel_for(int n, F f) {
  int nt = std::min(orc_get_threads(), n);
  if (nt <= 1) {
    for (int i = 0; i < n; i++) f(i);
    return;
  }
  std::atomic<int> next(0);
  std::vector<std::thread> th;
  for (int t = 0; t < nt; t++)
    th.emplace_back([&]() {
      int i;
      while ((i = next.fetch_add(1)) < n) f(i);
    });
  for (auto& t : th) t.join();
}

// ------------------------------------------------------------------------------------
// 1D FFT (Cooley-Tukey).  Lengths 2^a or 3*2^a.  Powers of two: iterative radix-2 with
// bit reversal; 3*2^a: one radix-3 split on top of three radix-2 transforms.
// sign = -1 forward, +1 inverse; unnormalised.
// ------------------------------------------------------------------------------------
struct Plan1D {
  int n = 0, m = 0;         // n = length, m = power-of-two part
  std::vector<int> rev;      // bit reversal of m
  std::vector<cd> tw_m;      // exp(-2 pi i k / m), k < m/2
  std::vector<cd> tw_n;      // exp(-2 pi i k / n), k < n   (radix-3 stage)
};

static bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

static std::shared_ptr<Plan1D> get_plan(int n) {
  thread_local std::map<int, std::shared_ptr<Plan1D>> cache;
  auto it = cache.find(n);
  if (it != cache.end()) return it->second;
  auto p = std::make_shared<Plan1D>();
  p->n = n;
  p->m = is_pow2(n) ? n : n / 3;
  int m = p->m, bits = 0;
  while ((1 << bits) < m) bits++;
  p->rev.resize(m);
  for (int i = 0; i < m; i++) {
    int r = 0;
    for (int b = 0; b < bits; b++)
      if (i & (1 << b)) r |= 1 << (bits - 1 - b);
    p->rev[i] = r;
  }
  p->tw_m.resize(std::max(1, m / 2));
  for (int k = 0; k < m / 2; k++) p->tw_m[k] = std::polar(1.0, -2.0 * PI * k / m);
  if (n != m) {
    p->tw_n.resize(n);
    for (int k = 0; k < n; k++) p->tw_n[k] = std::polar(1.0, -2.0 * PI * k / n);
  }
  cache[n] = p;
  return p;
}

// radix-2 in-place transform of length m (power of two); sign selects direction
static void fft_pow2(cd* a, const Plan1D& p, int sign) {
  int m = p.m;
  for (int i = 0; i < m; i++)
    if (p.rev[i] > i) std::swap(a[i], a[p.rev[i]]);
  for (int len = 2; len <= m; len <<= 1) {
    int half = len / 2, step = m / len;
    for (int i = 0; i < m; i += len)
      for (int j = 0; j < half; j++) {
        cd w = p.tw_m[j * step];
        if (sign > 0) w = std::conj(w);
        cd u = a[i + j], v = a[i + j + half] * w;
        a[i + j] = u + v;
        a[i + j + half] = u - v;
      }
  }
}

// length-n transform of a[0..n) in place (n = 2^a or 3*2^a)
static void fft1d(cd* a, int n, int sign) {
  const Plan1D& p = *get_plan(n);
  if (n == p.m) {
    fft_pow2(a, p, sign);
    return;
  }
  // n = 3m: X[k] = sum_q W_n^{qk} Y_q[k mod m],  Y_q = DFT_m(a[3j+q])
  int m = p.m;
  std::vector<cd> y(n);
  for (int q = 0; q < 3; q++) {
    for (int j = 0; j < m; j++) y[q * m + j] = a[3 * j + q];
    fft_pow2(&y[q * m], p, sign);
  }
  for (int k = 0; k < n; k++) {
    cd acc = 0;
    for (int q = 0; q < 3; q++) {
      cd w = p.tw_n[(q * k) % n];
      if (sign > 0) w = std::conj(w);
      acc += w * y[q * m + (k % m)];
    }
    a[k] = acc;
  }
}

static bool valid_side(int n) {
  if (n < 2) return false;
  if (is_pow2(n)) return true;
  return n % 3 == 0 && is_pow2(n / 3);
}

// unitary 2D DFT of one N x N image in place: rows, then columns, then 1/N
static void fft2_inplace(cd* x, int n, int inverse) {
  int sign = inverse ? +1 : -1;
  for (int r = 0; r < n; r++) fft1d(x + (size_t)r * n, n, sign);
  std::vector<cd> col(n);
  for (int c = 0; c < n; c++) {
    for (int r = 0; r < n; r++) col[r] = x[(size_t)r * n + c];
    fft1d(col.data(), n, sign);
    for (int r = 0; r < n; r++) x[(size_t)r * n + c] = col[r];
  }
  double s = 1.0 / n;
  for (size_t i = 0; i < (size_t)n * n; i++) x[i] *= s;
}

static inline cd* as_cd(double* p) { return reinterpret_cast<cd*>(p); }
static inline const cd* as_cd(const double* p) { return reinterpret_cast<const cd*>(p); }

// Batched unitary 2D DFT (a1, a3).  data: batch x N x N interleaved complex.
extern "C" int orc_fft2(double* data, int batch, int n, int inverse) {
  if (!valid_side(n) || batch < 0) return 1;
  parallel_for(batch, [&](int b) { fft2_inplace(as_cd(data) + (size_t)b * n * n, n, inverse); });
  return 0;
}

// Brute-force O(N^4) unitary 2D DFT, the textbook definition written out (for pins).
extern "C" void orc_dft2_naive(const double* in, double* out, int n, int inverse) {
  const cd* x = as_cd(in);
  cd* X = as_cd(out);
  double sign = inverse ? +1.0 : -1.0;
  for (int q = 0; q < n; q++)
    for (int k = 0; k < n; k++) {
      cd acc = 0;
      for (int r = 0; r < n; r++)
        for (int c = 0; c < n; c++) {
          long ph = ((long)q * r + (long)k * c) % n;
          acc += x[(size_t)r * n + c] * std::polar(1.0, sign * 2.0 * PI * ph / n);
        }
      X[(size_t)q * n + k] = acc / (double)n;
    }
}

// ------------------------------------------------------------------------------------
// Projectors (App. "The phase problem as an optimization problem", Eqs. ps, pm; and
// App. "Constraining intensities at large scattering angles", Eq. pm_full).
// ------------------------------------------------------------------------------------

// Eq. pm_full on a spectrum: where the mask is 1, replace the modulus by M (a zero
// modulus takes phase 0); elsewhere leave the value free.  With upper bounds U (may be
// null; U < 0 = no bound at that pixel) this is Eq. pm_bounds: where the mask is 0 and a
// bound exists, a modulus above U is brought down to U with the phase kept.
static void modulus_constraint(cd* X, const double* M, const uint8_t* mask, const double* U, int n) {
  for (size_t i = 0; i < (size_t)n * n; i++) {
    double a = std::abs(X[i]);
    if (mask[i]) {
      X[i] = (a > 0.0) ? X[i] * (M[i] / a) : cd(M[i], 0.0);
    } else if (U && U[i] >= 0.0 && a > U[i]) {
      X[i] = X[i] * (U[i] / a);
    }
  }
}

// P_M x = F^-1[ masked modulus constraint (F x) ]   (Eq. pm with Eq. pm_full / pm_bounds)
static void project_modulus(const cd* x, cd* out, const double* M, const uint8_t* mask,
                            const double* U, int n) {
  size_t nn = (size_t)n * n;
  std::copy(x, x + nn, out);
  fft2_inplace(out, n, 0);
  modulus_constraint(out, M, mask, U, n);
  fft2_inplace(out, n, 1);
}

extern "C" int orc_project_modulus(const double* x, double* out, const double* M,
                                   const uint8_t* mask, int batch, int n) {
  if (!valid_side(n)) return 1;
  size_t nn = (size_t)n * n;
  parallel_for(batch, [&](int b) {
    project_modulus(as_cd(x) + b * nn, as_cd(out) + b * nn, M, mask, nullptr, n);
  });
  return 0;
}

// P_M with the upper bounds U of Eq. pm_bounds (DFT order, U < 0 = no bound).
extern "C" int orc_project_modulus_ub(const double* x, double* out, const double* M,
                                      const uint8_t* mask, const double* U, int batch, int n) {
  if (!valid_side(n)) return 1;
  size_t nn = (size_t)n * n;
  parallel_for(batch, [&](int b) {
    project_modulus(as_cd(x) + b * nn, as_cd(out) + b * nn, M, mask, U, n);
  });
  return 0;
}

// ------------------------------------------------------------------------------------
// Upper bounds for missing intensities (App. "Constraining intensities at large
// scattering angles", Eqs. avgint, stdint, upperbound).  Pixels are grouped by their
// distance q from the detector centre (pixel (N/2, N/2) of the centred array) rounded to
// the nearest integer.  Over the measured pixels of each ring:
//   mu(q) = mean I,  sigma(q)^2 = mean (I - mu)^2  (= mean I^2 - mu^2 of Eq. stdint,
//   taken as the mean squared deviation so that no cancellation occurs),
//   U_I(q) = mu + eta sigma.
// The bound is used at a missing pixel only if it is not saturated, at most max_missing of
// the ring's pixels are missing, and at most max_saturated of them are saturated.  The
// projector compares moduli, so the per-pixel bound is the amplitude sqrt(U_I(q)).
// Input and output are detector-centred; U = -1 where no bound applies.
// ------------------------------------------------------------------------------------
extern "C" void orc_upper_bounds(const double* I, const uint8_t* mask, const uint8_t* sat, int n,
                                 double eta, double max_missing, double max_saturated, double* U) {
  const int h = n / 2;
  int nb = (int)std::lround(std::sqrt(2.0 * h * h)) + 1;
  std::vector<double> s1(nb, 0.0), s2(nb, 0.0), mu(nb, 0.0);
  std::vector<long> cnt(nb, 0), meas(nb, 0), satc(nb, 0);
  auto ring = [&](int i, int j) {
    long dy = i - h, dx = j - h;
    return (int)std::lround(std::sqrt((double)(dy * dy + dx * dx)));
  };
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) {
      size_t k = (size_t)i * n + j;
      int q = ring(i, j);
      cnt[q]++;
      if (sat && sat[k]) satc[q]++;
      if (mask[k]) {
        meas[q]++;
        s1[q] += I[k];
      }
    }
  for (int q = 0; q < nb; q++) mu[q] = meas[q] ? s1[q] / meas[q] : 0.0;
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) {
      size_t k = (size_t)i * n + j;
      if (mask[k]) {
        int q = ring(i, j);
        s2[q] += (I[k] - mu[q]) * (I[k] - mu[q]);
      }
    }
  std::vector<double> Uq(nb, -1.0);
  for (int q = 0; q < nb; q++) {
    if (cnt[q] == 0 || meas[q] == 0) continue;
    double missing = (double)(cnt[q] - meas[q]);
    if (missing > max_missing * (double)cnt[q]) continue;
    if ((double)satc[q] > max_saturated * (double)cnt[q]) continue;
    double sd = std::sqrt(s2[q] / meas[q]);
    Uq[q] = std::sqrt(std::max(0.0, mu[q] + eta * sd));
  }
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) {
      size_t k = (size_t)i * n + j;
      bool free_px = !mask[k] && !(sat && sat[k]);
      U[k] = free_px ? Uq[ring(i, j)] : -1.0;
    }
}

// cos(chi*pi) with the positivity case chi = 1/2 made exact (the half-plane Re >= 0).
static double chi_cos(double chi) { return (chi == 0.5) ? 0.0 : std::cos(chi * PI); }

// The real-space constraint set C (Eq. ps plus App. "Real-space constraints"): inside
// the support and with phase in [-chi*pi, chi*pi].  chi >= 1 removes the phase limit.
static inline bool in_constraint(uint8_t s, cd m, double chi, double cchi) {
  if (!s) return false;
  if (chi >= 1.0) return true;
  return m.real() >= std::abs(m) * cchi;
}

// One real-space update given m = P_M x (Sec. "The phase problem and conventional
// approaches": ER, HIO [Fienup 1982], RAAR [Luke 2005]).  alg: 0 ER, 1 HIO, 2 RAAR.
static inline cd update_pixel(int alg, cd x, cd m, bool in_c, double beta) {
  if (in_c) return m;
  switch (alg) {
    case 0: return cd(0.0, 0.0);                   // ER: x' = P_S P_M x
    case 1: return x - beta * m;                   // HIO outside C
    default: return beta * x + (1.0 - 2.0 * beta) * m;  // RAAR outside C
  }
}

static void iterate_one(cd* x, const uint8_t* S, const double* M, const uint8_t* mask,
                        const double* U, int n, int alg, double beta, double chi, int n_iter) {
  size_t nn = (size_t)n * n;
  std::vector<cd> m(nn);
  double cchi = chi_cos(chi);
  for (int it = 0; it < n_iter; it++) {
    project_modulus(x, m.data(), M, mask, U, n);
    for (size_t i = 0; i < nn; i++)
      x[i] = update_pixel(alg, x[i], m[i], in_constraint(S[i], m[i], chi, cchi), beta);
  }
}

// n_iter iterations of ER/HIO/RAAR on each image of the batch (a1-a4).
extern "C" int orc_iterate(double* x, const uint8_t* S, const double* M, const uint8_t* mask,
                           int batch, int n, int alg, double beta, double chi, int n_iter) {
  if (!valid_side(n) || alg < 0 || alg > 2) return 1;
  size_t nn = (size_t)n * n;
  parallel_for(batch, [&](int b) {
    iterate_one(as_cd(x) + b * nn, S + b * nn, M, mask, nullptr, n, alg, beta, chi, n_iter);
  });
  return 0;
}

// the same with the upper bounds U of Eq. pm_bounds (DFT order, U < 0 = no bound)
extern "C" int orc_iterate_ub(double* x, const uint8_t* S, const double* M, const uint8_t* mask,
                              const double* U, int batch, int n, int alg, double beta, double chi,
                              int n_iter) {
  if (!valid_side(n) || alg < 0 || alg > 2) return 1;
  size_t nn = (size_t)n * n;
  parallel_for(batch, [&](int b) {
    iterate_one(as_cd(x) + b * nn, S + b * nn, M, mask, U, n, alg, beta, chi, n_iter);
  });
  return 0;
}

// P_S (Eq. ps): element-wise product with the support.
extern "C" void orc_project_support(double* x, const uint8_t* S, int n) {
  cd* z = as_cd(x);
  for (size_t i = 0; i < (size_t)n * n; i++)
    if (!S[i]) z[i] = 0.0;
}

// ------------------------------------------------------------------------------------
// Shrink-wrap (Sec. "The phase problem and conventional approaches", Eq. shrinkwrap;
// App. "The modified Shrink-wrap").
// ------------------------------------------------------------------------------------

// Normalised 1D Gaussian taps w[d], d = -r..r, r = ceil(4 sigma); sigma = 0 -> identity.
static std::vector<double> gauss_taps(double sigma, int* radius) {
  if (sigma <= 0.0) {
    *radius = 0;
    return {1.0};
  }
  int r = (int)std::ceil(4.0 * sigma);
  std::vector<double> w(2 * r + 1);
  double s = 0.0;
  for (int d = -r; d <= r; d++) s += (w[d + r] = std::exp(-(double)d * d / (2.0 * sigma * sigma)));
  for (double& v : w) v /= s;
  *radius = r;
  return w;
}

// rho_sigma = periodic convolution of |x| with the separable Gaussian of width sigma.
static void smooth_abs(const cd* x, double* out, int n, double sigma) {
  int r;
  std::vector<double> w = gauss_taps(sigma, &r);
  size_t nn = (size_t)n * n;
  std::vector<double> a(nn), t(nn);
  for (size_t i = 0; i < nn; i++) a[i] = std::abs(x[i]);
  for (int y = 0; y < n; y++)  // along rows
    for (int c = 0; c < n; c++) {
      double acc = 0.0;
      for (int d = -r; d <= r; d++) acc += w[d + r] * a[(size_t)y * n + (((c + d) % n) + n) % n];
      t[(size_t)y * n + c] = acc;
    }
  for (int y = 0; y < n; y++)  // along columns
    for (int c = 0; c < n; c++) {
      double acc = 0.0;
      for (int d = -r; d <= r; d++) acc += w[d + r] * t[(size_t)((((y + d) % n) + n) % n) * n + c];
      out[(size_t)y * n + c] = acc;
    }
}

extern "C" void orc_smooth(const double* x, double* out, int batch, int n, double sigma) {
  size_t nn = (size_t)n * n;
  parallel_for(batch, [&](int b) { smooth_abs(as_cd(x) + b * nn, out + b * nn, n, sigma); });
}

// UpdateSupport: S = [rho_sigma >= tau * max rho_sigma]
static void update_support(const cd* x, uint8_t* S, int n, double sigma, double tau) {
  size_t nn = (size_t)n * n;
  std::vector<double> s(nn);
  smooth_abs(x, s.data(), n, sigma);
  double mx = *std::max_element(s.begin(), s.end());
  double thr = tau * mx;
  for (size_t i = 0; i < nn; i++) S[i] = (s[i] >= thr) ? 1 : 0;
}

extern "C" void orc_update_support(const double* x, uint8_t* S, int batch, int n, double sigma,
                                   double tau) {
  size_t nn = (size_t)n * n;
  parallel_for(batch, [&](int b) { update_support(as_cd(x) + b * nn, S + b * nn, n, sigma, tau); });
}

// UpdateSupportSize: the alpha pixels of largest rho_sigma; equal values are taken in
// increasing linear index, so the area is exactly alpha.
static void update_support_size(const cd* x, uint8_t* S, int n, double sigma, long alpha) {
  size_t nn = (size_t)n * n;
  std::vector<double> s(nn);
  smooth_abs(x, s.data(), n, sigma);
  if (alpha < 0) alpha = 0;
  if (alpha > (long)nn) alpha = (long)nn;
  std::vector<size_t> idx(nn);
  std::iota(idx.begin(), idx.end(), (size_t)0);
  std::stable_sort(idx.begin(), idx.end(), [&](size_t a, size_t b) { return s[a] > s[b]; });
  std::fill(S, S + nn, 0);
  for (long k = 0; k < alpha; k++) S[idx[k]] = 1;
}

extern "C" void orc_update_support_size(const double* x, uint8_t* S, int batch, int n,
                                        double sigma, const long* alpha) {
  size_t nn = (size_t)n * n;
  parallel_for(batch, [&](int b) {
    update_support_size(as_cd(x) + b * nn, S + b * nn, n, sigma, alpha[b]);
  });
}

// ------------------------------------------------------------------------------------
// GetError (Sec. "Monitoring the reconstruction process", Eq. error_calc)
//   E = sqrt( sum Xi (|F[S x]| - M)^2 / sum Xi M^2 )
// ------------------------------------------------------------------------------------
static double fourier_error(const cd* x, const uint8_t* S, const double* M, const uint8_t* mask,
                            int n) {
  size_t nn = (size_t)n * n;
  std::vector<cd> X(x, x + nn);
  for (size_t i = 0; i < nn; i++)
    if (!S[i]) X[i] = 0.0;
  fft2_inplace(X.data(), n, 0);
  double num = 0.0, den = 0.0;
  for (size_t i = 0; i < nn; i++) {
    if (!mask[i]) continue;
    double d = std::abs(X[i]) - M[i];
    num += d * d;
    den += M[i] * M[i];
  }
  return den > 0.0 ? std::sqrt(num / den) : 0.0;
}

extern "C" void orc_fourier_error(const double* x, const uint8_t* S, const double* M,
                                  const uint8_t* mask, int batch, int n, double* err) {
  size_t nn = (size_t)n * n;
  parallel_for(batch, [&](int b) { err[b] = fourier_error(as_cd(x) + b * nn, S + b * nn, M, mask, n); });
}

// ------------------------------------------------------------------------------------
// Counter-based random numbers: Philox-4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11).  Each round multiplies two
// counter words by fixed constants, mixes the high halves with the other words and the
// key; the key advances by the Weyl increments between rounds.
// ------------------------------------------------------------------------------------
static void philox_4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; round++) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

extern "C" void orc_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  philox_4x32_10(ctr, key, out);
}

// Counter layout: (generation, individual, tag << 24 | a, b).
static void draw(uint64_t seed, uint32_t g, uint32_t p, uint32_t tag, uint32_t a, uint32_t b,
                 uint32_t out[4]) {
  uint32_t ctr[4] = {g, p, (tag << 24) | (a & 0xFFFFFFu), b};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  philox_4x32_10(ctr, key, out);
}

// integer uniform on [0, m): floor(u * m / 2^32)
static inline uint32_t uniform_below(uint32_t u, uint32_t m) {
  return (uint32_t)(((uint64_t)u * m) >> 32);
}

// RandomChoice (App. "Crossover", Alg. crossover): three distinct individuals a, b, c,
// all different from p.  Each is drawn among the remaining candidates, then the excluded
// indices are skipped in increasing order.
static void random_choice(uint64_t seed, int g, int p, int P, int abc[3]) {
  uint32_t u[4];
  draw(seed, (uint32_t)g, (uint32_t)p, 1, 0, 0, u);
  std::vector<int> taken = {p};
  for (int k = 0; k < 3; k++) {
    int v = (int)uniform_below(u[k], (uint32_t)(P - 1 - k));
    std::vector<int> ex = taken;
    std::sort(ex.begin(), ex.end());
    for (int e : ex)
      if (v >= e) v++;
    abc[k] = v;
    taken.push_back(v);
  }
}

extern "C" void orc_random_choice(uint64_t seed, int g, int p, int P, int* abc) {
  random_choice(seed, g, p, P, abc);
}

// CrossoverMap (App. "Crossover", Fig. crossmap): the Fourier plane is cut into tiles of
// random size t_x, t_y in [t_min, t_max]; the tiling is shifted by (o_x, o_y) and rotated
// by theta_k = (pi/2) k / 1024; each tile is elected with probability C_p.  Geometry is
// evaluated in integer fixed point (Q30 rotation) so that it is reproducible exactly.
struct MapGeom {
  int tx, ty, ox, oy, k;
};

static MapGeom map_geometry(uint64_t seed, int g, int p, int tmin, int tmax) {
  uint32_t u[4], v[4];
  draw(seed, (uint32_t)g, (uint32_t)p, 2, 0, 0, u);
  draw(seed, (uint32_t)g, (uint32_t)p, 2, 0, 1, v);
  MapGeom m;
  uint32_t span = (uint32_t)(tmax - tmin + 1);
  m.tx = tmin + (int)uniform_below(u[0], span);
  m.ty = tmin + (int)uniform_below(u[1], span);
  m.ox = (int)uniform_below(u[2], (uint32_t)m.tx);
  m.oy = (int)uniform_below(v[0], (uint32_t)m.ty);
  m.k = (int)uniform_below(v[1], 1024u);
  return m;
}

static void rotation_q30(int k, int64_t* c, int64_t* s) {
  double th = (PI / 2.0) * (double)k / 1024.0;
  *c = std::llround(std::cos(th) * 1073741824.0);
  *s = std::llround(std::sin(th) * 1073741824.0);
}

static int64_t floor_div(int64_t a, int64_t b) {  // b > 0
  int64_t q = a / b;
  if ((a % b != 0) && (a < 0)) q--;
  return q;
}

// A tile is elected iff its 32-bit draw is below floor(C_p 2^32) (64-bit, so C_p = 1
// elects every tile and C_p = 0 none).
static uint64_t cp_threshold(double cp) {
  double t = std::floor(cp * 4294967296.0);
  if (t > 4294967296.0) t = 4294967296.0;
  if (t < 0.0) t = 0.0;
  return (uint64_t)t;
}

static int resolve_tmax(int n, int tmin, int tmax) {
  if (tmax <= 0) tmax = n / 8;
  if (tmax < tmin) tmax = tmin;
  return tmax;
}

static void crossover_map(uint64_t seed, int g, int p, int n, int tmin, int tmax, double cp,
                          uint8_t* map) {
  tmax = resolve_tmax(n, tmin, tmax);
  MapGeom G = map_geometry(seed, g, p, tmin, tmax);
  int64_t ck, sk;
  rotation_q30(G.k, &ck, &sk);
  const int64_t ONE = (int64_t)1 << 30;
  uint64_t thr = cp_threshold(cp);
  for (int i = 0; i < n; i++) {
    int64_t v = ((i + n / 2) % n) - n / 2;  // centred row frequency
    for (int j = 0; j < n; j++) {
      int64_t u = ((j + n / 2) % n) - n / 2;  // centred column frequency
      int64_t U = ck * u + sk * v + (int64_t)G.ox * ONE;
      int64_t V = -sk * u + ck * v + (int64_t)G.oy * ONE;
      int64_t tix = floor_div(U, (int64_t)G.tx * ONE);
      int64_t tiy = floor_div(V, (int64_t)G.ty * ONE);
      uint32_t r[4];
      draw(seed, (uint32_t)g, (uint32_t)p, 3, (uint32_t)(tix + 32768), (uint32_t)(tiy + 32768), r);
      map[(size_t)i * n + j] = ((uint64_t)r[0] < thr) ? 1 : 0;
    }
  }
}

extern "C" void orc_crossover_map(uint64_t seed, int g, int p, int n, int tmin, int tmax,
                                  double cp, uint8_t* map) {
  crossover_map(seed, g, p, n, tmin, tmax, cp, map);
}

extern "C" void orc_map_geometry(uint64_t seed, int g, int p, int n, int tmin, int tmax, int* out5) {
  MapGeom G = map_geometry(seed, g, p, tmin, resolve_tmax(n, tmin, tmax));
  out5[0] = G.tx; out5[1] = G.ty; out5[2] = G.ox; out5[3] = G.oy; out5[4] = G.k;
}

// ------------------------------------------------------------------------------------
// Reshift (App. "Aligning the reconstructions", Eq. crosscorr).
//   c      = F^-1[ Xi conj(F x) F ref ]    (x translated / phased onto ref)
//   c_twin = F^-1[ Xi      F x  F ref ]    (the same for the twin conj(x(-r)))
// The larger peak |c| decides twin or not (ties: not twin), its position s the shift
// (ties: lowest linear index) and its phase the global phase:
//   x'(r) = e^{i phi} x(r - s)          or   x'(r) = e^{i phi} conj(x(s - r)).
// ------------------------------------------------------------------------------------
struct ShiftParams {
  int sy, sx, twin;
  double phase;
};

static void cross_correlations(const cd* x, const cd* ref, const uint8_t* mask, int n, cd* c,
                               cd* ct) {
  size_t nn = (size_t)n * n;
  std::vector<cd> X(x, x + nn), R(ref, ref + nn);
  fft2_inplace(X.data(), n, 0);
  fft2_inplace(R.data(), n, 0);
  for (size_t i = 0; i < nn; i++) {
    double xi = mask[i] ? 1.0 : 0.0;
    c[i] = xi * std::conj(X[i]) * R[i];
    ct[i] = xi * X[i] * R[i];
  }
  fft2_inplace(c, n, 1);
  fft2_inplace(ct, n, 1);
}

static ShiftParams reshift_params(const cd* x, const cd* ref, const uint8_t* mask, int n) {
  size_t nn = (size_t)n * n;
  std::vector<cd> c(nn), ct(nn);
  cross_correlations(x, ref, mask, n, c.data(), ct.data());
  size_t i1 = 0, i2 = 0;
  double m1 = -1.0, m2 = -1.0;
  for (size_t i = 0; i < nn; i++) {
    double a = std::norm(c[i]), b = std::norm(ct[i]);
    if (a > m1) { m1 = a; i1 = i; }
    if (b > m2) { m2 = b; i2 = i; }
  }
  ShiftParams s;
  s.twin = (m2 > m1) ? 1 : 0;
  size_t i = s.twin ? i2 : i1;
  s.sy = (int)(i / n);
  s.sx = (int)(i % n);
  s.phase = std::arg(s.twin ? ct[i] : c[i]);
  return s;
}

static void apply_shift(const cd* x, const uint8_t* S, int n, const ShiftParams& s, cd* xo,
                        uint8_t* So) {
  cd ph = std::polar(1.0, s.phase);
  for (int r = 0; r < n; r++)
    for (int c = 0; c < n; c++) {
      int yr, xc;
      if (s.twin) {
        yr = ((s.sy - r) % n + n) % n;
        xc = ((s.sx - c) % n + n) % n;
      } else {
        yr = ((r - s.sy) % n + n) % n;
        xc = ((c - s.sx) % n + n) % n;
      }
      size_t src = (size_t)yr * n + xc, dst = (size_t)r * n + c;
      cd v = s.twin ? std::conj(x[src]) : x[src];
      if (xo) xo[dst] = ph * v;
      if (So) So[dst] = S ? S[src] : 0;
    }
}

extern "C" void orc_cross_correlation(const double* x, const double* ref, const uint8_t* mask,
                                      int n, double* c, double* ct) {
  cross_correlations(as_cd(x), as_cd(ref), mask, n, as_cd(c), as_cd(ct));
}

// Align x (and its support) onto ref.  info = (sy, sx, twin); *phase = global phase.
extern "C" void orc_reshift(const double* x, const uint8_t* S, const double* ref,
                            const uint8_t* mask, int n, double* x_out, uint8_t* S_out, int* info,
                            double* phase) {
  ShiftParams s = reshift_params(as_cd(x), as_cd(ref), mask, n);
  apply_shift(as_cd(x), S, n, s, x_out ? as_cd(x_out) : nullptr, S_out);
  if (info) { info[0] = s.sy; info[1] = s.sx; info[2] = s.twin; }
  if (phase) *phase = s.phase;
}

// ------------------------------------------------------------------------------------
// Crossover (App. "Crossover", Alg. crossover) for all P new individuals.
// ------------------------------------------------------------------------------------
struct CrossCfg {
  double cw, cp;
  int tmin, tmax;
  double ca = 0.0;              // crossover averaging C_a
  const double* Mavg = nullptr;  // (M-dot + M-double-dot) / 2, DFT order (C_a > 0)
};

static void crossover_one(const cd* pop_x, const uint8_t* pop_S, const uint8_t* mask, int P,
                          int n, uint64_t seed, int g, int p, const CrossCfg& cf, cd* new_x,
                          uint8_t* new_S, int* abc_out) {
  size_t nn = (size_t)n * n;
  int abc[3];
  random_choice(seed, g, p, P, abc);
  if (abc_out) std::copy(abc, abc + 3, abc_out);
  const cd* xp = pop_x + (size_t)p * nn;
  // Reshift the three parents onto individual p
  std::vector<cd> xa(nn), xb(nn), xc(nn);
  std::vector<uint8_t> Sa(nn), Sb(nn), Sc(nn);
  cd* xs[3] = {xa.data(), xb.data(), xc.data()};
  uint8_t* Ss[3] = {Sa.data(), Sb.data(), Sc.data()};
  for (int k = 0; k < 3; k++) {
    const cd* xk = pop_x + (size_t)abc[k] * nn;
    ShiftParams s = reshift_params(xk, xp, mask, n);
    apply_shift(xk, pop_S + (size_t)abc[k] * nn, n, s, xs[k], Ss[k]);
  }
  // Fourier representations
  std::vector<cd> Xp(xp, xp + nn);
  fft2_inplace(Xp.data(), n, 0);
  for (int k = 0; k < 3; k++) fft2_inplace(xs[k], n, 0);
  // crossover averaging (Eq. crossavg): parent a's moduli move towards the population's
  // average moduli by C_a, its phases are kept (a zero modulus takes phase 0)
  if (cf.ca > 0.0) {
    for (size_t i = 0; i < nn; i++) {
      double a = std::abs(xa[i]);
      double m = cf.ca * cf.Mavg[i] + (1.0 - cf.ca) * a;
      xa[i] = (a > 0.0) ? xa[i] * (m / a) : cd(m, 0.0);
    }
  }
  std::vector<uint8_t> map(nn);
  crossover_map(seed, g, p, n, cf.tmin, cf.tmax, cf.cp, map.data());
  cd* out = new_x + (size_t)p * nn;
  for (size_t i = 0; i < nn; i++)
    out[i] = map[i] ? xa[i] + cf.cw * (xb[i] - xc[i]) : Xp[i];
  fft2_inplace(out, n, 1);
  const uint8_t* Sp = pop_S + (size_t)p * nn;
  uint8_t* So = new_S + (size_t)p * nn;
  for (size_t i = 0; i < nn; i++) So[i] = (Sa[i] | (Sb[i] & Sc[i] & Sp[i])) ? 1 : 0;
}

extern "C" void orc_crossover(const double* pop_x, const uint8_t* pop_S, const uint8_t* mask,
                              int P, int n, uint64_t seed, int g, double cw, double cp, int tmin,
                              int tmax, double* new_x, uint8_t* new_S, int* parents) {
  CrossCfg cf{cw, cp, tmin, tmax};
  parallel_for(P, [&](int p) {
    crossover_one(as_cd(pop_x), pop_S, mask, P, n, seed, g, p, cf, as_cd(new_x), new_S,
                  parents ? parents + 3 * p : nullptr);
  });
}

// the same with crossover averaging: Mavg = (M-dot + M-double-dot) / 2 in DFT order
extern "C" void orc_crossover_ca(const double* pop_x, const uint8_t* pop_S, const uint8_t* mask,
                                 int P, int n, uint64_t seed, int g, double cw, double cp, int tmin,
                                 int tmax, double ca, const double* Mavg, double* new_x,
                                 uint8_t* new_S, int* parents) {
  CrossCfg cf{cw, cp, tmin, tmax, ca, Mavg};
  parallel_for(P, [&](int p) {
    crossover_one(as_cd(pop_x), pop_S, mask, P, n, seed, g, p, cf, as_cd(new_x), new_S,
                  parents ? parents + 3 * p : nullptr);
  });
}

// ------------------------------------------------------------------------------------
// Select (App. "The Selection step", Alg. select): the new individual replaces the old
// one iff its error is strictly lower.  Returns the number of replacements.
// ------------------------------------------------------------------------------------
extern "C" int orc_select(const double* e_old, const double* e_new, int P, uint8_t* replace) {
  int cnt = 0;
  for (int p = 0; p < P; p++) {
    replace[p] = (e_new[p] < e_old[p]) ? 1 : 0;
    cnt += replace[p];
  }
  return cnt;
}

static int argmin_first(const std::vector<double>& e) {
  int b = 0;
  for (int i = 1; i < (int)e.size(); i++)
    if (e[i] < e[b]) b = i;
  return b;
}

// ------------------------------------------------------------------------------------
// Average (Sec. "Monitoring the reconstruction process", Eq. avgrec): every density is
// aligned onto the best one, then averaged; the support is the union of all supports.
// ------------------------------------------------------------------------------------
static void average(const cd* pop_x, const uint8_t* pop_S, const uint8_t* mask, int P, int n,
                    int best, cd* avg, uint8_t* Savg) {
  size_t nn = (size_t)n * n;
  std::vector<std::vector<cd>> al(P, std::vector<cd>(nn));
  std::vector<std::vector<uint8_t>> Sal(P, std::vector<uint8_t>(nn));
  const cd* ref = pop_x + (size_t)best * nn;
  parallel_for(P, [&](int p) {
    const cd* xp = pop_x + (size_t)p * nn;
    const uint8_t* Sp = pop_S + (size_t)p * nn;
    if (p == best) {
      std::copy(xp, xp + nn, al[p].begin());
      std::copy(Sp, Sp + nn, Sal[p].begin());
      return;
    }
    ShiftParams s = reshift_params(xp, ref, mask, n);
    apply_shift(xp, Sp, n, s, al[p].data(), Sal[p].data());
  });
  for (size_t i = 0; i < nn; i++) {
    cd acc = 0;
    uint8_t u = 0;
    for (int p = 0; p < P; p++) {
      acc += al[p][i];
      u |= Sal[p][i];
    }
    avg[i] = acc / (double)P;
    Savg[i] = u ? 1 : 0;
  }
}

extern "C" void orc_average(const double* pop_x, const uint8_t* pop_S, const uint8_t* mask, int P,
                            int n, int best, double* avg, uint8_t* Savg) {
  average(as_cd(pop_x), pop_S, mask, P, n, best, as_cd(avg), Savg);
}

// Complexity Gamma (Eq. complexity) and density sum |sum rho|.
// Average moduli for crossover averaging (App. "Crossover averaging"): M-dot = |F rho_avg|
// of the average reconstruction (Eq. avgint1; rho_avg aligned onto individual `best` as in
// Eq. avgrec), M-double-dot = mean_p |F rho_p| (Eq. avgint2); out = (M-dot + M-double-dot) / 2.
extern "C" void orc_average_moduli(const double* pop_x, const uint8_t* pop_S, const uint8_t* mask,
                                   int P, int n, int best, double* out) {
  size_t nn = (size_t)n * n;
  std::vector<cd> avg(nn);
  std::vector<uint8_t> Savg(nn);
  average(as_cd(pop_x), pop_S, mask, P, n, best, avg.data(), Savg.data());
  fft2_inplace(avg.data(), n, 0);
  std::vector<double> mdd(nn, 0.0);
  std::vector<cd> X(nn);
  for (int p = 0; p < P; p++) {
    std::copy(as_cd(pop_x) + p * nn, as_cd(pop_x) + (p + 1) * nn, X.begin());
    fft2_inplace(X.data(), n, 0);
    for (size_t i = 0; i < nn; i++) mdd[i] += std::abs(X[i]);
  }
  for (size_t i = 0; i < nn; i++) out[i] = 0.5 * (std::abs(avg[i]) + mdd[i] / P);
}

static double complexity(const cd* x, int n, double* sum_abs) {
  cd s = 0;
  double a = 0.0;
  for (size_t i = 0; i < (size_t)n * n; i++) {
    s += x[i];
    a += std::abs(x[i]);
  }
  *sum_abs = std::abs(s);
  return a > 0.0 ? 1.0 - std::abs(s) / a : 0.0;
}

extern "C" double orc_complexity(const double* x, int n, double* sum_abs) {
  return complexity(as_cd(x), n, sum_abs);
}

// ------------------------------------------------------------------------------------
// Initialize (App. "Initialization of the starting densities", Eq. norm).
// Sigma_init is the side of the bounding square of the initial support.  Each density
// is a sum of N_init projected spheres (thickness 2 sqrt(R^2 - d^2)) with diameters in
// [0.2, 0.9] Sigma_init, centres inside the square and phases in [-phi_max, phi_max];
// then |rho|^gamma (phase kept), restriction to the support, and the scale sqrt(nu)
// that matches the known part of the Fourier power (Eq. norm read as an intensity ratio).
// ------------------------------------------------------------------------------------
struct InitCfg {
  int n_spheres;
  double gamma, phi_max;
};

static bool support_box(const uint8_t* S0, int n, double* y0, double* x0, double* side) {
  int r0 = n, r1 = -1, c0 = n, c1 = -1;
  for (int r = 0; r < n; r++)
    for (int c = 0; c < n; c++)
      if (S0[(size_t)r * n + c]) {
        r0 = std::min(r0, r); r1 = std::max(r1, r);
        c0 = std::min(c0, c); c1 = std::max(c1, c);
      }
  if (r1 < 0) return false;
  double h = r1 - r0 + 1, w = c1 - c0 + 1;
  *side = std::max(h, w);
  *y0 = r0 + (h - *side) / 2.0;
  *x0 = c0 + (w - *side) / 2.0;
  return true;
}

static inline double unit24(uint32_t u) { return (double)(u >> 8) * (1.0 / 16777216.0); }

static void initialize_one(uint64_t seed, int p, const uint8_t* S0, const double* I,
                           const uint8_t* mask, int n, const InitCfg& cf, cd* x) {
  size_t nn = (size_t)n * n;
  std::fill(x, x + nn, cd(0.0, 0.0));
  double y0, x0, side;
  if (!support_box(S0, n, &y0, &x0, &side)) return;
  for (int s = 0; s < cf.n_spheres; s++) {
    uint32_t u[4];
    draw(seed, 0u, (uint32_t)p, 4, (uint32_t)s, 0u, u);
    double D = side * (0.2 + 0.7 * unit24(u[0]));
    double R = D / 2.0;
    double cy = y0 + R + unit24(u[1]) * (side - D);
    double cx = x0 + R + unit24(u[2]) * (side - D);
    double phi = cf.phi_max * (2.0 * unit24(u[3]) - 1.0);
    cd e = std::polar(1.0, phi);
    for (int r = 0; r < n; r++)
      for (int c = 0; c < n; c++) {
        double d2 = (r - cy) * (r - cy) + (c - cx) * (c - cx);
        if (d2 < R * R) x[(size_t)r * n + c] += e * (2.0 * std::sqrt(R * R - d2));
      }
  }
  for (size_t i = 0; i < nn; i++) {
    double a = std::abs(x[i]);
    if (a > 0.0 && cf.gamma != 1.0) x[i] *= std::pow(a, cf.gamma) / a;
    if (!S0[i]) x[i] = 0.0;
  }
  std::vector<cd> X(x, x + nn);
  fft2_inplace(X.data(), n, 0);
  double num = 0.0, den = 0.0;
  for (size_t i = 0; i < nn; i++)
    if (mask[i]) {
      num += I[i];
      den += std::norm(X[i]);
    }
  if (den > 0.0) {
    double sc = std::sqrt(num / den);
    for (size_t i = 0; i < nn; i++) x[i] *= sc;
  }
}

// I and mask in DFT order; S0 in real space.
extern "C" void orc_initialize(uint64_t seed, const uint8_t* S0, const double* I,
                               const uint8_t* mask, int n, int P, int n_spheres, double gamma,
                               double phi_max, double* x) {
  InitCfg cf{n_spheres, gamma, phi_max};
  size_t nn = (size_t)n * n;
  parallel_for(P, [&](int p) { initialize_one(seed, p, S0, I, mask, n, cf, as_cd(x) + p * nn); });
}

// ------------------------------------------------------------------------------------
// MPR (Sec. "Memetic Phase Retrieval", Alg. mpr) with the self-improvement of
// App. "The self-improvement" (Alg. improve) in the iteration-count form:
//   R = iters / K blocks; blocks 1..R-2: K IA iterations + UpdateSupport;
//   block R-1: K IA iterations + UpdateSupportSize(alpha_best);
//   block R: (rest - n_ER) IA iterations + UpdateSupportSize(alpha_eval),
//            n_ER ER iterations (EvalSequence), GetError, UpdateSupport.
// ------------------------------------------------------------------------------------
struct orc_params {
  int pop, iters_per_gen, generations, algorithm;
  double beta, sw_sigma, sw_threshold, sw_sigma_end, sw_threshold_end;
  int sw_period, er_tail;
  double chi, cw, cp;
  int tile_min, tile_max, init_n_spheres;
  double init_gamma, init_phi_max;
  uint64_t seed;
  double ub_eta, ub_max_missing, ub_max_saturated;  // upper bounds (eta <= 0: off)
  // schedule 0: the configs' blocks (iters_per_gen, sw_period, er_tail); schedule 1: the
  // paper's Sequence of seq_ia IA + seq_er ER iterations repeated `repetitions` times, with
  // seq_eval ER iterations of EvalSequence (App. "The algorithms sequence")
  int schedule;
  // mode 0: MPR (Alg. mpr); mode 1: independent reconstructions (Alg. randomsearch)
  int mode;
  int seq_ia, seq_er, seq_eval, repetitions;
  double ca;  // crossover averaging C_a (App. "Crossover averaging"), 0 = off
  int monitor_avg;  // 1: the average reconstruction's error every generation
};

struct orc_result {
  double* rho_avg;      // n*n interleaved complex (real-space order), may be null
  double* rho_best;     // same, may be null
  uint8_t* support_avg; // n*n, may be null
  double* pop_x;        // P*n*n interleaved complex final population, may be null
  uint8_t* pop_S;       // P*n*n final supports, may be null
  double* pop_err;      // P final errors, may be null
  double* gen_stats;    // G x 9, may be null
  double final_error_avg, final_error_best;
};

static long area(const uint8_t* S, size_t nn) {
  long a = 0;
  for (size_t i = 0; i < nn; i++) a += S[i] ? 1 : 0;
  return a;
}

// Sequence lengths of generation g (App. "Changing values over generations", "The
// algorithms sequence"): the IA count falls linearly from seq_ia to 0 and the ER count rises
// from seq_er to seq_ia + seq_er over g = 1..G, each rounded to the nearest integer (halves
// up), evaluated exactly in integers.
static void sequence_counts(const orc_params& pr, int g, int G, int* ia, int* er) {
  if (G <= 1) {
    *ia = pr.seq_ia;
    *er = pr.seq_er;
    return;
  }
  const long den = 2L * (G - 1);
  *ia = (int)((2L * pr.seq_ia * (G - g) + (G - 1)) / den);
  *er = pr.seq_er + (int)((2L * pr.seq_ia * (g - 1) + (G - 1)) / den);
}

extern "C" void orc_sequence_counts(int seq_ia, int seq_er, int g, int G, int* out) {
  orc_params pr{};
  pr.seq_ia = seq_ia;
  pr.seq_er = seq_er;
  sequence_counts(pr, g, G, &out[0], &out[1]);
}

// Sequence (Eq. sequence): ia iterations of the IA (HIO or RAAR), then er of ER
static void sequence(cd* x, const uint8_t* S, const double* M, const uint8_t* mask, const double* U,
                     int n, const orc_params& pr, int ia, int er) {
  iterate_one(x, S, M, mask, U, n, pr.algorithm, pr.beta, pr.chi, ia);
  iterate_one(x, S, M, mask, U, n, 0, pr.beta, pr.chi, er);
}

// Self-improvement of one individual (Alg. improve; Eq. sequence; App. "The modified
// Shrink-wrap").  A generation's iterations fall into R blocks, each an iteration segment
// followed by a support update.  The update after a block depends on its position: the
// plain Shrink-wrap threshold after the first R - 2 blocks, the support resized to the best
// parent's area after block R - 1, and to alpha_eval after block R.  Then come the ER
// iterations of the evaluation sequence, the error (Eq. error_calc) and a last plain
// Shrink-wrap.  The two schedules differ only in the segments:
//   schedule 1 (the paper's Sequence): every block is seq(ia IA + er ER) with the counts
//     of generation g, and the evaluation sequence has seq_eval ER iterations;
//   schedule 0 (the configs: N_it iterations, support update every K, last er_tail ER):
//     blocks of K IA iterations, the last block shortened to N_it - (R - 1) K - er_tail so
//     that the er_tail ER iterations of the evaluation sequence complete N_it.
static void improve_one(cd* x, uint8_t* S, const double* M, const uint8_t* mask, const double* U,
                        int n, const orc_params& pr, double sigma, double tau, long a_best, long a_eval,
                        double* err, int g, int G) {
  int R, ia = 0, er = 0, eval_er;
  if (pr.schedule == 1) {
    R = pr.repetitions;
    sequence_counts(pr, g, G, &ia, &er);
    eval_er = pr.seq_eval;
  } else {
    R = pr.iters_per_gen / pr.sw_period;
    eval_er = pr.er_tail;
  }
  for (int blk = 1; blk <= R; blk++) {
    if (pr.schedule == 1) {
      sequence(x, S, M, mask, U, n, pr, ia, er);
    } else {
      const int len = blk < R ? pr.sw_period : pr.iters_per_gen - (R - 1) * pr.sw_period - pr.er_tail;
      iterate_one(x, S, M, mask, U, n, pr.algorithm, pr.beta, pr.chi, len);
    }
    if (blk <= R - 2)
      update_support(x, S, n, sigma, tau);
    else
      update_support_size(x, S, n, sigma, blk == R - 1 ? a_best : a_eval);
  }
  iterate_one(x, S, M, mask, U, n, 0, pr.beta, pr.chi, eval_er);  // EvalSequence: ER only
  *err = fourier_error(x, S, M, mask, n);
  update_support(x, S, n, sigma, tau);
}

// Improve of the independent reconstructions (Alg. normalimprove): a Sequence and an
// UpdateSupport per generation.  Schedule 0 splits the generation's iterations into blocks
// of sw_period, each followed by UpdateSupport, the last er_tail iterations being ER.  The
// error (Eq. error_calc) is taken after the last Sequence, before the last UpdateSupport.
static void improve_independent(cd* x, uint8_t* S, const double* M, const uint8_t* mask,
                                const double* U, int n, const orc_params& pr, double sigma,
                                double tau, double* err, int g, int G) {
  if (pr.schedule == 1) {
    int ia, er;
    sequence_counts(pr, g, G, &ia, &er);
    sequence(x, S, M, mask, U, n, pr, ia, er);
  } else {
    int K = pr.sw_period, R = pr.iters_per_gen / K;
    int last = pr.iters_per_gen - (R - 1) * K;
    for (int blk = 1; blk < R; blk++) {
      iterate_one(x, S, M, mask, U, n, pr.algorithm, pr.beta, pr.chi, K);
      update_support(x, S, n, sigma, tau);
    }
    sequence(x, S, M, mask, U, n, pr, last - pr.er_tail, pr.er_tail);
  }
  *err = fourier_error(x, S, M, mask, n);
  update_support(x, S, n, sigma, tau);
}

static void ifftshift2(const void* src, void* dst, int n, size_t esz) {
  // DFT-order index (r, c) takes the detector-centred value at ((r + n/2) % n, (c + n/2) % n)
  const char* s = (const char*)src;
  char* d = (char*)dst;
  int h = n / 2;
  for (int r = 0; r < n; r++)
    for (int c = 0; c < n; c++)
      std::memcpy(d + ((size_t)r * n + c) * esz, s + ((size_t)((r + h) % n) * n + (c + h) % n) * esz,
                  esz);
}

// Checks of a run's parameters; true if a run can be made with them.
static bool valid_run_params(const orc_params& pr, int n) {
  if (!valid_side(n) || pr.pop < 4 || pr.generations < 1) return false;
  if (pr.mode != 0 && pr.mode != 1) return false;
  if (pr.schedule == 0) {
    if (pr.sw_period < 1) return false;
    int R = pr.iters_per_gen / pr.sw_period;
    if (R < 2) return false;
    int last = pr.iters_per_gen - (R - 1) * pr.sw_period;
    if (pr.er_tail < 0 || pr.er_tail > last) return false;
  } else if (pr.schedule == 1) {
    if (pr.repetitions < 2 || pr.seq_ia < 0 || pr.seq_er < 0 || pr.seq_eval < 0) return false;
    if (pr.seq_ia + pr.seq_er < 1) return false;
  } else {
    return false;
  }
  return true;
}

// The pattern as a run uses it: moduli M = sqrt(I), the mask and (if enabled) the upper
// bounds of the missing intensities (Eq. pm_bounds), all in DFT order.
struct RunProblem {
  int n = 0;
  size_t nn = 0;
  std::vector<double> M, U;
  std::vector<uint8_t> mask;
  const double* Up = nullptr;
};

static void make_problem(const double* I_c, const uint8_t* mask_c, const uint8_t* sat_c, int n,
                         const orc_params& pr, RunProblem* pb) {
  pb->n = n;
  pb->nn = (size_t)n * n;
  std::vector<double> I(pb->nn);
  pb->M.resize(pb->nn);
  pb->mask.resize(pb->nn);
  ifftshift2(I_c, I.data(), n, sizeof(double));
  ifftshift2(mask_c, pb->mask.data(), n, 1);
  for (size_t i = 0; i < pb->nn; i++) pb->M[i] = std::sqrt(std::max(0.0, I[i]));
  if (pr.ub_eta > 0.0) {
    std::vector<double> Uc(pb->nn);
    orc_upper_bounds(I_c, mask_c, sat_c, n, pr.ub_eta, pr.ub_max_missing, pr.ub_max_saturated, Uc.data());
    pb->U.resize(pb->nn);
    ifftshift2(Uc.data(), pb->U.data(), n, sizeof(double));
    pb->Up = pb->U.data();
  }
}

// The state of a run: the parent population (x, S, errors) and the new individuals that a
// generation's crossover produces.
struct RunPop {
  std::vector<cd> px, nx;
  std::vector<uint8_t> pS, nS;
  std::vector<double> pe, ne;
  void resize(int P, size_t nn) {
    px.resize(P * nn);
    nx.resize(P * nn);
    pS.resize(P * nn);
    nS.resize(P * nn);
    pe.assign(P, std::numeric_limits<double>::infinity());
    ne.assign(P, 0.0);
  }
};

// What one generation decided (orc_mpr_step); pointer members may be null.
struct orc_trace {
  double* err_parents;  // P: errors of the improved parents, before Select
  double* err_new;      // P: errors of the improved new individuals
  uint8_t* replaced;    // P: 1 where Select took the new individual
  int* parents;         // 3 P: (a, b, c) of new individual p at 3p .. 3p + 2
  int64_t areas[3];     // alpha_best, alpha_all, alpha_eval of Alg. improve
  int best;             // the parent whose area is alpha_best
  double gen_stats[9];  // this generation's monitors (the gen_stats row)
};

// Per-generation monitors (Sec. "Monitoring the reconstruction process") of the parent
// population after Select: best, mean and worst error, E(avg) (NaN unless monitored),
// O_d, replacement fraction, mean Gamma, mean |sum rho| and its relative spread.
static void monitors(const RunProblem& pb, const orc_params& pr, int g, int G, const RunPop& pop, int repl,
                     double* st) {
  const int P = pr.pop, n = pb.n;
  const size_t nn = pb.nn;
  int b = argmin_first(pop.pe);
  double mn = 0.0, mx = pop.pe[0], gam = 0.0, sm = 0.0;
  std::vector<double> sums(P);
  for (int p = 0; p < P; p++) {
    mn += pop.pe[p];
    mx = std::max(mx, pop.pe[p]);
    gam += complexity(&pop.px[p * nn], n, &sums[p]);
    sm += sums[p];
  }
  st[0] = pop.pe[b];
  st[1] = mn / P;
  st[2] = mx;
  st[3] = std::numeric_limits<double>::quiet_NaN();  // E(avg): final generation (set by the run)
  if (pr.monitor_avg && g < G) {  // Sec. "Monitoring the reconstruction process"
    std::vector<cd> av(nn);
    std::vector<uint8_t> Sv(nn);
    average(pop.px.data(), pop.pS.data(), pb.mask.data(), P, n, b, av.data(), Sv.data());
    st[3] = fourier_error(av.data(), Sv.data(), pb.M.data(), pb.mask.data(), n);
  }
  st[4] = (double)nn / (double)std::max(1L, area(&pop.pS[b * nn], nn));
  st[5] = (double)repl / P;
  st[6] = gam / P;
  st[7] = sm / P;
  // spread of the density sums (Sec. "Crossover averaging"): population standard
  // deviation relative to the mean, by the two-pass formula
  double var = 0.0;
  for (int p = 0; p < P; p++) var += (sums[p] - sm / P) * (sums[p] - sm / P);
  st[8] = sm > 0.0 ? std::sqrt(var / P) / (sm / P) : 0.0;
}

// Linear parameter schedule over generations (App. "Changing values over generations")
static void sw_params(const orc_params& pr, int g, int G, double* sigma, double* tau) {
  double t = (G > 1) ? (double)(g - 1) / (double)(G - 1) : 0.0;
  *sigma = pr.sw_sigma + (pr.sw_sigma_end - pr.sw_sigma) * t;
  *tau = pr.sw_threshold + (pr.sw_threshold_end - pr.sw_threshold) * t;
}

// Generation g of the independent reconstructions (Alg. randomsearch): Improve only.
static void independent_generation(const RunProblem& pb, const orc_params& pr, int g, RunPop& pop, double* st) {
  const int P = pr.pop, G = pr.generations;
  const size_t nn = pb.nn;
  double sigma, tau;
  sw_params(pr, g, G, &sigma, &tau);
  parallel_for(P, [&](int p) {
    improve_independent(&pop.px[p * nn], &pop.pS[p * nn], pb.M.data(), pb.mask.data(), pb.Up, pb.n, pr, sigma,
                        tau, &pop.pe[p], g, G);
  });
  monitors(pb, pr, g, G, pop, 0, st);
}

// Generation g of MPR (Alg. mpr): Crossover of the parents into new individuals, the
// areas of Alg. improve from the parents, Improve of both populations, Select.
static void mpr_generation(const RunProblem& pb, const orc_params& pr, int g, RunPop& pop, orc_trace* tr,
                           double* st) {
  const int P = pr.pop, G = pr.generations, n = pb.n;
  const size_t nn = pb.nn;
  CrossCfg cf{pr.cw, pr.cp, pr.tile_min, pr.tile_max};
  std::vector<double> Mavg;
  if (pr.ca > 0.0) {  // the parents' average moduli for crossover averaging
    Mavg.resize(nn);
    orc_average_moduli(reinterpret_cast<const double*>(pop.px.data()), pop.pS.data(), pb.mask.data(), P, n,
                       argmin_first(pop.pe), Mavg.data());
    cf.ca = pr.ca;
    cf.Mavg = Mavg.data();
  }
  // Crossover (Alg. crossover): new population from the parents
  parallel_for(P, [&](int p) {
    crossover_one(pop.px.data(), pop.pS.data(), pb.mask.data(), P, n, pr.seed, g, p, cf, pop.nx.data(),
                  pop.nS.data(), nullptr);
  });
  // Areas (Alg. improve, first three steps), from the parent population
  int best = (g == 1) ? 0 : argmin_first(pop.pe);
  long a_best = area(&pop.pS[best * nn], nn);
  std::vector<uint8_t> uni(nn, 0);
  for (int p = 0; p < P; p++)
    for (size_t i = 0; i < nn; i++) uni[i] |= pop.pS[p * nn + i];
  long a_all = area(uni.data(), nn);
  // alpha_eval = (g/G) alpha_best + (1 - g/G) alpha_all, rounded half up; evaluated
  // exactly in integers so that no floating-point contraction can move a half-way case
  long a_eval = (2L * ((long)g * a_best + (long)(G - g) * a_all) + G) / (2L * G);
  double sigma, tau;
  sw_params(pr, g, G, &sigma, &tau);
  // Improve both populations
  parallel_for(2 * P, [&](int q) {
    bool old = q < P;
    int p = old ? q : q - P;
    cd* x = old ? &pop.px[p * nn] : &pop.nx[p * nn];
    uint8_t* S = old ? &pop.pS[p * nn] : &pop.nS[p * nn];
    double* e = old ? &pop.pe[p] : &pop.ne[p];
    improve_one(x, S, pb.M.data(), pb.mask.data(), pb.Up, n, pr, sigma, tau, a_best, a_eval, e, g, G);
  });
  if (tr) {
    if (tr->err_parents) std::copy(pop.pe.begin(), pop.pe.end(), tr->err_parents);
    if (tr->err_new) std::copy(pop.ne.begin(), pop.ne.end(), tr->err_new);
    if (tr->parents)
      for (int p = 0; p < P; p++) random_choice(pr.seed, g, p, P, &tr->parents[3 * p]);
    tr->areas[0] = a_best;
    tr->areas[1] = a_all;
    tr->areas[2] = a_eval;
    tr->best = best;
  }
  // Select (Alg. select): strict <, ties keep the parent
  int repl = 0;
  for (int p = 0; p < P; p++) {
    const bool r = pop.ne[p] < pop.pe[p];
    if (r) {
      std::copy(pop.nx.begin() + p * nn, pop.nx.begin() + (p + 1) * nn, pop.px.begin() + p * nn);
      std::copy(pop.nS.begin() + p * nn, pop.nS.begin() + (p + 1) * nn, pop.pS.begin() + p * nn);
      pop.pe[p] = pop.ne[p];
      repl++;
    }
    if (tr && tr->replaced) tr->replaced[p] = r ? 1 : 0;
  }
  monitors(pb, pr, g, G, pop, repl, st);
}

// Returns 0 on success, 1 on invalid parameters.  I, mask: detector-centred; S0 real space.
// sat_c: detector-centred saturation map (may be null), used by the upper bounds only
extern "C" int orc_mpr_run_sat(const double* I_c, const uint8_t* mask_c, const uint8_t* sat_c,
                               const uint8_t* S0, int n, const orc_params* prm, orc_result* res) {
  const orc_params& pr = *prm;
  if (!valid_run_params(pr, n)) return 1;
  RunProblem pb;
  make_problem(I_c, mask_c, sat_c, n, pr, &pb);
  const size_t nn = pb.nn;
  const int P = pr.pop, G = pr.generations;
  std::vector<double> I(nn);
  ifftshift2(I_c, I.data(), n, sizeof(double));
  RunPop pop;
  pop.resize(P, nn);
  orc_initialize(pr.seed, S0, I.data(), pb.mask.data(), n, P, pr.init_n_spheres, pr.init_gamma,
                 pr.init_phi_max, reinterpret_cast<double*>(pop.px.data()));
  for (int p = 0; p < P; p++) std::copy(S0, S0 + nn, pop.pS.begin() + p * nn);
  double scratch[9];
  for (int g = 1; g <= G; g++) {
    double* st = res->gen_stats ? res->gen_stats + (size_t)(g - 1) * 9 : scratch;
    if (pr.mode == 1)
      independent_generation(pb, pr, g, pop, st);
    else
      mpr_generation(pb, pr, g, pop, nullptr, st);
  }
  int b = argmin_first(pop.pe);
  std::vector<cd> avg(nn);
  std::vector<uint8_t> Savg(nn);
  average(pop.px.data(), pop.pS.data(), pb.mask.data(), P, n, b, avg.data(), Savg.data());
  res->final_error_avg = fourier_error(avg.data(), Savg.data(), pb.M.data(), pb.mask.data(), n);
  res->final_error_best = pop.pe[b];
  if (res->gen_stats) res->gen_stats[(size_t)(G - 1) * 9 + 3] = res->final_error_avg;
  if (res->rho_avg) std::copy(avg.begin(), avg.end(), as_cd(res->rho_avg));
  if (res->rho_best) std::copy(pop.px.begin() + b * nn, pop.px.begin() + (b + 1) * nn, as_cd(res->rho_best));
  if (res->support_avg) std::copy(Savg.begin(), Savg.end(), res->support_avg);
  if (res->pop_x) std::copy(pop.px.begin(), pop.px.end(), as_cd(res->pop_x));
  if (res->pop_S) std::copy(pop.pS.begin(), pop.pS.end(), res->pop_S);
  if (res->pop_err) std::copy(pop.pe.begin(), pop.pe.end(), res->pop_err);
  return 0;
}

extern "C" int orc_mpr_run(const double* I_c, const uint8_t* mask_c, const uint8_t* S0, int n,
                           const orc_params* prm, orc_result* res) {
  return orc_mpr_run_sat(I_c, mask_c, nullptr, S0, n, prm, res);
}

// One generation g = g_from + 1 of the run (1 <= g <= G) from a given parent population
// (pop_x: P x n x n interleaved complex, pop_S, pop_err; errors +inf before generation 1),
// which it replaces by the population after that generation.  tr (may be null) receives
// what the generation decided.  Returns 0 on success, 1 on invalid arguments.
extern "C" int orc_mpr_step(const double* I_c, const uint8_t* mask_c, const uint8_t* sat_c, int n,
                            const orc_params* prm, int g_from, double* pop_x, uint8_t* pop_S, double* pop_err,
                            orc_trace* tr) {
  const orc_params& pr = *prm;
  if (!valid_run_params(pr, n) || g_from < 0 || g_from >= pr.generations) return 1;
  RunProblem pb;
  make_problem(I_c, mask_c, sat_c, n, pr, &pb);
  const size_t nn = pb.nn;
  const int P = pr.pop, g = g_from + 1;
  RunPop pop;
  pop.resize(P, nn);
  std::copy(as_cd(pop_x), as_cd(pop_x) + P * nn, pop.px.begin());
  std::copy(pop_S, pop_S + P * nn, pop.pS.begin());
  std::copy(pop_err, pop_err + P, pop.pe.begin());
  double scratch[9];
  double* st = tr ? tr->gen_stats : scratch;
  if (pr.mode == 1)
    independent_generation(pb, pr, g, pop, st);
  else
    mpr_generation(pb, pr, g, pop, tr, st);
  std::copy(pop.px.begin(), pop.px.end(), as_cd(pop_x));
  std::copy(pop.pS.begin(), pop.pS.end(), pop_S);
  std::copy(pop.pe.begin(), pop.pe.end(), pop_err);
  return 0;
}

// Improve on an explicit batch (used by the CPU-baseline timing and by parity tests of
// the whole self-improvement step).  x, S: batch images; err: batch errors out.
extern "C" int orc_improve(double* x, uint8_t* S, const double* M, const uint8_t* mask, int batch,
                           int n, const orc_params* prm, double sigma, double tau, long a_best,
                           long a_eval, double* err) {
  const orc_params& pr = *prm;
  if (!valid_side(n) || pr.sw_period < 1) return 1;
  int R = pr.iters_per_gen / pr.sw_period;
  if (R < 2) return 1;
  int last = pr.iters_per_gen - (R - 1) * pr.sw_period;
  if (pr.er_tail < 0 || pr.er_tail > last) return 1;
  size_t nn = (size_t)n * n;
  parallel_for(batch, [&](int b) {
    improve_one(as_cd(x) + b * nn, S + b * nn, M, mask, nullptr, n, pr, sigma, tau, a_best, a_eval,
                &err[b], 1, 1);
  });
  return 0;
}
