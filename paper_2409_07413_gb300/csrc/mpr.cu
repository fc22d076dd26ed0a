// mpr.cu -- the MPR run (Alg. mpr) on one GPU, contexts, problems and serving.
//
// A run keeps its whole state resident on the device: two populations of P densities
// (x), their supports (S), the FFT intermediate (w), the smoothed maps of shrink-wrap and
// the per-individual errors.  Every decision of the run (best individual, areas, parents,
// crossover tiles, selection) is taken on the device, so one run is a fixed sequence of
// kernel launches with no host round trip: it can be enqueued generation by generation
// (serving) or captured whole in a CUDA graph.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <limits>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <nvtx3/nvToolsExt.h>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"

using namespace spring;

struct spring_problem {
  spring_ctx* ctx = nullptr;
  int n = 0;
  float* M = nullptr;     // device, N x N, DFT order, negative = not measured
  float* s16 = nullptr;   // device scalar in M's allocation (M + N x N): FP16 storage scale
  uint8_t* S0 = nullptr;  // device, N x N, initial support (real space)
  std::atomic<int> refs{0};
};

namespace spring {

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static spring_status validate_params(int n, const spring_params& p) {
  if (!valid_n(n)) return invalid("unsupported pattern side");
  if (p.pop < 4) return invalid("pop must be >= 4");
  if (p.generations < 1) return invalid("generations must be >= 1");
  if (p.algorithm < 0 || p.algorithm > 2) return invalid("algorithm must be 0, 1 or 2");
  if (!(p.beta > 0.f && p.beta <= 1.f)) return invalid("beta must be in (0, 1]");
  if (p.mode != 0 && p.mode != 1) return invalid("mode must be 0 (MPR) or 1 (independent reconstructions)");
  if (p.schedule == 0) {
    if (p.sw_period < 1) return invalid("sw_period must be >= 1");
    const int R = p.iters_per_gen / p.sw_period;
    if (R < 2) return invalid("iters_per_gen must be >= 2 * sw_period (R >= 2 repetitions)");
    const int last = p.iters_per_gen - (R - 1) * p.sw_period;
    if (p.er_tail < 0 || p.er_tail > last) return invalid("er_tail must be in [0, last block length]");
  } else if (p.schedule == 1) {
    if (p.repetitions < 2) return invalid("repetitions must be >= 2");
    if (p.seq_ia < 0 || p.seq_er < 0 || p.seq_eval < 0) return invalid("sequence lengths must be >= 0");
    if (p.seq_ia + p.seq_er < 1) return invalid("a Sequence needs at least one iteration");
  } else {
    return invalid("schedule must be 0 (blocks) or 1 (the paper's Sequence)");
  }
  if (!(p.ca >= 0.f && p.ca <= 1.f)) return invalid("ca must be in [0, 1]");
  if (!(p.sw_sigma >= 0.f && p.sw_sigma <= 64.f && p.sw_sigma_end >= 0.f && p.sw_sigma_end <= 64.f))
    return invalid("shrink-wrap sigma must be in [0, 64]");
  if (!(p.sw_threshold > 0.f && p.sw_threshold <= 1.f && p.sw_threshold_end > 0.f && p.sw_threshold_end <= 1.f))
    return invalid("shrink-wrap threshold must be in (0, 1]");
  if (!(p.chi > 0.f)) return invalid("chi must be > 0");
  if (!(p.cw >= 0.f && p.cw <= 2.f)) return invalid("cw must be in [0, 2]");
  if (!(p.cp >= 0.f && p.cp <= 1.f)) return invalid("cp must be in [0, 1]");
  if (p.tile_min < 1) return invalid("tile_min must be >= 1");
  if (p.init_n_spheres < 1) return invalid("init_n_spheres must be >= 1");
  if (!(p.init_gamma > 0.f)) return invalid("init_gamma must be > 0");
  if (p.precision != 0 && p.precision != 1) return invalid("precision must be 0 (FP32) or 1 (FP16 storage)");
  return SPRING_OK;
}

// ------------------------------------------------------------------ device layout of a run
struct Layout {
  size_t x, w, S, Sb, sm0, sm1, err, abc, ix, ir, info, best, ph, alpha, repl, dens, part_err,
      part_norm, part_dens, imgmax, stats, avg, Savg, err_avg, status, peaks, init, mavg, mall, msplit, m2, total;
};

static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// K patterns of side n run together (K = 1: a single run); per-pattern state is K times
// the single run's, GA scratch is shared (the patterns' GA steps run one after another)
static Layout make_layout(int n, const spring_params& p, int K = 1) {
  const size_t nn = (size_t)n * n, P = p.pop, B = 2 * P * K, G = p.generations, Q = 3 * P;
  Layout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o += align256(bytes);
    return at;
  };
  L.x = take(sizeof(float2) * B * nn);
  L.w = take(sizeof(float2) * B * nn);
  L.S = take(B * nn);
  L.Sb = take(B * nn / 8);  // the supports packed to one bit per pixel for the row pass
  L.sm0 = take(sizeof(float) * B * nn);
  L.sm1 = take(sizeof(float) * B * nn);
  L.err = take(sizeof(double) * B);
  L.abc = take(sizeof(int32_t) * Q);
  L.ix = take(sizeof(int32_t) * Q);
  L.ir = take(sizeof(int32_t) * Q);
  L.info = take(sizeof(int32_t) * 3 * Q);
  L.best = take(sizeof(int32_t) * 4 * K);
  L.ph = take(sizeof(float2) * Q);
  L.alpha = take(sizeof(int64_t) * 4 * K);
  L.repl = take(P);
  L.dens = take(sizeof(double) * 2 * P);
  L.part_err = take(sizeof(double) * 2 * B * err_strips(n));
  L.part_norm = take(normalise_scratch_bytes((int)P));
  L.part_dens = take(density_scratch_bytes((int)P));
  L.imgmax = take(sizeof(unsigned) * B);
  L.stats = take(sizeof(double) * SPRING_GEN_STATS_COLS * G * K);
  L.avg = take(sizeof(float2) * nn * K);
  L.Savg = take(nn * K);
  L.err_avg = take(sizeof(double) * 2 * K);
  L.status = take(sizeof(int) * 4);
  L.peaks = take(peaks_scratch_bytes(n, (int)P));
  L.init = take(init_scratch_bytes((int)P, p.init_n_spheres) + 128);
  L.mavg = take(p.ca > 0.f ? sizeof(float) * nn : 0);
  L.mall = take(K > 1 ? sizeof(float) * nn * K : 0);  // the K modulus arrays, gathered
  L.msplit = take(split_supported(n) ? sizeof(float) * nn * K : 0);  // M in the split passes' layout
  L.m2 = take(sizeof(double) * K);  // sum of M^2 over the measured pixels, per pattern
  L.total = o;
  return L;
}

// Host-side NVTX range around one phase of a run (enqueue time; a profiler attributes
// the kernels launched inside it to the phase).  No-op unless a tool is attached.
struct Phase {
  explicit Phase(const char* name) { nvtxRangePushA(name); }
  ~Phase() { nvtxRangePop(); }
  Phase(const Phase&) = delete;
  Phase& operator=(const Phase&) = delete;
};

class Run {
 public:
  // B: image slots (both populations); NB: individuals improved per generation (B for MPR,
  // P for independent reconstructions, which use the second half as scratch)
  int n = 0, P = 0, B = 0, NB = 0, G = 0, R = 0, last = 0;
  // a batch: K patterns of side n, each with its own population (B image slots each, one
  // after another); whole-batch launches cover NBT = K NB images; the GA steps of pattern
  // cq use the accessors below
  int K = 1, cq = 0, NBT = 0;
  std::vector<const spring_problem*> probs;
  std::vector<uint64_t> seeds;
  const float* Mall = nullptr;  // K modulus arrays one after another (K = 1: the problem's)
  int mgroup = 0;               // images per modulus array in whole-batch launches (0: one)
  spring_params prm{};
  const float* s16 = nullptr;  // FP16 storage scale of the problem (device scalar)
  cudaStream_t s = nullptr;
  char* mem = nullptr;
  Layout L{};
  int next_gen = 1;  // generation to enqueue next (G + 1: finish; G + 2: done)
  int stop_after = 0;    // > 0: stop after this generation (no average)
  bool resumed = false;  // the population was uploaded (checkpoint): no Initialize
  int first_gen = 1;     // first generation this run executes

  float2 *x = nullptr, *w = nullptr, *avg = nullptr;
  uint8_t *S = nullptr, *repl = nullptr, *Savg = nullptr;
  uint32_t* Sb = nullptr;  // S packed to bits (before each block of iterations)
  float *sm0 = nullptr, *sm1 = nullptr;
  double *err = nullptr, *dens = nullptr, *part_err = nullptr, *part_norm = nullptr,
         *part_dens = nullptr, *stats = nullptr, *err_avg = nullptr;
  int32_t *abc = nullptr, *ix = nullptr, *ir = nullptr, *info = nullptr, *best = nullptr;
  float2* ph = nullptr;
  int64_t* alpha = nullptr;
  unsigned* imgmax = nullptr;
  int* status = nullptr;
  float* mavg = nullptr;  // crossover averaging: (M-dot + M-double-dot) / 2
  float* Msplit = nullptr;  // the K modulus arrays in the split column pass's layout (split sides)
  double* m2 = nullptr;     // per pattern: sum of M^2 over its measured pixels (Eq. error_calc)
  // spring_mpr_step's trace (single-pattern runs): the improved parents' errors before
  // Select, and the parent whose area is alpha_best (device buffers owned by the caller)
  double* tr_err = nullptr;
  int32_t* tr_best = nullptr;
  void *peaks = nullptr, *init_sc = nullptr;
  bool z_valid = false;
  int z_path = 0;  // layout of the spectra in w while z_valid: 0 natural rows, 2 chunked (split passes)
  // precision 1: the iteration blocks keep x and w as half2 inside the w buffer
  bool fp16 = false, z16_valid = false, x16_newer = false;

  ~Run() { release(); }

  void release() {
    if (mem) {
      cudaFreeAsync(mem, s);
      mem = nullptr;
    }
  }

  spring_status setup(const spring_problem* prob, const spring_params& p, cudaStream_t stream) {
    return setup_batch(&prob, 1, &p.seed, p, stream);
  }

  spring_status setup_batch(const spring_problem* const* pr, int k, const uint64_t* sd, const spring_params& p,
                            cudaStream_t stream) {
    K = k;
    probs.assign(pr, pr + k);
    seeds.assign(sd, sd + k);
    n = pr[0]->n;
    prm = p;
    P = p.pop;
    B = 2 * P;
    NB = p.mode == 1 ? P : B;
    G = p.generations;
    if (p.schedule == 1) {
      R = p.repetitions;
    } else {
      R = p.iters_per_gen / p.sw_period;
      last = p.iters_per_gen - (R - 1) * p.sw_period;
    }
    NBT = K * NB;
    mgroup = K > 1 ? B : 0;
    s16 = pr[0]->s16;
    s = stream;
    fp16 = p.precision == 1;
    L = make_layout(n, p, K);
    SPRING_TRY(prepare_fft_kernels(n));
    SPRING_TRY(ensure_tuned(n, B, s));
    DeviceTables tb;
    SPRING_TRY(device_tables(&tb));
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&mem), L.total, s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      mem = nullptr;
      set_error(std::string("run allocation of ") + std::to_string(L.total) + " bytes failed");
      return SPRING_E_NOMEM;
    }
    x = reinterpret_cast<float2*>(mem + L.x);
    w = reinterpret_cast<float2*>(mem + L.w);
    S = reinterpret_cast<uint8_t*>(mem + L.S);
    Sb = reinterpret_cast<uint32_t*>(mem + L.Sb);
    sm0 = reinterpret_cast<float*>(mem + L.sm0);
    sm1 = reinterpret_cast<float*>(mem + L.sm1);
    err = reinterpret_cast<double*>(mem + L.err);
    abc = reinterpret_cast<int32_t*>(mem + L.abc);
    ix = reinterpret_cast<int32_t*>(mem + L.ix);
    ir = reinterpret_cast<int32_t*>(mem + L.ir);
    info = reinterpret_cast<int32_t*>(mem + L.info);
    best = reinterpret_cast<int32_t*>(mem + L.best);
    ph = reinterpret_cast<float2*>(mem + L.ph);
    alpha = reinterpret_cast<int64_t*>(mem + L.alpha);
    repl = reinterpret_cast<uint8_t*>(mem + L.repl);
    dens = reinterpret_cast<double*>(mem + L.dens);
    part_err = reinterpret_cast<double*>(mem + L.part_err);
    part_norm = reinterpret_cast<double*>(mem + L.part_norm);
    part_dens = reinterpret_cast<double*>(mem + L.part_dens);
    imgmax = reinterpret_cast<unsigned*>(mem + L.imgmax);
    stats = reinterpret_cast<double*>(mem + L.stats);
    avg = reinterpret_cast<float2*>(mem + L.avg);
    Savg = reinterpret_cast<uint8_t*>(mem + L.Savg);
    err_avg = reinterpret_cast<double*>(mem + L.err_avg);
    status = reinterpret_cast<int*>(mem + L.status);
    peaks = mem + L.peaks;
    init_sc = mem + L.init;
    mavg = p.ca > 0.f ? reinterpret_cast<float*>(mem + L.mavg) : nullptr;
    if (K > 1) {
      float* m = reinterpret_cast<float*>(mem + L.mall);
      for (int q = 0; q < K; ++q)
        SPRING_CUDA(cudaMemcpyAsync(m + q * nn(), probs[q]->M, sizeof(float) * nn(), cudaMemcpyDeviceToDevice, s));
      Mall = m;
    } else {
      Mall = probs[0]->M;
    }
    if (split_supported(n)) {
      Msplit = reinterpret_cast<float*>(mem + L.msplit);
      SPRING_TRY(launch_split_modulus(n, Mall, Msplit, K, s));
    }
    m2 = reinterpret_cast<double*>(mem + L.m2);
    SPRING_TRY(launch_m2_sum(n, Mall, K, m2, s));
    return SPRING_OK;
  }

  size_t nn() const { return (size_t)n * n; }
  void* wh() { return w; }                                                    // B x nn half2
  void* xh() { return reinterpret_cast<char*>(w) + (size_t)B * nn() * 4; }  // B x nn half2

  // bring the FP32 state up to date with the FP16 iteration state
  spring_status sync_x() {
    if (x16_newer) {
      SPRING_TRY(launch_half_to_float(xh(), x, (long long)NBT * nn(), s16, s));
      x16_newer = false;
    }
    return SPRING_OK;
  }
  // pattern cq of the batch
  float2* x_pop() { return x + (size_t)cq * B * nn(); }
  float2* x_new() { return x_pop() + P * nn(); }
  float2* w_pop() { return w + (size_t)cq * B * nn(); }
  float2* w_new() { return w_pop() + P * nn(); }
  uint8_t* S_pop() { return S + (size_t)cq * B * nn(); }
  uint8_t* S_new() { return S_pop() + P * nn(); }
  double* err_pop() { return err + (size_t)cq * B; }
  double* err_new() { return err_pop() + P; }
  int32_t* bestq() { return best + 4 * cq; }
  int64_t* alphaq() { return alpha + 4 * cq; }
  double* statsq() { return stats + (size_t)SPRING_GEN_STATS_COLS * G * cq; }
  float2* avgq() { return avg + (size_t)cq * nn(); }
  uint8_t* Savgq() { return Savg + (size_t)cq * nn(); }
  double* err_avgq() { return err_avg + 2 * cq; }
  const float* Mq() { return Mall + (K > 1 ? (size_t)cq * nn() : 0); }
  const uint8_t* S0q() { return probs[cq]->S0; }
  uint64_t seed() const { return seeds[cq]; }

  // Initialize (App. "Initialization of the starting densities")
  spring_status enqueue_init() {
    const Phase range("spring:initialize");
    SPRING_CUDA(cudaMemsetAsync(status, 0, sizeof(int) * 4, s));
    for (cq = 0; cq < K; ++cq) {
      SPRING_TRY(launch_init_spheres(n, seed(), S0q(), P, prm.init_n_spheres, prm.init_gamma,
                                     prm.init_phi_max, x_pop(), init_sc, s));
      SPRING_TRY(fft2_unitary(n, -1, x_pop(), w_pop(), nullptr, P, s));
      SPRING_TRY(launch_normalise(n, w_pop(), Mq(), P, x_pop(), part_norm, s));
      SPRING_TRY(launch_broadcast_support(n, S0q(), P, S_pop(), s));
    }
    cq = 0;
    z_valid = z16_valid = x16_newer = false;
    return SPRING_OK;
  }

  // alignment of P pairs (ix, ir) given population spectra in w_pop; correlations go to
  // the free new-population halves of x and w
  spring_status align(const int32_t* pix, const int32_t* pir, int32_t* pinfo, float2* pph) {
    SPRING_TRY(launch_xcorr_spectra(n, w_pop(), pix, pir, P, Mq(), x_new(), w_new(), s));
    SPRING_TRY(fft2_unitary(n, +1, x_new(), x_new(), nullptr, P, s));
    SPRING_TRY(fft2_unitary(n, +1, w_new(), w_new(), nullptr, P, s));
    return launch_peaks(n, x_new(), w_new(), P, pinfo, pph, peaks, s);
  }

  // Crossover averaging (App. "Crossover averaging"): the parents' average moduli
  // (|F rho_avg| + mean_p |F rho_p|) / 2 into mavg, with rho_avg the population aligned onto
  // its best individual (Eq. avgrec).  Needs the population spectra in w_pop.
  spring_status average_moduli(int g) {
    SPRING_TRY(launch_argmin(g == 1 ? nullptr : err_pop(), P, bestq(), s));
    SPRING_TRY(launch_pairs_onto_best(P, bestq(), ix, ir, s));
    SPRING_TRY(align(ix, ir, info, ph));
    SPRING_TRY(launch_average(n, x_pop(), S_pop(), info, ph, bestq(), P, avgq(), Savgq(), s));
    SPRING_TRY(fft2_unitary(n, -1, avgq(), avgq(), nullptr, 1, s));
    return launch_average_moduli(n, w_pop(), avgq(), P, mavg, s);
  }

  // Crossover (Alg. crossover)
  spring_status crossover(int g) {
    const Phase range("spring:crossover");
    SPRING_TRY(fft2_unitary(n, -1, x_pop(), w_pop(), nullptr, P, s));
    if (prm.ca > 0.f) SPRING_TRY(average_moduli(g));
    SPRING_TRY(launch_random_choice(seed(), g, P, abc, s));
    SPRING_TRY(launch_pairs_crossover(P, abc, ix, ir, s));
    for (int c = 0; c < 3; ++c) SPRING_TRY(align(ix + c * P, ir + c * P, info + 3 * c * P, ph + c * P));
    SPRING_TRY(launch_crossover_mix(n, w_pop(), abc, info, ph, P, seed(), g, prm.cw, prm.cp,
                                    prm.tile_min, prm.tile_max, prm.ca, mavg, x_new(), s));
    SPRING_TRY(fft2_unitary(n, +1, x_new(), x_new(), nullptr, P, s));
    SPRING_TRY(launch_crossover_support(n, S_pop(), abc, info, P, S_new(), s));
    z_valid = z16_valid = false;
    return SPRING_OK;
  }

  spring_status iterations(int alg, int k) {
    if (k <= 0) return SPRING_OK;
    const int path = iteration_path(n);  // one path for the whole block
    if (fp16 || path != 1)  // the row passes read the supports as bits
      SPRING_TRY(launch_pack_support(S, Sb, (long long)NBT * nn(), s));
    if (fp16) {
      if (!z16_valid) {
        SPRING_TRY(launch_row_init16(n, x, xh(), wh(), NB, s16, s));
        z16_valid = true;
      }
      for (int it = 0; it < k; ++it) {
        SPRING_TRY(launch_col_pm16(n, wh(), Mall, NB, s16, s));
        SPRING_TRY(launch_row_iter16(n, alg, wh(), xh(), Sb, NB, prm.beta, prm.chi, s16, s));
      }
      x16_newer = true;
      return SPRING_OK;
    }
    if (path == 1) {  // on chip: x in, x out; w is left stale
      SPRING_TRY(launch_cluster_iter(n, alg, x, S, Mall, NBT, prm.beta, prm.chi, k, s, mgroup));
      z_valid = false;
      return SPRING_OK;
    }
    if (path == 2) {  // split passes: w holds the chunked spectra
      if (!z_valid || z_path != 2) {
        SPRING_TRY(launch_row_split(n, 0, true, w, x, nullptr, NBT, prm.beta, prm.chi, s));
        z_valid = true;
        z_path = 2;
      }
      return iterate_split(n, alg, w, x, Sb, Msplit, NBT, mgroup, prm.beta, prm.chi, k, s);
    }
    if (!z_valid || z_path != 0) {
      SPRING_TRY(launch_row_fft(n, -1, x, w, nullptr, NBT, 1.0f, s));
      z_valid = true;
      z_path = 0;
    }
    for (int it = 0; it < k; ++it) {
      SPRING_TRY(launch_col_pm(n, w, Mall, NBT, s, mgroup));
      SPRING_TRY(launch_row_iter(n, alg, w, x, Sb, NBT, prm.beta, prm.chi, true, s));
    }
    return SPRING_OK;
  }

  spring_status shrinkwrap(float sigma, float tau) {
    const Phase range("spring:update_support");
    SPRING_TRY(sync_x());
    SPRING_TRY(launch_smooth(n, x, sm0, sm1, NBT, sigma, imgmax, s));
    return launch_threshold(n, sm1, imgmax, tau, S, NBT, s);
  }

  // area k of the statistics (0: alpha_best, 2: alpha_eval), each pattern's own
  spring_status shrinkwrap_area(float sigma, int k) {
    const Phase range("spring:update_support_size");
    SPRING_TRY(sync_x());
    SPRING_TRY(launch_smooth(n, x, sm0, sm1, NBT, sigma, nullptr, s));
    return launch_select_area(n, sm1, alpha + k, 4, S, NBT, s, NB, sm0);  // sm0 is free after the smoothing
  }

  spring_status errors() {
    const Phase range("spring:get_error");
    SPRING_TRY(sync_x());
    SPRING_TRY(launch_row_fft(n, -1, x, w, S, NBT, 1.0f, s));
    SPRING_TRY(launch_col_err(n, w, Mall, NBT, part_err, s, mgroup, true));
    SPRING_TRY(launch_err_finalize(n, part_err, NBT, err, status, s, m2, mgroup));
    z_valid = z16_valid = false;  // w served as scratch
    return SPRING_OK;
  }

  // Sequence lengths of generation g for schedule 1 (App. "Changing values over
  // generations"): IA count linear from seq_ia to 0, ER count from seq_er to
  // seq_ia + seq_er, each rounded to the nearest integer with halves up (exact integers)
  void sequence_counts(int g, int* ia, int* er) const {
    if (G <= 1) {
      *ia = prm.seq_ia;
      *er = prm.seq_er;
      return;
    }
    const long long den = 2LL * (G - 1);
    *ia = (int)((2LL * prm.seq_ia * (G - g) + (G - 1)) / den);
    *er = prm.seq_er + (int)((2LL * prm.seq_ia * (g - 1) + (G - 1)) / den);
  }

  // Sequence (Eq. sequence): ia iterations of the IA, then er of ER
  spring_status sequence(int ia, int er) {
    SPRING_TRY(iterations(prm.algorithm, ia));
    return iterations(0, er);
  }

  // Improve (Alg. improve) of both populations with the paper's Sequence
  spring_status improve_paper(int g, float sigma, float tau) {
    const Phase range("spring:improve");
    int ia = 0, er = 0;
    sequence_counts(g, &ia, &er);
    for (int r = 1; r <= R - 2; ++r) {
      SPRING_TRY(sequence(ia, er));
      SPRING_TRY(shrinkwrap(sigma, tau));
    }
    SPRING_TRY(sequence(ia, er));
    SPRING_TRY(shrinkwrap_area(sigma, 0));  // UpdateSupportSize(alpha_best)
    SPRING_TRY(sequence(ia, er));
    SPRING_TRY(shrinkwrap_area(sigma, 2));  // UpdateSupportSize(alpha_eval)
    SPRING_TRY(iterations(0, prm.seq_eval));        // EvalSequence: ER
    SPRING_TRY(errors());                           // GetError
    SPRING_TRY(shrinkwrap(sigma, tau));
    return sync_x();
  }

  // Improve of independent reconstructions (Alg. normalimprove): one Sequence and one
  // UpdateSupport per generation (schedule 0: blocks of sw_period, each followed by
  // UpdateSupport, the last er_tail iterations ER); the error is taken before the last
  // UpdateSupport
  spring_status improve_independent(int g, float sigma, float tau) {
    const Phase range("spring:improve");
    if (prm.schedule == 1) {
      int ia = 0, er = 0;
      sequence_counts(g, &ia, &er);
      SPRING_TRY(sequence(ia, er));
    } else {
      for (int blk = 1; blk < R; ++blk) {
        SPRING_TRY(iterations(prm.algorithm, prm.sw_period));
        SPRING_TRY(shrinkwrap(sigma, tau));
      }
      SPRING_TRY(sequence(last - prm.er_tail, prm.er_tail));
    }
    SPRING_TRY(errors());
    SPRING_TRY(shrinkwrap(sigma, tau));
    return sync_x();
  }

  // Improve (Alg. improve) of both populations at once
  spring_status improve(float sigma, float tau) {
    const Phase range("spring:improve");
    const int K = prm.sw_period, alg = prm.algorithm;
    for (int blk = 1; blk <= R; ++blk) {
      if (blk < R) SPRING_TRY(iterations(alg, K));
      if (blk <= R - 2) {
        SPRING_TRY(shrinkwrap(sigma, tau));
      } else if (blk == R - 1) {
        SPRING_TRY(shrinkwrap_area(sigma, 0));  // UpdateSupportSize(alpha_best)
      } else {
        SPRING_TRY(iterations(alg, last - prm.er_tail));
        SPRING_TRY(shrinkwrap_area(sigma, 2));  // UpdateSupportSize(alpha_eval)
        SPRING_TRY(iterations(0, prm.er_tail));         // EvalSequence: ER
        SPRING_TRY(errors());                           // GetError
        SPRING_TRY(shrinkwrap(sigma, tau));
      }
    }
    return sync_x();
  }

  spring_status generation(int g) {
    const Phase range("spring:generation");
    const double t = G > 1 ? (double)(g - 1) / (double)(G - 1) : 0.0;
    const float sigma = (float)(prm.sw_sigma + (prm.sw_sigma_end - prm.sw_sigma) * t);
    const float tau = (float)(prm.sw_threshold + (prm.sw_threshold_end - prm.sw_threshold) * t);
    if (prm.mode == 1) {  // independent reconstructions (Alg. randomsearch)
      SPRING_TRY(improve_independent(g, sigma, tau));
      if (tr_err) SPRING_CUDA(cudaMemcpyAsync(tr_err, err_pop(), sizeof(double) * P, cudaMemcpyDeviceToDevice, s));
      SPRING_CUDA(cudaMemsetAsync(repl, 0, P, s));
      SPRING_TRY(launch_density_sums(n, x_pop(), P, part_dens, dens, s));
      SPRING_TRY(launch_gen_stats(n, err_pop(), S_pop(), repl, dens, P, statsq() + SPRING_GEN_STATS_COLS * (g - 1), s));
      return monitor(g);
    }
    // the GA steps pattern by pattern, the improvement of all K patterns' populations at once
    for (cq = 0; cq < K; ++cq) {
      SPRING_TRY(crossover(g));
      SPRING_TRY(launch_argmin(g == 1 ? nullptr : err_pop(), P, bestq(), s));
      SPRING_TRY(launch_area_stats(n, S_pop(), bestq(), P, g, G, alphaq(), s));
      if (tr_best) SPRING_CUDA(cudaMemcpyAsync(tr_best, bestq(), sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    }
    cq = 0;
    if (prm.schedule == 1)
      SPRING_TRY(improve_paper(g, sigma, tau));
    else
      SPRING_TRY(improve(sigma, tau));
    for (cq = 0; cq < K; ++cq) {
      if (tr_err) SPRING_CUDA(cudaMemcpyAsync(tr_err, err_pop(), sizeof(double) * P, cudaMemcpyDeviceToDevice, s));
      SPRING_TRY(launch_select(n, x_pop(), S_pop(), err_pop(), x_new(), S_new(), err_new(), P, repl, s));
      SPRING_TRY(launch_density_sums(n, x_pop(), P, part_dens, dens, s));
      SPRING_TRY(launch_gen_stats(n, err_pop(), S_pop(), repl, dens, P, statsq() + SPRING_GEN_STATS_COLS * (g - 1), s));
      SPRING_TRY(monitor(g));
    }
    cq = 0;
    return SPRING_OK;
  }

  // the average reconstruction's error every generation (gen_stats column 3)
  spring_status monitor(int g) {
    if (!prm.monitor_avg || g == G) return SPRING_OK;  // generation G: finish() computes it
    SPRING_TRY(average_and_error());
    SPRING_CUDA(cudaMemcpyAsync(statsq() + SPRING_GEN_STATS_COLS * (g - 1) + 3, err_avgq(), sizeof(double),
                                cudaMemcpyDeviceToDevice, s));
    return SPRING_OK;
  }

  // Average (Eq. avgrec) of each pattern's final population and its error
  spring_status finish() {
    const Phase range("spring:average");
    for (cq = 0; cq < K; ++cq) SPRING_TRY(average_and_error());
    cq = 0;
    return SPRING_OK;
  }

  spring_status average_and_error() {
    SPRING_TRY(fft2_unitary(n, -1, x_pop(), w_pop(), nullptr, P, s));
    SPRING_TRY(launch_argmin(err_pop(), P, bestq(), s));
    SPRING_TRY(launch_pairs_onto_best(P, bestq(), ix, ir, s));
    SPRING_TRY(align(ix, ir, info, ph));
    SPRING_TRY(launch_average(n, x_pop(), S_pop(), info, ph, bestq(), P, avgq(), Savgq(), s));
    SPRING_TRY(launch_row_fft(n, -1, avgq(), w_new(), Savgq(), 1, 1.0f, s));
    SPRING_TRY(launch_col_err(n, w_new(), Mq(), 1, part_err, s, 0, true));
    SPRING_TRY(launch_err_finalize(n, part_err, 1, err_avgq(), status, s, m2 + (K > 1 ? cq : 0)));
    return SPRING_OK;
  }

  // checkpoint: the population after generation g0 (host buffers), uploaded before any
  // other work of the run; the run continues at generation g0 + 1
  spring_status upload_population(const spring_population& from) {
    SPRING_CUDA(cudaMemsetAsync(status, 0, sizeof(int) * 4, s));
    SPRING_CUDA(cudaMemcpyAsync(x_pop(), from.pop_x, sizeof(float2) * P * nn(), cudaMemcpyHostToDevice, s));
    SPRING_CUDA(cudaMemcpyAsync(S_pop(), from.pop_S, (size_t)P * nn(), cudaMemcpyHostToDevice, s));
    SPRING_CUDA(cudaMemcpyAsync(err_pop(), from.pop_err, sizeof(double) * P, cudaMemcpyHostToDevice, s));
    SPRING_CUDA(cudaStreamSynchronize(s));
    next_gen = from.generation + 1;
    first_gen = next_gen;
    resumed = true;
    z_valid = z16_valid = x16_newer = false;
    return SPRING_OK;
  }

  // after the stream has completed: the population to host buffers
  spring_status download_population(spring_population* to) {
    SPRING_CUDA(cudaMemcpy(to->pop_x, x_pop(), sizeof(float2) * P * nn(), cudaMemcpyDeviceToHost));
    SPRING_CUDA(cudaMemcpy(to->pop_S, S_pop(), (size_t)P * nn(), cudaMemcpyDeviceToHost));
    SPRING_CUDA(cudaMemcpy(to->pop_err, err_pop(), sizeof(double) * P, cudaMemcpyDeviceToHost));
    to->generation = next_gen - 1 < G ? next_gen - 1 : G;  // next_gen passes G + 1 once the average ran
    return SPRING_OK;
  }

  // after the stream has completed: what generation g decided (spring_mpr_step)
  spring_status download_trace(int g, spring_generation_trace* tr) {
    SPRING_CUDA(cudaMemcpy(tr->gen_stats, statsq() + SPRING_GEN_STATS_COLS * (g - 1),
                           sizeof(double) * SPRING_GEN_STATS_COLS, cudaMemcpyDeviceToHost));
    if (tr->err_parents) SPRING_CUDA(cudaMemcpy(tr->err_parents, tr_err, sizeof(double) * P, cudaMemcpyDeviceToHost));
    if (prm.mode == 1) return SPRING_OK;
    if (tr->err_new) SPRING_CUDA(cudaMemcpy(tr->err_new, err_new(), sizeof(double) * P, cudaMemcpyDeviceToHost));
    if (tr->replaced) SPRING_CUDA(cudaMemcpy(tr->replaced, repl, P, cudaMemcpyDeviceToHost));
    if (tr->parents) SPRING_CUDA(cudaMemcpy(tr->parents, abc, sizeof(int32_t) * 3 * P, cudaMemcpyDeviceToHost));
    SPRING_CUDA(cudaMemcpy(tr->areas, alphaq(), sizeof(int64_t) * 3, cudaMemcpyDeviceToHost));
    SPRING_CUDA(cudaMemcpy(&tr->best, tr_best, sizeof(int32_t), cudaMemcpyDeviceToHost));
    return SPRING_OK;
  }

  // enqueue the next chunk of work: init with generation 1, then one generation per call,
  // then the average; returns true when nothing is left
  spring_status step(bool* done) {
    *done = false;
    if (next_gen == 1 && !resumed) SPRING_TRY(enqueue_init());
    if (stop_after > 0 && next_gen > stop_after) {
      *done = true;
      return SPRING_OK;
    }
    if (next_gen <= G) {
      SPRING_TRY(generation(next_gen));
      ++next_gen;
      if (next_gen <= G) return SPRING_OK;
    }
    if (next_gen == G + 1) {
      SPRING_TRY(finish());
      ++next_gen;
      return SPRING_OK;
    }
    *done = true;
    return SPRING_OK;
  }

  spring_status enqueue_all() {
    bool done = false;
    while (!done) SPRING_TRY(step(&done));
    return SPRING_OK;
  }

  // after the stream has completed: copy results to host buffers (K of them for a batch)
  spring_status collect(spring_result* outs) {
    int st[4] = {0, 0, 0, 0};
    SPRING_CUDA(cudaMemcpy(st, status, sizeof(st), cudaMemcpyDeviceToHost));
    for (cq = 0; cq < K; ++cq) {
      spring_result* out = outs + cq;
      int32_t b = 0;
      double ea = 0.0, eb = 0.0;
      SPRING_CUDA(cudaMemcpy(&b, bestq(), sizeof(b), cudaMemcpyDeviceToHost));
      SPRING_CUDA(cudaMemcpy(&ea, err_avgq(), sizeof(ea), cudaMemcpyDeviceToHost));
      SPRING_CUDA(cudaMemcpy(&eb, err_pop() + b, sizeof(eb), cudaMemcpyDeviceToHost));
      out->final_error_avg = ea;
      out->final_error_best = eb;
      if (out->rho_avg) SPRING_CUDA(cudaMemcpy(out->rho_avg, avgq(), sizeof(float2) * nn(), cudaMemcpyDeviceToHost));
      if (out->rho_best)
        SPRING_CUDA(cudaMemcpy(out->rho_best, x_pop() + (size_t)b * nn(), sizeof(float2) * nn(), cudaMemcpyDeviceToHost));
      if (out->support_avg) SPRING_CUDA(cudaMemcpy(out->support_avg, Savgq(), nn(), cudaMemcpyDeviceToHost));
      if (out->gen_stats) {
        SPRING_CUDA(cudaMemcpy(out->gen_stats, statsq(), sizeof(double) * SPRING_GEN_STATS_COLS * G,
                               cudaMemcpyDeviceToHost));
        out->gen_stats[SPRING_GEN_STATS_COLS * (G - 1) + 3] = ea;
        for (int g = 1; g < first_gen; ++g)  // generations run before a resume
          for (int k = 0; k < SPRING_GEN_STATS_COLS; ++k)
            out->gen_stats[SPRING_GEN_STATS_COLS * (g - 1) + k] = std::numeric_limits<double>::quiet_NaN();
      }
    }
    cq = 0;
    if (st[0]) {
      set_error("non-finite Fourier error in the run");
      return SPRING_E_NUMERIC;
    }
    return SPRING_OK;
  }
};

}  // namespace spring

// ------------------------------------------------------------------ context and serving
namespace {

enum TState { T_QUEUED = 0, T_RUNNING = 1, T_DONE = 2, T_FAILED = 3, T_CANCELLED = 4 };

struct Ticket {
  uint64_t id = 0;
  spring_problem* prob = nullptr;
  spring_params prm{};
  TState state = T_QUEUED;
  bool cancel = false;
  size_t footprint = 0;       // of the request alone (the admission check at submission)
  struct Cohort* cohort = nullptr;  // while admitted: the requests it advances with
  spring_status status = SPRING_OK;
  std::string message;
  // host staging of the results
  std::vector<float> rho_avg, rho_best;
  std::vector<uint8_t> support_avg;
  std::vector<double> gen_stats;
  double e_avg = 0.0, e_best = 0.0;
  double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
};

// Requests that advance together: one Run over K problems of the same side and the same
// parameters (seeds aside), whose launches cover all K populations (K = 1: one request).
// Each member's result equals its run alone bit for bit (see spring_mpr_run_batch).
struct Cohort {
  std::unique_ptr<Run> run;
  std::vector<Ticket*> members;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  bool ev_pending = false;
  size_t footprint = 0;
};

}  // namespace

struct spring_ctx {
  int device = 0;
  size_t budget = 0;
  size_t used = 0;
  int max_active = 4;             // cohorts advancing concurrently (SPRING_MAX_ACTIVE)
  int max_cohort = 32;            // requests per cohort (SPRING_MAX_COHORT; 1 = no batching)
  double cohort_pixels = 67108864.0;  // a cohort's pixels per launch at most (2P N^2 per member)
  std::list<std::unique_ptr<Cohort>> cohorts;
  uint64_t n_cohorts = 0, n_admitted = 0;  // statistics: cohorts formed, requests admitted
  int prio_lo = 0, prio_hi = 0;   // stream priority range of the device
  std::mutex mu;
  std::condition_variable cv;       // scheduler wake-ups
  std::condition_variable done_cv;  // ticket completions
  std::deque<uint64_t> queue;
  std::map<uint64_t, std::unique_ptr<Ticket>> tickets;
  uint64_t next_id = 1;
  bool stop = false;
  std::thread worker;
};

namespace spring {

static bool reserve(spring_ctx* c, size_t bytes) {
  if (c->used + bytes > c->budget) return false;
  c->used += bytes;
  return true;
}

// a member leaves: its state, time and the reference to its problem (resources stay with
// its cohort)
static void finish_member(spring_ctx* c, Ticket* t, TState st) {
  t->state = st;
  t->t_done = now_s();
  t->cohort = nullptr;
  t->prob->refs.fetch_sub(1);
  c->done_cv.notify_all();
}

static void release_cohort(spring_ctx* c, Cohort* k) {
  if (k->run) {
    k->run->release();
    k->run.reset();
  }
  if (k->stream) {
    cudaStreamSynchronize(k->stream);
    cudaStreamDestroy(k->stream);
    k->stream = nullptr;
  }
  if (k->ev) {
    cudaEventDestroy(k->ev);
    k->ev = nullptr;
  }
  c->used -= k->footprint;
  k->footprint = 0;
}

// every member of k fails with status st (k's resources are released by the caller)
static void fail_cohort(spring_ctx* c, Cohort* k, spring_status st, const std::string& msg) {
  for (Ticket* t : k->members)
    if (t->cohort == k) {
      t->status = st;
      t->message = msg;
      finish_member(c, t, T_FAILED);
    }
}

// requests that may share a cohort: same side, same parameters apart from the seed, and a
// form that batched runs support (FP32 storage, MPR mode)
static bool cohort_key_equal(const Ticket* a, const Ticket* b) {
  if (a->prob->n != b->prob->n) return false;
  spring_params pa = a->prm, pb = b->prm;
  pa.seed = pb.seed = 0;
  pa.use_graph = pb.use_graph = 0;
  return std::memcmp(&pa, &pb, sizeof(pa)) == 0;
}
static bool batchable(const Ticket* t) { return t->prm.precision == 0 && t->prm.mode == 0; }

// the cohort that starts with the queue's head: the head, then queued requests with the same
// key in arrival order, while the batch stays within max_cohort and cohort_pixels and its
// footprint fits the budget (reserved here).  Returns the members' queue positions, empty
// if the head does not fit.
static std::vector<size_t> form_cohort(spring_ctx* c, size_t* footprint) {
  Ticket* head = c->tickets[c->queue.front()].get();
  std::vector<size_t> pos{0};
  if (batchable(head)) {
    const double px = 2.0 * head->prm.pop * (double)head->prob->n * head->prob->n;
    const size_t kmax = (size_t)std::max(1.0, std::min((double)c->max_cohort, c->cohort_pixels / px));
    for (size_t i = 1; i < c->queue.size() && pos.size() < kmax; ++i) {
      Ticket* u = c->tickets[c->queue[i]].get();
      if (!u->cancel && cohort_key_equal(head, u)) pos.push_back(i);
    }
  }
  while (!pos.empty()) {
    const size_t fp = make_layout(head->prob->n, head->prm, (int)pos.size()).total;
    if (reserve(c, fp)) {
      *footprint = fp;
      return pos;
    }
    pos.pop_back();
  }
  return pos;
}

// scheduler: admit queued requests in arrival order while their footprint fits, grouping
// each admitted request with queued ones of the same side and parameters into a cohort
// (one set of launches over all their populations); then keep every cohort's stream fed
// with one generation at a time.  Requests arriving while others run are admitted as
// memory frees up, and the cohorts' kernels overlap on the device through separate
// streams (continuous batching).
static void scheduler(spring_ctx* c) {
  cudaSetDevice(c->device);
  std::unique_lock<std::mutex> lk(c->mu);
  while (!c->stop) {
    bool progress = false;
    // admission in arrival order, while memory and the concurrency cap allow
    while (!c->queue.empty()) {
      Ticket* t = c->tickets[c->queue.front()].get();
      if (t->cancel) {
        c->queue.pop_front();
        t->state = T_CANCELLED;
        t->t_done = now_s();
        t->prob->refs.fetch_sub(1);
        progress = true;
        c->done_cv.notify_all();
        continue;
      }
      if ((int)c->cohorts.size() >= c->max_active) break;
      size_t fp = 0;
      std::vector<size_t> pos = form_cohort(c, &fp);
      if (pos.empty()) break;
      std::unique_ptr<Cohort> k(new Cohort());
      k->footprint = fp;
      for (size_t i : pos) k->members.push_back(c->tickets[c->queue[i]].get());
      for (size_t j = pos.size(); j-- > 0;) c->queue.erase(c->queue.begin() + (long)pos[j]);
      const double t_admit = now_s();
      std::vector<const spring_problem*> probs;
      std::vector<uint64_t> seeds;
      for (Ticket* m : k->members) {
        m->t_admit = t_admit;
        m->state = T_RUNNING;
        m->cohort = k.get();
        probs.push_back(m->prob);
        seeds.push_back(m->prm.seed);
      }
      ++c->n_cohorts;
      c->n_admitted += k->members.size();
      // smaller requests get higher stream priority: short jobs do not queue behind long ones
      const size_t each = t->footprint;
      const int prio = each < (64u << 20) ? c->prio_hi
                       : each < (512u << 20) ? (c->prio_hi + c->prio_lo) / 2 : c->prio_lo;
      cudaStreamCreateWithPriority(&k->stream, cudaStreamNonBlocking, prio);
      cudaEventCreateWithFlags(&k->ev, cudaEventDisableTiming);
      k->run.reset(new Run());
      spring_status st = k->run->setup_batch(probs.data(), (int)probs.size(), seeds.data(), t->prm, k->stream);
      if (st != SPRING_OK) {
        fail_cohort(c, k.get(), st, spring_last_error());
        release_cohort(c, k.get());
      } else {
        c->cohorts.push_back(std::move(k));
      }
      progress = true;
    }
    // feed running cohorts
    for (auto it = c->cohorts.begin(); it != c->cohorts.end();) {
      Cohort* k = it->get();
      bool retire = false;
      if (k->ev_pending) {
        cudaError_t q = cudaEventQuery(k->ev);
        if (q == cudaErrorNotReady) {
          ++it;
          continue;
        }
        k->ev_pending = false;
        if (q != cudaSuccess) {
          fail_cohort(c, k, SPRING_E_CUDA, cudaGetErrorString(q));
          retire = true;
        }
      }
      if (!retire) {
        bool all_cancelled = true;
        for (Ticket* m : k->members) all_cancelled = all_cancelled && m->cancel;
        if (all_cancelled) {
          for (Ticket* m : k->members) finish_member(c, m, T_CANCELLED);
          retire = true;
        }
      }
      if (!retire) {
        bool done = false;
        spring_status st = k->run->step(&done);
        if (st != SPRING_OK) {
          fail_cohort(c, k, st, spring_last_error());
          retire = true;
        } else if (done) {
          const int n = k->run->n, G = k->run->G, K = (int)k->members.size();
          const size_t nn = (size_t)n * n;
          std::vector<spring_result> rs(K);
          for (int q = 0; q < K; ++q) {
            Ticket* m = k->members[q];
            m->rho_avg.resize(2 * nn);
            m->rho_best.resize(2 * nn);
            m->support_avg.resize(nn);
            m->gen_stats.resize(SPRING_GEN_STATS_COLS * (size_t)G);
            rs[q] = spring_result{};
            rs[q].rho_avg = m->rho_avg.data();
            rs[q].rho_best = m->rho_best.data();
            rs[q].support_avg = m->support_avg.data();
            rs[q].gen_stats = m->gen_stats.data();
          }
          st = check_device_waits();  // a bounded device-side wait that gave up
          if (st == SPRING_OK) st = k->run->collect(rs.data());
          const std::string msg = st == SPRING_OK ? std::string() : std::string(spring_last_error());
          for (int q = 0; q < K; ++q) {
            Ticket* m = k->members[q];
            m->e_avg = rs[q].final_error_avg;
            m->e_best = rs[q].final_error_best;
            if (m->cancel) {
              finish_member(c, m, T_CANCELLED);
            } else if (st != SPRING_OK) {
              m->status = st;
              m->message = msg;
              finish_member(c, m, T_FAILED);
            } else {
              finish_member(c, m, T_DONE);
            }
          }
          retire = true;
        } else {
          cudaEventRecord(k->ev, k->stream);
          k->ev_pending = true;
        }
      }
      progress = true;
      if (retire) {
        release_cohort(c, k);
        it = c->cohorts.erase(it);
      } else {
        ++it;
      }
    }
    if (!progress) c->cv.wait_for(lk, std::chrono::microseconds(200));
  }
}

}  // namespace spring

extern "C" {

void spring_params_default(spring_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->pop = 8;
  p->iters_per_gen = 100;
  p->generations = 5;
  p->algorithm = 2;
  p->beta = 0.9f;
  p->sw_sigma = 1.5f;
  p->sw_threshold = 0.2f;
  p->sw_sigma_end = 1.5f;
  p->sw_threshold_end = 0.2f;
  p->sw_period = 20;
  p->er_tail = 10;
  p->chi = 0.5f;
  p->cw = 0.4f;
  p->cp = 0.6f;
  p->tile_min = 4;
  p->tile_max = 0;
  p->init_n_spheres = 5;
  p->init_gamma = 1.0f;
  p->init_phi_max = 0.0f;
  p->precision = 0;
  p->use_graph = 0;
  p->schedule = 0;
  p->mode = 0;
  p->seq_ia = 40;
  p->seq_er = 40;
  p->seq_eval = 40;
  p->repetitions = 3;
  p->ca = 0.0f;
  p->monitor_avg = 0;
  p->seed = 0;
}

size_t spring_footprint_bytes(int n, const spring_params* p) {
  if (!p || !valid_n(n) || p->pop < 1 || p->generations < 1) return 0;
  return make_layout(n, *p).total;
}

spring_status spring_init(int device, size_t hbm_budget_bytes, spring_ctx** out) {
  if (!out) return invalid("null output handle");
  int count = 0;
  SPRING_CUDA(cudaGetDeviceCount(&count));
  if (device < 0 || device >= count) return invalid("no such CUDA device");
  SPRING_CUDA(cudaSetDevice(device));
  size_t fr = 0, tot = 0;
  SPRING_CUDA(cudaMemGetInfo(&fr, &tot));
  // keep freed run memory in the device pool for reuse by the next run
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  DeviceTables tb;
  SPRING_TRY(device_tables(&tb));
  spring_ctx* c = new spring_ctx();
  c->device = device;
  c->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.9 * (double)fr);
  if (const char* e = std::getenv("SPRING_MAX_ACTIVE")) {
    const int v = std::atoi(e);
    if (v > 0) c->max_active = v;
  }
  if (const char* e = std::getenv("SPRING_MAX_COHORT")) {
    const int v = std::atoi(e);
    if (v > 0) c->max_cohort = v;
  }
  cudaDeviceGetStreamPriorityRange(&c->prio_lo, &c->prio_hi);
  c->worker = std::thread(scheduler, c);
  *out = c;
  return SPRING_OK;
}

spring_status spring_shutdown(spring_ctx* c) {
  if (!c) return invalid("null context");
  {
    std::lock_guard<std::mutex> lk(c->mu);
    for (auto& kv : c->tickets)
      if (kv.second->state == T_QUEUED || kv.second->state == T_RUNNING) {
        set_error("context has queued or running tickets");
        return SPRING_E_BUSY;
      }
    c->stop = true;
  }
  c->cv.notify_all();
  if (c->worker.joinable()) c->worker.join();
  delete c;
  return SPRING_OK;
}

static spring_status problem_alloc(spring_ctx* ctx, int n, spring_problem** out, spring_problem** p) {
  if (!ctx || !out) return invalid("null context or output handle");
  if (!valid_n(n)) return invalid("unsupported pattern side " + std::to_string(n));
  SPRING_CUDA(cudaSetDevice(ctx->device));
  std::unique_ptr<spring_problem> pr(new spring_problem());
  pr->ctx = ctx;
  pr->n = n;
  const size_t nn = (size_t)n * n;
  SPRING_CUDA(cudaMalloc(&pr->M, sizeof(float) * (nn + 64)));
  pr->s16 = pr->M + nn;
  cudaError_t e = cudaMalloc(&pr->S0, nn);
  if (e != cudaSuccess) {
    cudaFree(pr->M);
    return cuda_fail(e, "cudaMalloc", __FILE__, __LINE__);
  }
  *p = pr.release();
  return SPRING_OK;
}

static spring_status problem_fill(spring_problem* pr, const float* d_I, const uint8_t* d_mask,
                                  const uint8_t* d_sat, const spring_bounds* b, double* ring_scratch,
                                  const uint8_t* d_S0, cudaStream_t s) {
  const int n = pr->n;
  SPRING_TRY(launch_modulus_encode(n, d_I, d_mask, d_sat, b, ring_scratch, pr->M, s));
  SPRING_TRY(launch_fp16_scale(n, pr->M, pr->s16, s));
  SPRING_CUDA(cudaMemcpyAsync(pr->S0, d_S0, (size_t)n * n, cudaMemcpyDeviceToDevice, s));
  return SPRING_OK;
}

void spring_bounds_default(spring_bounds* b) {
  if (!b) return;
  b->eta = 1.5f;
  b->max_missing = 0.2f;
  b->max_saturated = 0.05f;
}

spring_status spring_problem_create(spring_ctx* ctx, int ny, int nx, const float* I, const uint8_t* mask,
                                    const uint8_t* S0, spring_problem** out) {
  return spring_problem_create_bounded(ctx, ny, nx, I, mask, S0, nullptr, nullptr, out);
}

spring_status spring_problem_create_bounded(spring_ctx* ctx, int ny, int nx, const float* I,
                                            const uint8_t* mask, const uint8_t* S0, const uint8_t* sat,
                                            const spring_bounds* b, spring_problem** out) {
  if (ny != nx) return invalid("patterns must be square");
  if (!I || !mask || !S0) return invalid("null input array");
  if (b && b->eta > 0.f && !(b->max_missing >= 0.f && b->max_saturated >= 0.f && std::isfinite(b->eta)))
    return invalid("bounds: eta must be finite and the fractions >= 0");
  spring_problem* pr = nullptr;
  SPRING_TRY(problem_alloc(ctx, nx, out, &pr));
  const size_t nn = (size_t)nx * nx;
  // device staging: ring scratch (doubles) | I | mask | S0 | saturated
  const size_t ring_bytes = sizeof(double) * (size_t)ring_count(nx);
  char* tmp = nullptr;
  spring_status st = SPRING_OK;
  cudaError_t e = cudaMalloc(&tmp, ring_bytes + nn * (sizeof(float) + 3));
  char* dI = tmp + ring_bytes;
  char* dmask = dI + sizeof(float) * nn;
  char* dS0 = dmask + nn;
  char* dsat = dS0 + nn;
  if (e == cudaSuccess) e = cudaMemcpy(dI, I, sizeof(float) * nn, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dmask, mask, nn, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dS0, S0, nn, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && sat) e = cudaMemcpy(dsat, sat, nn, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    st = cuda_fail(e, "problem upload", __FILE__, __LINE__);
  } else {
    st = problem_fill(pr, reinterpret_cast<float*>(dI), reinterpret_cast<uint8_t*>(dmask),
                      sat ? reinterpret_cast<uint8_t*>(dsat) : nullptr, b, reinterpret_cast<double*>(tmp),
                      reinterpret_cast<uint8_t*>(dS0), nullptr);
    if (st == SPRING_OK) {
      e = cudaStreamSynchronize(nullptr);
      if (e != cudaSuccess) st = cuda_fail(e, "problem set-up", __FILE__, __LINE__);
    }
  }
  if (tmp) cudaFree(tmp);
  if (st != SPRING_OK) {
    cudaFree(pr->M);
    cudaFree(pr->S0);
    delete pr;
    return st;
  }
  *out = pr;
  return SPRING_OK;
}

spring_status spring_problem_create_device(spring_ctx* ctx, int ny, int nx, const float* d_I,
                                           const uint8_t* d_mask, const uint8_t* d_S0, void* stream,
                                           spring_problem** out) {
  if (ny != nx) return invalid("patterns must be square");
  if (!d_I || !d_mask || !d_S0) return invalid("null input array");
  spring_problem* pr = nullptr;
  SPRING_TRY(problem_alloc(ctx, nx, out, &pr));
  spring_status st = problem_fill(pr, d_I, d_mask, nullptr, nullptr, nullptr, d_S0,
                                  reinterpret_cast<cudaStream_t>(stream));
  if (st != SPRING_OK) {
    cudaFree(pr->M);
    cudaFree(pr->S0);
    delete pr;
    return st;
  }
  *out = pr;
  return SPRING_OK;
}

spring_status spring_problem_destroy(spring_problem* pr) {
  if (!pr) return invalid("null problem");
  if (pr->refs.load() > 0) {
    set_error("problem is referenced by an unfinished ticket");
    return SPRING_E_BUSY;
  }
  cudaSetDevice(pr->ctx->device);
  cudaDeviceSynchronize();
  cudaFree(pr->M);
  cudaFree(pr->S0);
  delete pr;
  return SPRING_OK;
}

// A blocking run of K problems of one side (K = 1: a single run; seeds[q] is problem q's
// seed): from Initialize (from = NULL) or from a saved population, up to generation stop
// (0 = all, then the averages into out[0..K)), saving the population if asked.
static spring_status run_blocking_k(spring_problem* const* probs, int K, const uint64_t* seeds,
                                    const spring_params* p, const spring_population* from, int stop,
                                    spring_population* save, spring_result* out,
                                    spring_generation_trace* trace = nullptr) {
  spring_problem* pr = probs[0];
  SPRING_TRY(validate_params(pr->n, *p));
  spring_ctx* c = pr->ctx;
  SPRING_CUDA(cudaSetDevice(c->device));
  const size_t fp = make_layout(pr->n, *p, K).total;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    if (!reserve(c, fp)) {
      set_error("run footprint " + std::to_string(fp) + " B exceeds the context's HBM budget");
      return SPRING_E_NOMEM;
    }
  }
  cudaStream_t s = nullptr;
  spring_status st = SPRING_OK;
  {
    Run run;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaStreamCreate", __FILE__, __LINE__);
    if (st == SPRING_OK) st = run.setup_batch(probs, K, seeds, *p, s);
    if (st == SPRING_OK && from) st = run.upload_population(*from);
    run.stop_after = stop;
    void* trace_mem = nullptr;
    if (st == SPRING_OK && trace) {
      e = cudaMalloc(&trace_mem, sizeof(double) * p->pop + 64);
      if (e != cudaSuccess) st = cuda_fail(e, "cudaMalloc", __FILE__, __LINE__);
      run.tr_err = static_cast<double*>(trace_mem);
      run.tr_best = reinterpret_cast<int32_t*>(static_cast<char*>(trace_mem) + sizeof(double) * p->pop);
    }
    if (st == SPRING_OK) {
      if (p->use_graph) {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) st = cuda_fail(e, "cudaStreamBeginCapture", __FILE__, __LINE__);
        if (st == SPRING_OK) {
          st = run.enqueue_all();
          e = cudaStreamEndCapture(s, &graph);
          if (st == SPRING_OK && e != cudaSuccess) st = cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
        }
        if (st == SPRING_OK) {
          e = cudaGraphInstantiate(&exec, graph, 0);
          if (e != cudaSuccess) st = cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__);
        }
        if (st == SPRING_OK) {
          e = cudaGraphLaunch(exec, s);
          if (e != cudaSuccess) st = cuda_fail(e, "cudaGraphLaunch", __FILE__, __LINE__);
        }
        if (st == SPRING_OK) {
          e = cudaStreamSynchronize(s);
          if (e != cudaSuccess) st = cuda_fail(e, "graph execution", __FILE__, __LINE__);
        }
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
      } else {
        st = run.enqueue_all();
        if (st == SPRING_OK) {
          e = cudaStreamSynchronize(s);
          if (e != cudaSuccess) st = cuda_fail(e, "run execution", __FILE__, __LINE__);
        }
      }
    }
    if (st == SPRING_OK) st = check_device_waits();  // a bounded device-side wait that gave up
    if (st == SPRING_OK && trace) st = run.download_trace(stop, trace);
    if (trace_mem) cudaFree(trace_mem);
    if (st == SPRING_OK && save) st = run.download_population(save);
    if (st == SPRING_OK && out) {
      const double t0 = now_s();
      st = run.collect(out);
      const double t1 = now_s();
      for (int q = 0; q < K; ++q) {
        out[q].t_submit_s = out[q].t_admit_s = t0;
        out[q].t_done_s = t1;
      }
    }
    run.release();
    if (s) {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
  }
  std::lock_guard<std::mutex> lk(c->mu);
  c->used -= fp;
  return st;
}

static spring_status run_blocking(spring_problem* pr, const spring_params* p, const spring_population* from,
                                  int stop, spring_population* save, spring_result* out) {
  return run_blocking_k(&pr, 1, &p->seed, p, from, stop, save, out);
}

spring_status spring_mpr_run(spring_problem* pr, const spring_params* p, spring_result* out) {
  if (!pr || !p || !out) return invalid("null argument");
  return run_blocking(pr, p, nullptr, 0, nullptr, out);
}

// A blocking batch of problems of several sides: one batched Run per side (the side's
// problems share every launch), the sides advancing concurrently on their own streams —
// as parallel branches of one CUDA graph when p->use_graph — so one launch covers all of
// them.  Results go to out[] in the callers' order.
static spring_status run_blocking_mixed(spring_problem* const* probs, int K, const uint64_t* seeds,
                                        const spring_params* p, spring_result* out) {
  std::vector<int> sides;
  std::vector<std::vector<int>> idx;
  for (int q = 0; q < K; ++q) {
    int gi = -1;
    for (size_t g = 0; g < sides.size(); ++g)
      if (sides[g] == probs[q]->n) gi = (int)g;
    if (gi < 0) {
      sides.push_back(probs[q]->n);
      idx.emplace_back();
      gi = (int)sides.size() - 1;
    }
    idx[gi].push_back(q);
  }
  const int NG = (int)sides.size();
  for (int g = 0; g < NG; ++g) SPRING_TRY(validate_params(sides[g], *p));
  spring_ctx* c = probs[0]->ctx;
  SPRING_CUDA(cudaSetDevice(c->device));
  size_t fp = 0;
  for (int g = 0; g < NG; ++g) fp += make_layout(sides[g], *p, (int)idx[g].size()).total;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    if (!reserve(c, fp)) {
      set_error("batch footprint " + std::to_string(fp) + " B exceeds the context's HBM budget");
      return SPRING_E_NOMEM;
    }
  }
  spring_status st = SPRING_OK;
  {
    std::vector<std::unique_ptr<Run>> runs(NG);
    std::vector<cudaStream_t> ss(NG, nullptr);
    std::vector<cudaEvent_t> done(NG, nullptr);
    cudaStream_t origin = nullptr;
    cudaEvent_t fork = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    for (int g = 0; g < NG && e == cudaSuccess; ++g) {
      e = cudaStreamCreateWithFlags(&ss[g], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done[g], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) st = cuda_fail(e, "stream set-up", __FILE__, __LINE__);
    for (int g = 0; g < NG && st == SPRING_OK; ++g) {
      std::vector<const spring_problem*> pg;
      std::vector<uint64_t> sg;
      for (int q : idx[g]) {
        pg.push_back(probs[q]);
        sg.push_back(seeds[q]);
      }
      runs[g].reset(new Run());
      st = runs[g]->setup_batch(pg.data(), (int)pg.size(), sg.data(), *p, ss[g]);
    }
    if (st == SPRING_OK) {
      // the origin stream first waits for every side's set-up (the graph is launched on it);
      // then every side's stream starts after a fork from the origin, and the origin waits
      // for all of them at the end (join)
      for (int g = 0; g < NG && e == cudaSuccess; ++g) {
        e = cudaEventRecord(done[g], ss[g]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(origin, done[g], 0);
      }
      if (e != cudaSuccess) st = cuda_fail(e, "stream join", __FILE__, __LINE__);
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      if (st == SPRING_OK && p->use_graph) {
        e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) st = cuda_fail(e, "cudaStreamBeginCapture", __FILE__, __LINE__);
      }
      if (st == SPRING_OK) {
        e = cudaEventRecord(fork, origin);
        for (int g = 0; g < NG && e == cudaSuccess; ++g) e = cudaStreamWaitEvent(ss[g], fork, 0);
        if (e != cudaSuccess) st = cuda_fail(e, "stream fork", __FILE__, __LINE__);
      }
      if (st != SPRING_OK) {
      } else if (p->use_graph) {
        for (int g = 0; g < NG && st == SPRING_OK; ++g) st = runs[g]->enqueue_all();
      } else {  // one generation of every side in turn, so that the sides' work interleaves
        std::vector<bool> fin(NG, false);
        for (int left = NG; left > 0 && st == SPRING_OK;)
          for (int g = 0; g < NG && st == SPRING_OK; ++g) {
            if (fin[g]) continue;
            bool d = false;
            st = runs[g]->step(&d);
            if (d) {
              fin[g] = true;
              --left;
            }
          }
      }
      for (int g = 0; g < NG && st == SPRING_OK; ++g) {
        e = cudaEventRecord(done[g], ss[g]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(origin, done[g], 0);
        if (e != cudaSuccess) st = cuda_fail(e, "stream join", __FILE__, __LINE__);
      }
      if (p->use_graph && graph == nullptr) {
        e = cudaStreamEndCapture(origin, &graph);
        if (st == SPRING_OK && e != cudaSuccess) st = cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
        if (st == SPRING_OK) {
          e = cudaGraphInstantiate(&exec, graph, 0);
          if (e != cudaSuccess) st = cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__);
        }
        if (st == SPRING_OK) {
          e = cudaGraphLaunch(exec, origin);
          if (e != cudaSuccess) st = cuda_fail(e, "cudaGraphLaunch", __FILE__, __LINE__);
        }
      }
      if (st == SPRING_OK) {
        e = cudaStreamSynchronize(origin);
        if (e != cudaSuccess) st = cuda_fail(e, "batch execution", __FILE__, __LINE__);
      }
      if (exec) cudaGraphExecDestroy(exec);
      if (graph) cudaGraphDestroy(graph);
    }
    if (st == SPRING_OK) st = check_device_waits();
    if (st == SPRING_OK) {
      const double t = now_s();
      for (int g = 0; g < NG && st == SPRING_OK; ++g) {
        std::vector<spring_result> rs(idx[g].size());
        for (size_t j = 0; j < idx[g].size(); ++j) rs[j] = out[idx[g][j]];
        st = runs[g]->collect(rs.data());
        for (size_t j = 0; j < idx[g].size(); ++j) {
          out[idx[g][j]] = rs[j];
          out[idx[g][j]].t_submit_s = out[idx[g][j]].t_admit_s = out[idx[g][j]].t_done_s = t;
        }
      }
    }
    for (int g = 0; g < NG; ++g) {
      if (runs[g]) runs[g]->release();
      if (ss[g]) {
        cudaStreamSynchronize(ss[g]);
        cudaStreamDestroy(ss[g]);
      }
      if (done[g]) cudaEventDestroy(done[g]);
    }
    if (fork) cudaEventDestroy(fork);
    if (origin) cudaStreamDestroy(origin);
  }
  std::lock_guard<std::mutex> lk(c->mu);
  c->used -= fp;
  return st;
}

spring_status spring_mpr_run_batch(spring_problem* const* probs, int K, const spring_params* p,
                                   const uint64_t* seeds, spring_result* out) {
  if (!probs || !p || !seeds || !out) return invalid("null argument");
  if (K <= 0) return invalid("batch size must be positive");
  bool mixed = false;
  for (int q = 0; q < K; ++q) {
    if (!probs[q]) return invalid("null problem in the batch");
    if (probs[q]->ctx != probs[0]->ctx) return invalid("the problems of a batch must share a context");
    mixed = mixed || probs[q]->n != probs[0]->n;
  }
  if (K > 1 && p->precision != 0) return invalid("batched runs keep FP32 storage (precision 0)");
  if (K > 1 && p->mode != 0) return invalid("batched runs are memetic (mode 0)");
  if (mixed) return run_blocking_mixed(probs, K, seeds, p, out);
  return run_blocking_k(probs, K, seeds, p, nullptr, 0, nullptr, out);
}

spring_status spring_mpr_run_until(spring_problem* pr, const spring_params* p, int g_stop,
                                   spring_population* save) {
  if (!pr || !p || !save || !save->pop_x || !save->pop_S || !save->pop_err) return invalid("null argument");
  if (g_stop < 1 || g_stop > p->generations) return invalid("g_stop must be in [1, generations]");
  return run_blocking(pr, p, nullptr, g_stop, save, nullptr);
}

spring_status spring_mpr_resume(spring_problem* pr, const spring_params* p, const spring_population* from,
                                spring_result* out) {
  if (!pr || !p || !from || !out || !from->pop_x || !from->pop_S || !from->pop_err)
    return invalid("null argument");
  if (from->generation < 0 || from->generation >= p->generations)
    return invalid("the saved generation must be in [0, generations)");
  return run_blocking(pr, p, from, 0, nullptr, out);
}

spring_status spring_mpr_step(spring_problem* pr, const spring_params* p, const spring_population* from,
                              spring_population* to, spring_generation_trace* trace) {
  if (!pr || !p || !from || !to || !from->pop_x || !from->pop_S || !from->pop_err || !to->pop_x ||
      !to->pop_S || !to->pop_err)
    return invalid("null argument");
  if (from->generation < 0 || from->generation >= p->generations)
    return invalid("the starting generation must be in [0, generations)");
  if (p->use_graph) return invalid("a single generation is not captured in a graph (use_graph = 0)");
  const int g = from->generation + 1;
  return run_blocking_k(&pr, 1, &p->seed, p, from, g, to, nullptr, trace);
}

spring_status spring_submit(spring_ctx* c, spring_problem* pr, const spring_params* p, uint64_t* ticket) {
  if (!c || !pr || !p || !ticket) return invalid("null argument");
  if (pr->ctx != c) return invalid("problem belongs to another context");
  SPRING_TRY(validate_params(pr->n, *p));
  std::unique_ptr<Ticket> t(new Ticket());
  t->prob = pr;
  t->prm = *p;
  t->footprint = make_layout(pr->n, *p).total;
  t->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(c->mu);
    if (t->footprint > c->budget) {
      set_error("request footprint exceeds the context's HBM budget");
      return SPRING_E_NOMEM;
    }
    t->id = c->next_id++;
    *ticket = t->id;
    pr->refs.fetch_add(1);
    c->queue.push_back(t->id);
    c->tickets[t->id] = std::move(t);
  }
  c->cv.notify_all();
  return SPRING_OK;
}

spring_status spring_poll(spring_ctx* c, uint64_t ticket, int timeout_us, spring_result* out) {
  if (!c) return invalid("null context");
  std::unique_lock<std::mutex> lk(c->mu);
  auto it = c->tickets.find(ticket);
  if (it == c->tickets.end()) {
    set_error("unknown ticket");
    return SPRING_E_NOT_FOUND;
  }
  Ticket* t = it->second.get();
  auto finished = [&]() { return t->state >= T_DONE; };
  if (!finished()) {
    if (timeout_us < 0)
      c->done_cv.wait(lk, finished);
    else if (timeout_us > 0)
      c->done_cv.wait_for(lk, std::chrono::microseconds(timeout_us), finished);
  }
  if (!finished()) return SPRING_E_BUSY;
  spring_status st = SPRING_OK;
  if (t->state == T_CANCELLED) {
    st = SPRING_E_CANCELLED;
    set_error("ticket was cancelled");
  } else if (t->state == T_FAILED) {
    st = t->status;
    set_error(t->message);
  } else if (out) {
    const size_t nn = t->support_avg.size();
    if (out->rho_avg) std::memcpy(out->rho_avg, t->rho_avg.data(), sizeof(float) * 2 * nn);
    if (out->rho_best) std::memcpy(out->rho_best, t->rho_best.data(), sizeof(float) * 2 * nn);
    if (out->support_avg) std::memcpy(out->support_avg, t->support_avg.data(), nn);
    if (out->gen_stats) std::memcpy(out->gen_stats, t->gen_stats.data(), sizeof(double) * t->gen_stats.size());
    out->final_error_avg = t->e_avg;
    out->final_error_best = t->e_best;
    out->t_submit_s = t->t_submit;
    out->t_admit_s = t->t_admit;
    out->t_done_s = t->t_done;
  }
  c->tickets.erase(it);
  return st;
}

spring_status spring_serving_stats(spring_ctx* c, uint64_t* cohorts, uint64_t* admitted) {
  if (!c) return invalid("null context");
  std::lock_guard<std::mutex> lk(c->mu);
  if (cohorts) *cohorts = c->n_cohorts;
  if (admitted) *admitted = c->n_admitted;
  return SPRING_OK;
}

spring_status spring_cancel(spring_ctx* c, uint64_t ticket) {
  if (!c) return invalid("null context");
  {
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->tickets.find(ticket);
    if (it == c->tickets.end()) {
      set_error("unknown ticket");
      return SPRING_E_NOT_FOUND;
    }
    it->second->cancel = true;
  }
  c->cv.notify_all();
  return SPRING_OK;
}

}  // extern "C"
