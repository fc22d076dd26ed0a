// internal.h -- launchers shared by the translation units of libspring.
// All pointers are device pointers; every launcher is asynchronous on stream s.
#pragma once

#include "common.cuh"

namespace spring {

// ---------------------------------------------------------------- k_fft.cu
// iteration row pass: w (column-pass output) -> P_M x -> update -> x, rowFFT(x) -> w
// split passes (sides 192, 384, 512, 768 and 1024; k_fft.cuh): the modulus permuted to the chunked layout,
// the split row pass (fwd_only: forward row transforms and first stage of x alone), the
// split column pass, and k iterations of the two
bool split_supported(int n);
spring_status launch_split_modulus(int n, const float* M, float* Mp, int K, cudaStream_t s);
spring_status launch_row_split(int n, int alg, bool fwd_only, float2* w, float2* x, const uint32_t* Sb,
                               long long batch, float beta, float chi, cudaStream_t s);
spring_status launch_col_split(int n, float2* w, const float* Mp, int batch, cudaStream_t s, int m_group = 0);
spring_status iterate_split(int n, int alg, float2* w, float2* x, const uint32_t* Sb, const float* Mp,
                            long long batch, int m_group, float beta, float chi, int k, cudaStream_t s);
// Sb: the supports packed to one bit per pixel (launch_pack_support)
spring_status launch_pack_support(const uint8_t* S, uint32_t* Sb, long long npix, cudaStream_t s);
spring_status launch_row_iter(int n, int alg, float2* w, float2* x, const uint32_t* Sb,
                              long long batch, float beta, float chi, bool zout, cudaStream_t s);
// iteration column pass: colFFT, masked modulus projection, colIFFT, in place on w.
// m_group > 0: M holds one N x N array per m_group consecutive images (a batch of patterns)
spring_status launch_col_pm(int n, float2* w, const float* M, int batch, cudaStream_t s, int m_group = 0,
                           int img0 = 0);
// plain row transform (dir -1 forward, +1 inverse), unnormalised times `scale`;
// Smul (forward only, may be null) multiplies the input by the support first
spring_status launch_row_fft(int n, int dir, const float2* in, float2* out, const uint8_t* Smul,
                             long long batch, float scale, cudaStream_t s);
// plain column transform in place, times `scale`
spring_status launch_col_fft(int n, int dir, float2* data, int batch, float scale, cudaStream_t s);
// column forward transform + per-block FP64 partial sums of the Fourier error
int err_strips(int n);
spring_status launch_col_err(int n, float2* w, const float* M, int batch, double* partials,
                             cudaStream_t s, int m_group = 0, bool skip_m2 = false);
// err = sqrt(num / den) per image; m2 != nullptr: den from m2 (one value per m_group
// consecutive images, or m2[0] for all with m_group 0) instead of the partials
spring_status launch_err_finalize(int n, const double* partials, int batch, double* err,
                                  int* status, cudaStream_t s, const double* m2 = nullptr,
                                  int m_group = 0);
// m2[k] = sum of M^2 over the measured pixels (M >= 0) of the k-th of K modulus arrays, FP64
spring_status launch_m2_sum(int n, const float* M, int K, double* m2, cudaStream_t s);
// the same two error launchers with a caller-supplied twiddle table (all sides, laid out
// at tw_offset(N)) instead of the per-device one
spring_status launch_row_fft_tw(int n, int dir, const float2* in, float2* out, const uint8_t* Smul,
                                long long batch, float scale, const float2* tw_all, cudaStream_t s);
spring_status launch_col_err_tw(int n, float2* w, const float* M, int batch, double* partials,
                                const float2* tw_all, cudaStream_t s, int m_group = 0,
                                bool skip_m2 = false);

// FP16 storage of the iteration buffers (precision 1): wh, xh are half2 arrays; x is kept
// scaled by the device scalar s16 (a power of two from launch_fp16_scale), w by s16 times a
// power of two near 1/sqrt(N)
spring_status launch_fp16_scale(int n, const float* M, float* s16, cudaStream_t s);
spring_status launch_row_iter16(int n, int alg, void* wh, void* xh, const uint32_t* Sb, long long batch,
                                float beta, float chi, const float* s16, cudaStream_t s);
spring_status launch_col_pm16(int n, void* wh, const float* M, int batch, const float* s16, cudaStream_t s);
spring_status launch_row_init16(int n, const float2* x, void* xh, void* wh, long long batch, const float* s16,
                                cudaStream_t s);
spring_status launch_half_to_float(const void* xh, float2* x, long long total, const float* s16, cudaStream_t s);

// the on-chip whole-iteration kernel (k_cluster.cu): n_iter iterations of ER/HIO/RAAR on
// `batch` images of side n <= 256 in place, one thread-block cluster per image
bool cluster_side(int n);
spring_status prepare_cluster_kernels(int n);
spring_status cluster_supported(int n, bool* ok);
spring_status launch_cluster_iter(int n, int alg, float2* x, const uint8_t* S, const float* M, long long batch,
                                  float beta, float chi, int n_iter, cudaStream_t s, int m_group = 0);
// 0: two passes through HBM per iteration; 1: the on-chip kernel (set by the autotuner)
int iteration_path(int n);

// kernel-variant autotuning of side n on `batch` images (once per process and side)
spring_status ensure_tuned(int n, int batch, cudaStream_t s);
spring_status prepare_fft_kernels(int n);

// tiled 3-D TMA descriptor of a float32 array (dim0 x dim1 x dim2, dim0 contiguous), box
// box0 x box1 x 1; the descriptor is encoded on the host (driver entry point)
spring_status encode_tmap_f32_3d(void* map, const void* base, int dim0, int dim1, int dim2, int box0,
                                 int box1);
// read and clear the per-device status word (bit 2: a kernel's bounded wait timed out)
spring_status take_device_status(int* out);
// SPRING_E_TIMEOUT (and clears the word) if a bounded device-side wait timed out
spring_status check_device_waits();

// ---------------------------------------------------------------- composite transforms
// unitary 2D transform of `batch` images: out = F x (dir -1) or F^-1 x (dir +1); in may
// equal out.  Smul (forward only): transform S x instead of x.
spring_status fft2_unitary(int n, int dir, const float2* in, float2* out, const uint8_t* Smul,
                           int batch, cudaStream_t s);

// ---------------------------------------------------------------- k_sw.cu
constexpr int SW_MAX_RADIUS = 256;
spring_status launch_smooth(int n, const float2* x, float* tmp, float* out, int batch, float sigma,
                            unsigned* img_max, cudaStream_t s);
spring_status launch_threshold(int n, const float* sm, const unsigned* img_max, float tau,
                               uint8_t* S, int batch, cudaStream_t s);
// image b uses alpha[(b / alpha_group) * alpha_stride]; scratch: device memory of
// select_area_scratch_bytes(n, batch) bytes (at most batch x N x N floats for N >= 64)
size_t select_area_scratch_bytes(int n, int batch);
spring_status launch_select_area(int n, const float* sm, const int64_t* alpha, int alpha_stride,
                                 uint8_t* S, int batch, cudaStream_t s, int alpha_group, void* scratch);

// ---------------------------------------------------------------- k_ga.cu
spring_status launch_random_choice(uint64_t seed, int g, int P, int32_t* abc, cudaStream_t s);
spring_status launch_crossover_map(uint64_t seed, int g, int p, int n, int tmin, int tmax, float cp,
                                   uint8_t* map, cudaStream_t s);
// cross-correlation spectra of pairs q = (x index ix[q], ref index ir[q]) from unitary
// spectra X:  A[q] = Xi conj(X[ix]) X[ir]   and   B[q] = Xi X[ix] X[ir]  (twin)
spring_status launch_xcorr_spectra(int n, const float2* X, const int32_t* ix, const int32_t* ir,
                                   int npairs, const float* M, float2* A, float2* B, cudaStream_t s);
// peak search over the correlation images A[q], B[q] -> info[3q..] = (s_y, s_x, twin),
// phasor[q] = c(s) / |c(s)|
size_t peaks_scratch_bytes(int n, int npairs);
spring_status launch_peaks(int n, const float2* A, const float2* B, int npairs, int32_t* info,
                           float2* phasor, void* scratch, cudaStream_t s);
// real-space alignment: out[q] = phasor[q] x[ix[q]](r - s)   (or phasor conj(x(s - r)))
spring_status launch_apply_shift(int n, const float2* x, const uint8_t* S, const int32_t* ix,
                                 int npairs, const int32_t* info, const float2* phasor,
                                 float2* x_out, uint8_t* S_out, cudaStream_t s);
// crossover mix in Fourier space (parents' alignment applied by the shift theorem); with
// ca > 0 parent a's moduli are blended towards mavg (Eq. crossavg)
spring_status launch_crossover_mix(int n, const float2* Xpop, const int32_t* abc,
                                   const int32_t* info, const float2* phasor, int P, uint64_t seed,
                                   int g, float cw, float cp, int tmin, int tmax, float ca,
                                   const float* mavg, float2* Xnew, cudaStream_t s);
// mavg = (|avg_spec| + mean_p |Xpop_p|) / 2 (Eqs. avgint1, avgint2; unitary spectra)
spring_status launch_average_moduli(int n, const float2* Xpop, const float2* avg_spec, int P, float* mavg,
                                    cudaStream_t s);
spring_status launch_crossover_support(int n, const uint8_t* Spop, const int32_t* abc,
                                       const int32_t* info, int P, uint8_t* Snew, cudaStream_t s);
spring_status launch_pairs_crossover(int P, const int32_t* abc, int32_t* ix, int32_t* ir,
                                     cudaStream_t s);
spring_status launch_select(int n, float2* pop_x, uint8_t* pop_S, double* pop_err,
                            const float2* new_x, const uint8_t* new_S, const double* new_err,
                            int P, uint8_t* replaced, cudaStream_t s);
// argmin of err (ties: lowest index); err null -> 0
spring_status launch_argmin(const double* err, int P, int32_t* best, cudaStream_t s);
spring_status launch_pairs_onto_best(int P, const int32_t* best, int32_t* ix, int32_t* ir,
                                     cudaStream_t s);
spring_status launch_average(int n, const float2* x, const uint8_t* S, const int32_t* info,
                             const float2* phasor, const int32_t* best, int P, float2* avg,
                             uint8_t* S_avg, cudaStream_t s);
spring_status launch_area_stats(int n, const uint8_t* S, const int32_t* best, int P, int g, int G,
                                int64_t* out3, cudaStream_t s);
size_t init_scratch_bytes(int P, int n_spheres);
spring_status launch_init_spheres(int n, uint64_t seed, const uint8_t* S0, int P, int n_spheres,
                                  float gamma, float phi_max, float2* x, void* scratch,
                                  cudaStream_t s);
size_t normalise_scratch_bytes(int P);
spring_status launch_normalise(int n, const float2* X, const float* M, int P, float2* x,
                               double* partials, cudaStream_t s);
size_t density_scratch_bytes(int P);
spring_status launch_density_sums(int n, const float2* x, int P, double* partials, double* out,
                                  cudaStream_t s);
spring_status launch_gen_stats(int n, const double* err, const uint8_t* S, const uint8_t* replaced,
                               const double* dens, int P, double* row, cudaStream_t s);
// M (DFT order) from detector-centred I, mask and optional saturation map, with the upper
// bounds of Eq. pm_bounds encoded as -2 - U when b enables them; ring_scratch holds
// ring_count(n) doubles
int ring_count(int n);
spring_status launch_modulus_encode(int n, const float* I_c, const uint8_t* mask_c, const uint8_t* sat_c,
                                    const spring_bounds* b, double* ring_scratch, float* M, cudaStream_t s);
spring_status launch_make_modulus(int n, const float* I_centred, const uint8_t* mask_centred,
                                  float* M, cudaStream_t s);
spring_status launch_broadcast_support(int n, const uint8_t* S0, int P, uint8_t* S, cudaStream_t s);

// ---------------------------------------------------------------- scratch
// stream-ordered device scratch (cudaMallocAsync on the current device's pool)
struct Scratch {
  void* p = nullptr;
  cudaStream_t s = nullptr;
  Scratch() = default;
  Scratch(const Scratch&) = delete;
  Scratch& operator=(const Scratch&) = delete;
  ~Scratch() {
    if (p) cudaFreeAsync(p, s);
  }
  spring_status alloc(size_t bytes, cudaStream_t stream);
  template <class T>
  T* as() const { return reinterpret_cast<T*>(p); }
};

}  // namespace spring
