// k_cluster.cu -- whole iterations on chip for N <= 256: one thread-block cluster per image.
//
// The same iteration as the two-pass path (row pass + column pass through HBM; see
// k_fft.cuh), with the image kept in the shared memory of a cluster of C = N / 32 CTAs
// for all n_iter iterations of a launch.  CTA `rank` owns rows and columns
// [32 rank, 32 rank + 32) and holds, in its shared memory:
//   X  [32][N]      its rows of the state x_n (complex64)
//   R  [32][PITCH]  row buffer: the column-phase output for its rows (the row transforms
//                   run in place here; PITCH is odd and covers the padded exchange)
//   Cc [N][32]      column buffer: the row-phase output for its columns (the column
//                   transforms run in place here, stride 32)
//   S  [32][N]      its rows of the support
// One iteration:
//   column phase: Cc -> forward column FFT -> P_M (Eq. pm_full / pm_bounds, M read from
//                 L2) -> inverse column FFT -> scattered into the owners' R buffers
//                 (distributed shared memory)
//   cluster barrier
//   row phase:    R -> inverse row FFT (= P_M x_n) -> update (ER / HIO / RAAR with S and
//                 chi) -> X = x_{n+1} -> forward row FFT -> scattered into the owners' Cc
//   cluster barrier
// HBM is touched only to load x and S at the start and to store x at the end; M (shared by
// every image) is read from L2.  The arithmetic is the two-pass path's with the default
// plan of side N in both directions, so the results equal those of the two-pass kernels
// with that plan bit for bit.
#include <cooperative_groups.h>

#include "k_fft.cuh"

namespace cg = cooperative_groups;

namespace spring {

template <int N>
struct ClusterLayout {
  static constexpr int RB = 32;                  // rows (and columns) per CTA
  static constexpr int C = N / RB;               // CTAs per image (cluster size, <= 8)
  using P = Plan<N>;
  static constexpr int T = P::T;                 // threads per transform
  static constexpr int THREADS = RB * T;         // one transform per owned row / column
  static constexpr int PITCH = pad_elems_p<P>() | 1;
  static constexpr size_t X_OFF = 0, R_OFF = (size_t)RB * N, C_OFF = R_OFF + (size_t)RB * PITCH,
                          END = C_OFF + (size_t)N * RB;
  static constexpr size_t SMEM = END * sizeof(float2) + (size_t)RB * N;
  // CTAs per SM the register budget is sized for (shared memory allows 2 at N = 128, 4 at 64)
  static constexpr int MINB = (N == 128) ? 2 : (N == 64) ? 4 : 1;
  static_assert(C >= 1 && C <= 8 && N % RB == 0, "cluster of at most 8 CTAs");
  static_assert(T <= 32, "row transforms are owned by lane groups inside a warp");
};

struct ClusterArgs {
  float2* x;          // batch images, updated in place
  const uint8_t* S;   // batch supports
  const float* M;     // modulus (encoded), DFT order
  const float2* tw;
  float beta, cchi;
  int chi_on, n_iter;
  int m_group;        // > 0: one modulus array per m_group consecutive images
};

template <int N, int ALG>
__global__ void __launch_bounds__(ClusterLayout<N>::THREADS, ClusterLayout<N>::MINB) k_cluster_iter(ClusterArgs a) {
  using L = ClusterLayout<N>;
  using P = typename L::P;
  constexpr int T = L::T, E = P::E, RB = L::RB, PITCH = L::PITCH;
  extern __shared__ __align__(16) float2 smem[];
  float2* X = smem + L::X_OFF;
  float2* R = smem + L::R_OFF;
  float2* Cc = smem + L::C_OFF;
  uint8_t* Ss = reinterpret_cast<uint8_t*>(smem + L::END);
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const long long img = blockIdx.x / L::C;
  const int r0 = rank * RB;  // first owned row and column
  const int tid = threadIdx.x;
  const int g = tid / T, t = tid % T;       // row phase: lane t of the group owning row g
  const int cc = tid % RB, ct = tid / RB;   // column phase: thread ct of column cc
  const auto gsync = GroupSync<T>::make();
  const BlockSync bsync;
  float2* xg = a.x + img * N * N + (long long)r0 * N;
  const uint8_t* Sg = a.S + img * N * N + (long long)r0 * N;
  const float* Mi = a.m_group > 0 ? a.M + (img / a.m_group) * N * N : a.M;
  constexpr float inv_n = 1.0f / N;

  for (int k = tid; k < RB * N; k += L::THREADS) {
    X[k] = xg[k];
    Ss[k] = Sg[k];
  }
  cl.sync();  // every CTA of the cluster runs (its shared memory may be written) and X is loaded

  float2 v[E];
  // forward row transform of x_n, scattered into the column owners' Cc
  auto row_forward_scatter = [&]() {
    fft_plan<P, -1, true, 1>(v, R + g * PITCH, t, a.tw, gsync);
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int j = t + m * T;
      float2* dst = cl.map_shared_rank(Cc, j / RB);
      dst[(r0 + g) * RB + (j % RB)] = v[m];
    }
  };
#pragma unroll
  for (int m = 0; m < E; ++m) v[m] = X[g * N + t + m * T];
  row_forward_scatter();
  cl.sync();

  for (int it = 0; it < a.n_iter; ++it) {
    // ---- column phase: my RB columns, N rows each
    float Mv[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int i = ct + m * T;
      v[m] = Cc[i * RB + cc];
      Mv[m] = __ldg(&Mi[(long long)i * N + r0 + cc]);
    }
    bsync();  // every input is in registers before the exchange reuses the tile
    fft_plan<P, -1, false, RB>(v, Cc + cc, ct, a.tw, bsync);
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = pm_value(v[m], Mv[m], inv_n);
    fft_plan<P, +1, false, RB>(v, Cc + cc, ct, a.tw, bsync);
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int i = ct + m * T;
      float2* dst = cl.map_shared_rank(R, i / RB);
      dst[(i % RB) * PITCH + r0 + cc] = v[m];
    }
    cl.sync();
    // ---- row phase: my RB rows
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = R[g * PITCH + t + m * T];
    gsync();
    fft_plan<P, +1, true, 1>(v, R + g * PITCH, t, a.tw, gsync);  // m = P_M x_n
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int k = g * N + t + m * T;
      const float2 pm = v[m];
      bool in_c = Ss[k] != 0;
      if (a.chi_on) in_c = in_c && (pm.x >= a.cchi * sqrtf(pm.x * pm.x + pm.y * pm.y));
      const float2 xn = update_pixel(ALG, ALG ? X[k] : pm, pm, in_c, a.beta);
      X[k] = xn;
      v[m] = xn;
    }
    if (it + 1 < a.n_iter) {
      row_forward_scatter();
      cl.sync();
    }
  }
  __syncthreads();
  for (int k = tid; k < RB * N; k += L::THREADS) xg[k] = X[k];
  cl.sync();  // no CTA leaves while another may still address its shared memory
}

template <int N, int ALG>
static spring_status cluster_launch(const ClusterArgs& a, long long batch, bool prepare_only, cudaStream_t s) {
  using L = ClusterLayout<N>;
  auto kern = k_cluster_iter<N, ALG>;
  if (prepare_only) return allow_smem(kern, L::SMEM);
  if (batch < 1 || a.n_iter < 1) return SPRING_OK;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(batch * L::C));
  cfg.blockDim = dim3(L::THREADS);
  cfg.dynamicSmemBytes = L::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = L::C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  // algorithmic HBM bytes: x and S (1 bit/px) in, x out, once per launch (M from L2)
  const double bytes = (double)batch * N * N * 16.125;
  launch_begin(SPRING_KC_FUSED, s);
  SPRING_CUDA(cudaLaunchKernelEx(&cfg, kern, a));
  launch_end(SPRING_KC_FUSED, s, bytes);
  return SPRING_OK;
}

template <int N>
static spring_status cluster_dispatch(int alg, const ClusterArgs& a, long long batch, bool prep,
                                      cudaStream_t s) {
  if (prep) {
    SPRING_TRY((cluster_launch<N, 0>(a, batch, true, s)));
    SPRING_TRY((cluster_launch<N, 1>(a, batch, true, s)));
    return cluster_launch<N, 2>(a, batch, true, s);
  }
  if (alg == 0) return cluster_launch<N, 0>(a, batch, false, s);
  if (alg == 1) return cluster_launch<N, 1>(a, batch, false, s);
  return cluster_launch<N, 2>(a, batch, false, s);
}

static spring_status cluster_any(int n, int alg, const ClusterArgs& a, long long batch, bool prep,
                                 cudaStream_t s) {
  switch (n) {
    case 64: return cluster_dispatch<64>(alg, a, batch, prep, s);
    case 128: return cluster_dispatch<128>(alg, a, batch, prep, s);
    case 192: return cluster_dispatch<192>(alg, a, batch, prep, s);
    case 256: return cluster_dispatch<256>(alg, a, batch, prep, s);
    default: return invalid("the on-chip iteration kernel covers N <= 256");
  }
}

bool cluster_side(int n) { return n == 64 || n == 128 || n == 192 || n == 256; }

// Raise the shared-memory limit of the cluster kernels of side n (before any capture).
spring_status prepare_cluster_kernels(int n) {
  if (!cluster_side(n)) return SPRING_OK;
  ClusterArgs a{};
  return cluster_any(n, 0, a, 0, true, nullptr);
}

// Can clusters of side n be resident on this device (shared memory, cluster shape)?
spring_status cluster_supported(int n, bool* ok) {
  *ok = false;
  if (!cluster_side(n)) return SPRING_OK;
  SPRING_TRY(prepare_cluster_kernels(n));
  int dev = 0;
  SPRING_CUDA(cudaGetDevice(&dev));
  int smem_optin = 0;
  SPRING_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  size_t need = 0;
  int threads = 0, csize = 0;
  const void* fn = nullptr;
  switch (n) {
    case 64: need = ClusterLayout<64>::SMEM; threads = ClusterLayout<64>::THREADS; csize = ClusterLayout<64>::C;
      fn = (const void*)k_cluster_iter<64, 2>; break;
    case 128: need = ClusterLayout<128>::SMEM; threads = ClusterLayout<128>::THREADS; csize = ClusterLayout<128>::C;
      fn = (const void*)k_cluster_iter<128, 2>; break;
    case 192: need = ClusterLayout<192>::SMEM; threads = ClusterLayout<192>::THREADS; csize = ClusterLayout<192>::C;
      fn = (const void*)k_cluster_iter<192, 2>; break;
    default: need = ClusterLayout<256>::SMEM; threads = ClusterLayout<256>::THREADS; csize = ClusterLayout<256>::C;
      fn = (const void*)k_cluster_iter<256, 2>; break;
  }
  if (need > (size_t)smem_optin) return SPRING_OK;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)csize);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = need;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = csize;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int clusters = 0;
  SPRING_CUDA(cudaOccupancyMaxActiveClusters(&clusters, fn, &cfg));
  *ok = clusters > 0;
  return SPRING_OK;
}

spring_status launch_cluster_iter(int n, int alg, float2* x, const uint8_t* S, const float* M, long long batch,
                                  float beta, float chi, int n_iter, cudaStream_t s, int m_group) {
  if (alg < 0 || alg > 2) return invalid("algorithm must be 0 (ER), 1 (HIO) or 2 (RAAR)");
  DeviceTables tb;
  SPRING_TRY(device_tables(&tb));
  ClusterArgs a{};
  a.x = x;
  a.S = S;
  a.M = M;
  a.tw = tb.tw + tw_offset(n);
  a.beta = beta;
  a.chi_on = chi < 1.0f;
  a.cchi = (float)((chi == 0.5f) ? 0.0 : std::cos((double)chi * 3.14159265358979323846));
  a.n_iter = n_iter;
  a.m_group = m_group;
  return cluster_any(n, alg, a, batch, false, s);
}

}  // namespace spring
