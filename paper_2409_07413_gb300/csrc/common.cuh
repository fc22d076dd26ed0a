// common.cuh -- shared device/host helpers of libspring (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cmath>
#include <stdint.h>

#include <string>

#include "spring.h"

namespace spring {

// ------------------------------------------------------------------ error plumbing
// Library calls never abort: failures become a spring_status plus a per-thread message.
void set_error(const std::string& msg);
spring_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define SPRING_CUDA(call)                                                         \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) return ::spring::cuda_fail(e_, #call, __FILE__, __LINE__); \
  } while (0)

#define SPRING_TRY(call)                      \
  do {                                        \
    spring_status s_ = (call);                \
    if (s_ != SPRING_OK) return s_;           \
  } while (0)

#define SPRING_CHECK_LAUNCH() SPRING_CUDA(cudaGetLastError())

spring_status invalid(const std::string& msg);

// ------------------------------------------------------------------ launch accounting
// Every kernel launch of the library goes through launch_begin/launch_end so that the
// benchmark can count launches and time the dominant kernel classes with CUDA events
// recorded on the launching stream.
void launch_begin(int kclass, cudaStream_t s);
void launch_end(int kclass, cudaStream_t s, double bytes);

// ------------------------------------------------------------------ sizes and plans
// The supported sides: even N in [64, 1024] of the form 2^a 3^b with b <= 1, in
// ascending order.  side_slot(N) is N's index (-1 if unsupported).
constexpr int N_SIDES = 9;
__host__ __device__ constexpr int side_at(int i) {
  return i == 0 ? 64 : i == 1 ? 96 : i == 2 ? 128 : i == 3 ? 192 : i == 4 ? 256
       : i == 5 ? 384 : i == 6 ? 512 : i == 7 ? 768 : i == 8 ? 1024 : 0;
}
__host__ __device__ constexpr int side_slot(int n) {
  for (int i = 0; i < N_SIDES; ++i)
    if (side_at(i) == n) return i;
  return -1;
}
inline bool valid_n(int n) { return side_slot(n) >= 0; }

// Per-device constant tables, built once on the host in double precision:
//   tw:      e^{-2 pi i k / N}, k < N, for every supported N (rounded once to float),
//            at offset tw_offset(N) (the sides' tables one after another);
//   rot_cos, rot_sin: Q30 fixed point cos/sin((pi/2) k / 1024), k < 1024 (crossover map).
__host__ __device__ constexpr int tw_offset(int n) {
  int o = 0;
  for (int i = 0; i < N_SIDES && side_at(i) != n; ++i) o += side_at(i);
  return o;
}
constexpr int TW_TOTAL = tw_offset(0);  // past the last side: the sum of all sides
// the twiddle tables of every side into tw[TW_TOTAL]
inline void fill_twiddles(float2* tw) {
  for (int i = 0; i < N_SIDES; ++i) {
    const int n = side_at(i);
    for (int k = 0; k < n; ++k) {
      const double ang = -2.0 * 3.14159265358979323846 * (double)k / (double)n;
      tw[tw_offset(n) + k] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
  }
}
struct DeviceTables {
  const float2* tw;
  const long long* rot_cos;
  const long long* rot_sin;
  int* status;  // device status word: bit 2 = a bounded wait in a kernel timed out
};
// Tables of the current device (allocated on first use and kept until process exit).
spring_status device_tables(DeviceTables* out);

// ------------------------------------------------------------------ complex helpers
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// ------------------------------------------------------------------ Philox-4x32-10
// Counter-based generator of Salmon et al. (SC'11): 10 rounds of two 32x32->64
// multiplications mixed with the other counter words and the key; the key advances by
// the Weyl increments between rounds.  Counter layout of this library:
// (generation, individual, tag << 24 | a, b).
__host__ __device__ inline void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              uint32_t k0, uint32_t k1, uint32_t out[4]) {
  for (int round = 0; round < 10; ++round) {
    if (round) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = n0;
    c2 = n2;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

__host__ __device__ inline void draw(uint64_t seed, uint32_t g, uint32_t p, uint32_t tag,
                                     uint32_t a, uint32_t b, uint32_t out[4]) {
  philox4x32_10(g, p, (tag << 24) | (a & 0xFFFFFFu), b, (uint32_t)seed, (uint32_t)(seed >> 32), out);
}

__host__ __device__ inline uint32_t uniform_below(uint32_t u, uint32_t m) {
  return (uint32_t)(((uint64_t)u * m) >> 32);
}

// ------------------------------------------------------------------ launch helpers
inline int div_up(long long a, long long b) { return (int)((a + b - 1) / b); }
int sm_count();  // of the current device

}  // namespace spring
