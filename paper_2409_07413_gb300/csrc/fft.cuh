// fft.cuh -- register / shared-memory Stockham FFT engine (sm_103a).
//
// A length-N transform is done by T = N / E threads; thread t holds E elements in
// registers, v[m] = x[t + m T] on entry and X[t + m T] on exit (natural order both
// ways, so global loads and stores of rows stay coalesced and a point-wise operation can
// sit between a forward and an inverse transform without touching memory).
//
// Stage s of radix R (NS = product of the earlier radices) takes, for butterfly
// j = t + u T (u < E/R), the inputs j + r N/R, multiplies input r by W_{NS R}^{(j mod NS) r},
// does a radix-R DFT in registers and writes output r to (j / NS) NS R + (j mod NS) + r NS
// (Stockham autosort).  Between stages the data goes through shared memory.  With
// PAD the exchange layout of the stage that produced groups of L = NS R is
// p(i) = i + (i / L) NS, which makes both the strided writes and the unit-stride reads of
// a half-warp hit distinct banks (64-bit accesses) for power-of-two radices.
//
// Unnormalised: DIR = -1 computes sum x e^{-2 pi i k n / N}, DIR = +1 the conjugate sum.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace spring {

// cos(2 pi k / 32) for k = 0..8 (mathematical constants).
__host__ __device__ constexpr double cos32_tab(int k) {
  return k == 0 ? 1.0 : k == 1 ? 0.98078528040323044913 : k == 2 ? 0.92387953251128675613
       : k == 3 ? 0.83146961230254523708 : k == 4 ? 0.70710678118654752440
       : k == 5 ? 0.55557023301960222474 : k == 6 ? 0.38268343236508977173
       : k == 7 ? 0.19509032201612826785 : 0.0;
}
__host__ __device__ constexpr double cos32(int k) {
  return (k & 31) <= 8 ? cos32_tab(k & 31)
       : (k & 31) <= 16 ? -cos32_tab(16 - (k & 31))
       : (k & 31) <= 24 ? -cos32_tab((k & 31) - 16)
       : cos32_tab(32 - (k & 31));
}
__host__ __device__ constexpr double sin32(int k) { return cos32(k - 8); }

// Two complex values moved and transformed together: a thread that owns two adjacent
// columns carries both through one transform, so every load, store and exchange is a
// 16-byte access.  Arithmetic is lane-wise (each half exactly as a float2 would be).
struct __align__(16) cpair {
  float2 a, b;
};
__device__ __forceinline__ cpair cadd(cpair x, cpair y) { return {cadd(x.a, y.a), cadd(x.b, y.b)}; }
__device__ __forceinline__ cpair csub(cpair x, cpair y) { return {csub(x.a, y.a), csub(x.b, y.b)}; }
__device__ __forceinline__ cpair cmul(cpair x, float2 w) { return {cmul(x.a, w), cmul(x.b, w)}; }
__device__ __forceinline__ cpair cscale(cpair x, float s) { return {cscale(x.a, s), cscale(x.b, s)}; }

// a * (DIR i)
template <int DIR>
__device__ __forceinline__ float2 rot90(float2 a) {
  return DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}
template <int DIR>
__device__ __forceinline__ cpair rot90(cpair x) {
  return {rot90<DIR>(x.a), rot90<DIR>(x.b)};
}

// a * W_R^k with W_R = e^{DIR 2 pi i / R}, R | 32, constant-folded special cases.
template <int R, int K, int DIR>
__device__ __forceinline__ float2 twc(float2 a) {
  constexpr int k = (K * (32 / R)) & 31;  // angle in units of 2 pi / 32
  if constexpr (k == 0) {
    return a;
  } else if constexpr (k == 8) {
    return rot90<DIR>(a);
  } else if constexpr (k == 16) {
    return make_float2(-a.x, -a.y);
  } else if constexpr (k == 24) {
    return rot90<-DIR>(a);
  } else if constexpr (k == 4 || k == 12 || k == 20 || k == 28) {
    constexpr float h = 0.70710678118654752440f;
    constexpr float c = (float)(cos32(k) > 0 ? 1 : -1), s = (float)(sin32(k) > 0 ? 1 : -1) * DIR;
    // (a.x + i a.y)(c + i s) / sqrt 2
    return make_float2((c * a.x - s * a.y) * h, (c * a.y + s * a.x) * h);
  } else {
    constexpr float c = (float)cos32(k), s = (float)(DIR * sin32(k));
    return make_float2(c * a.x - s * a.y, c * a.y + s * a.x);
  }
}
template <int R, int K, int DIR>
__device__ __forceinline__ cpair twc(cpair x) {
  return {twc<R, K, DIR>(x.a), twc<R, K, DIR>(x.b)};
}

// v0 - t / 2 (radix 3)
__device__ __forceinline__ float2 sub_half(float2 v0, float2 t) {
  return make_float2(v0.x - 0.5f * t.x, v0.y - 0.5f * t.y);
}
__device__ __forceinline__ cpair sub_half(cpair v0, cpair t) { return {sub_half(v0.a, t.a), sub_half(v0.b, t.b)}; }

// In-place radix-R DFT of v[0..R), natural order in and out.
template <int R, int DIR>
struct DFT {
  template <class V>
  __device__ __forceinline__ static void run(V* v) {
    V e[R / 2], o[R / 2];
#pragma unroll
    for (int k = 0; k < R / 2; ++k) {
      e[k] = v[2 * k];
      o[k] = v[2 * k + 1];
    }
    DFT<R / 2, DIR>::run(e);
    DFT<R / 2, DIR>::run(o);
    combine(v, e, o, std::integral_constant<int, 0>());
  }
  template <int K, class V>
  __device__ __forceinline__ static void combine(V* v, const V* e, const V* o, std::integral_constant<int, K>) {
    if constexpr (K < R / 2) {
      V t = twc<R, K, DIR>(o[K]);
      v[K] = cadd(e[K], t);
      v[K + R / 2] = csub(e[K], t);
      combine(v, e, o, std::integral_constant<int, K + 1>());
    }
  }
};
template <int DIR>
struct DFT<1, DIR> {
  template <class V>
  __device__ __forceinline__ static void run(V*) {}
};
template <int DIR>
struct DFT<2, DIR> {
  template <class V>
  __device__ __forceinline__ static void run(V* v) {
    V a = v[0];
    v[0] = cadd(a, v[1]);
    v[1] = csub(a, v[1]);
  }
};
template <int DIR>
struct DFT<4, DIR> {
  template <class V>
  __device__ __forceinline__ static void run(V* v) {
    V t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    V t2 = cadd(v[1], v[3]), t3 = rot90<DIR>(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
  }
};
template <int DIR>
struct DFT<3, DIR> {
  template <class V>
  __device__ __forceinline__ static void run(V* v) {
    constexpr float h3 = 0.86602540378443864676f;  // sqrt(3) / 2
    V t1 = cadd(v[1], v[2]), t2 = csub(v[1], v[2]);
    V m = sub_half(v[0], t1);
    V r = cscale(rot90<DIR>(t2), h3);
    v[0] = cadd(v[0], t1);
    v[1] = cadd(m, r);
    v[2] = csub(m, r);
  }
};

// ------------------------------------------------------------------ sync policies
struct WarpSync {  // a transform owned by a lane group inside one warp
  unsigned mask;
  __device__ __forceinline__ void operator()() const { __syncwarp(mask); }
};
struct BlockSync {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
// a transform owned by NT threads (whole warps) of a block: named barrier `id` (1..15)
struct NamedSync {
  unsigned id, nt;
  __device__ __forceinline__ void operator()() const {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nt) : "memory");
  }
};

// ------------------------------------------------------------------ plans
// A plan: transform length N, elements per thread E (T = N / E threads per transform),
// radices R0 .. R4 (two to five stages; the unused trailing radices are 0).  E is a
// multiple of every radix.
template <int N_, int E_, int R0_, int R1_, int R2_ = 0, int R3_ = 0, int R4_ = 0>
struct PlanT {
  static constexpr int N = N_, E = E_, R0 = R0_, R1 = R1_, R2 = R2_, R3 = R3_, R4 = R4_, T = N_ / E_;
  // radix of stage s (0 past the last stage)
  __host__ __device__ static constexpr int radix(int s) {
    return s == 0 ? R0_ : s == 1 ? R1_ : s == 2 ? R2_ : s == 3 ? R3_ : s == 4 ? R4_ : 0;
  }
  // product of the radices of the stages before s
  __host__ __device__ static constexpr int span(int s) { return s <= 0 ? 1 : span(s - 1) * radix(s - 1); }
  static_assert(R0_ * R1_ * (R2_ ? R2_ : 1) * (R3_ ? R3_ : 1) * (R4_ ? R4_ : 1) == N_,
                "radices must multiply to N");
  static_assert((R3_ == 0 || R2_ != 0) && (R4_ == 0 || R3_ != 0), "no gaps between stages");
  static_assert(E_ % R0_ == 0 && E_ % R1_ == 0 && (R2_ == 0 || E_ % R2_ == 0) && (R3_ == 0 || E_ % R3_ == 0) &&
                    (R4_ == 0 || E_ % R4_ == 0),
                "E vs radices");
};
// default plan for each supported N
template <int N> struct Plan;
template <> struct Plan<64>   : PlanT<64, 8, 8, 8> {};
template <> struct Plan<96>   : PlanT<96, 24, 4, 8, 3> {};
template <> struct Plan<128>  : PlanT<128, 16, 8, 16> {};
template <> struct Plan<192>  : PlanT<192, 24, 8, 8, 3> {};
template <> struct Plan<256>  : PlanT<256, 16, 16, 16> {};
template <> struct Plan<384>  : PlanT<384, 24, 8, 4, 4, 3> {};
template <> struct Plan<512>  : PlanT<512, 16, 8, 8, 8> {};
template <> struct Plan<768>  : PlanT<768, 24, 8, 8, 4, 3> {};
template <> struct Plan<1024> : PlanT<1024, 32, 32, 32> {};

// shared-memory elements of one transform's padded exchange buffer: the largest layout
// of a stage whose outputs go through shared memory (every stage but the last)
template <class P>
__host__ __device__ constexpr int pad_elems_p() {
  int m = 0;
  for (int s = 0; P::radix(s + 1) != 0; ++s) {
    const int e = P::N + P::N / P::radix(s);
    m = e > m ? e : m;
  }
  return m;
}
template <int N>
__host__ __device__ constexpr int pad_elems() { return pad_elems_p<Plan<N>>(); }

// ------------------------------------------------------------------ stage helpers
// twiddle multiplications of a stage: input r of butterfly u times W_{NS R}^{(j mod NS) r}
template <int N, int E, int R, int NS, int DIR, class V>
__device__ __forceinline__ void stage_twiddle(V (&b)[E], int t, const float2* __restrict__ tw) {
  constexpr int T = N / E;
  constexpr int STEP = N / (NS * R);  // table index of W_{NS R}^{1}
#pragma unroll
  for (int u = 0; u < E / R; ++u) {
    const int j = t + u * T;
    const int k1 = (j % NS) * STEP;
    // powers by binary decomposition from table entries W^1, W^2, W^4, ...
    float2 pw[6];
    int np = 0;
    // W^1 from the table, W^2, W^4, ... by squaring (one load per butterfly: the exchange
    // traffic already keeps the load/store pipe busy)
    {
      float2 w = __ldg(&tw[k1 % N]);
      w = DIR < 0 ? w : cconj(w);
#pragma unroll
      for (int q = 1; q < R; q <<= 1) {
        pw[np++] = w;
        w = cmul(w, w);
      }
    }
#pragma unroll
    for (int r = 1; r < R; ++r) {
      float2 w;
      bool have = false;
#pragma unroll
      for (int q = 0; q < 6; ++q)
        if ((r >> q) & 1) {
          w = have ? cmul(w, pw[q]) : pw[q];
          have = true;
        }
      b[u * R + r] = cmul(b[u * R + r], w);
    }
  }
}

// radix-3 stages (sides 3 x 2^k) use direct table loads
template <int N, int E, int NS, int DIR, class V>
__device__ __forceinline__ void stage_twiddle3(V (&b)[E], int t, const float2* __restrict__ tw) {
  constexpr int T = N / E, R = 3, STEP = N / (NS * R);
#pragma unroll
  for (int u = 0; u < E / R; ++u) {
    const int j = t + u * T;
    const int k1 = (j % NS) * STEP;
#pragma unroll
    for (int r = 1; r < R; ++r) {
      float2 w = __ldg(&tw[(k1 * r) % N]);
      b[u * R + r] = cmul(b[u * R + r], DIR < 0 ? w : cconj(w));
    }
  }
}

template <int L, int PADN, bool PAD>
__device__ __forceinline__ int xlayout(int i) {
  return PAD ? i + (i / L) * PADN : i;
}

// write the outputs of a stage (radix R, NS) in the exchange layout
template <int N, int E, int R, int NS, bool PAD, int STRIDE, class V>
__device__ __forceinline__ void stage_store(const V (&b)[E], V* sm, int t) {
  constexpr int T = N / E;
#pragma unroll
  for (int u = 0; u < E / R; ++u) {
    const int j = t + u * T;
    const int base = PAD ? (j / NS) * (NS * R + NS) + (j % NS) : (j / NS) * NS * R + (j % NS);
#pragma unroll
    for (int r = 0; r < R; ++r) sm[(base + r * NS) * STRIDE] = b[u * R + r];
  }
}

// read the inputs of a stage of radix R from the layout of the previous stage (groups L,
// padding PADN)
template <int N, int E, int R, int L, int PADN, bool PAD, int STRIDE, class V>
__device__ __forceinline__ void stage_load(V (&b)[E], const V* sm, int t) {
  constexpr int T = N / E;
#pragma unroll
  for (int u = 0; u < E / R; ++u) {
    const int j = t + u * T;
#pragma unroll
    for (int r = 0; r < R; ++r) b[u * R + r] = sm[xlayout<L, PADN, PAD>(j + r * (N / R)) * STRIDE];
  }
}

template <int N, int E, int R, int DIR, class V>
__device__ __forceinline__ void stage_dft(V (&b)[E]) {
#pragma unroll
  for (int u = 0; u < E / R; ++u) DFT<R, DIR>::run(&b[u * R]);
}

template <int N, int E, int R, int NS, int DIR, class V>
__device__ __forceinline__ void stage_tw(V (&b)[E], int t, const float2* __restrict__ tw) {
  if constexpr (NS > 1) {
    if constexpr (R == 3)
      stage_twiddle3<N, E, NS, DIR>(b, t, tw);
    else
      stage_twiddle<N, E, R, NS, DIR>(b, t, tw);
  }
}

// ------------------------------------------------------------------ the transform
// v: E registers of thread t (element t + m T).  sm: this transform's exchange buffer
// (with STRIDE between consecutive elements).  tw: table of e^{-2 pi i k / N}.
// TAIL = false leaves out the barrier after the last shared-memory read: for callers that
// synchronise themselves before the buffer is written again, or never write it again.
// stages S >= 1 of plan P: inputs from the layout of stage S - 1 (groups of span(S),
// padding span(S - 1)), twiddles, radix-R DFT; then the next stage through shared memory,
// or, after the last stage, the outputs into v
template <class P, int DIR, bool PAD, int STRIDE, bool TAIL, int S, class Sync, class V>
__device__ __forceinline__ void fft_stages(V (&v)[P::E], V (&b)[P::E], V* sm, int t, const float2* __restrict__ tw,
                                           const Sync& sync) {
  constexpr int N = P::N, E = P::E, R = P::radix(S), NS = P::span(S);
  constexpr bool LAST = P::radix(S + 1) == 0;
  stage_load<N, E, R, NS, P::span(S - 1), PAD, STRIDE>(b, sm, t);
  if (TAIL || !LAST) sync();
  stage_tw<N, E, R, NS, DIR>(b, t, tw);
  stage_dft<N, E, R, DIR>(b);
  if constexpr (LAST) {
#pragma unroll
    for (int u = 0; u < E / R; ++u)
#pragma unroll
      for (int r = 0; r < R; ++r) v[u + r * (E / R)] = b[u * R + r];
  } else {
    stage_store<N, E, R, NS, PAD, STRIDE>(b, sm, t);
    sync();
    fft_stages<P, DIR, PAD, STRIDE, TAIL, S + 1>(v, b, sm, t, tw, sync);
  }
}

// v: E registers of thread t (element t + m T).  sm: this transform's exchange buffer
// (with STRIDE between consecutive elements).  tw: table of e^{-2 pi i k / N}.
// TAIL = false leaves out the barrier after the last shared-memory read: for callers that
// synchronise themselves before the buffer is written again, or never write it again.
template <class P, int DIR, bool PAD, int STRIDE, bool TAIL = true, class Sync, class V>
__device__ __forceinline__ void fft_plan(V (&v)[P::E], V* sm, int t, const float2* __restrict__ tw,
                                         const Sync& sync) {
  constexpr int N = P::N, E = P::E, R0 = P::R0;
  V b[E];
  // stage 0 (NS = 1): inputs j + r N/R0 are the registers u + r E/R0
#pragma unroll
  for (int u = 0; u < E / R0; ++u)
#pragma unroll
    for (int r = 0; r < R0; ++r) b[u * R0 + r] = v[u + r * (E / R0)];
  stage_dft<N, E, R0, DIR>(b);
  stage_store<N, E, R0, 1, PAD, STRIDE>(b, sm, t);
  sync();
  fft_stages<P, DIR, PAD, STRIDE, TAIL, 1>(v, b, sm, t, tw, sync);
}

// the default plan of side N
template <int N, int DIR, bool PAD, int STRIDE, class Sync>
__device__ __forceinline__ void fft_regs(float2 (&v)[Plan<N>::E], float2* sm, int t,
                                         const float2* __restrict__ tw, const Sync& sync) {
  fft_plan<Plan<N>, DIR, PAD, STRIDE>(v, sm, t, tw, sync);
}

}  // namespace spring
