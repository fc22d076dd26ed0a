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

// Two complex values of two independent transforms packed by component: re = (real part of
// the first, real part of the second), im likewise.  Both lanes always take the same
// operation, so each step is one two-lane FP32 instruction (add / sub / mul / fma .f32x2 of
// sm_100 and later) where two float2 values take two each, and a product with +-i only
// renames the halves.  Each lane rounds exactly as the scalar operation does.
struct __align__(16) cpk {
  float2 re, im;
};
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) {
  float2 r;
  asm("{\n\t.reg .b64 pa, pb, pr;\n\t"
      "mov.b64 pa, {%2, %3};\n\t"
      "mov.b64 pb, {%4, %5};\n\t"
      "sub.rn.f32x2 pr, pa, pb;\n\t"
      "mov.b64 {%0, %1}, pr;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 f2dup(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 f2neg(float2 a) { return f2mul(a, f2dup(-1.0f)); }

__device__ __forceinline__ cpk cadd(cpk x, cpk y) { return {f2add(x.re, y.re), f2add(x.im, y.im)}; }
__device__ __forceinline__ cpk csub(cpk x, cpk y) { return {f2sub(x.re, y.re), f2sub(x.im, y.im)}; }
__device__ __forceinline__ cpk cscale(cpk x, float s) { return {f2mul(x.re, f2dup(s)), f2mul(x.im, f2dup(s))}; }
template <int DIR>
__device__ __forceinline__ cpk rot90(cpk x) {
  return DIR < 0 ? cpk{x.im, f2neg(x.re)} : cpk{f2neg(x.im), x.re};
}
// x * w for a twiddle held as a pair with equal lanes (w.re = (c, c), w.im = (s, s))
__device__ __forceinline__ cpk cmul_b(cpk x, cpk w) {
  return {f2sub(f2mul(x.re, w.re), f2mul(x.im, w.im)), f2fma(x.re, w.im, f2mul(x.im, w.re))};
}
__device__ __forceinline__ cpk cmul(cpk x, float2 w) { return cmul_b(x, cpk{f2dup(w.x), f2dup(w.y)}); }
__device__ __forceinline__ cpk pack_pair(cpair p) {
  return {make_float2(p.a.x, p.b.x), make_float2(p.a.y, p.b.y)};
}
__device__ __forceinline__ cpair unpack_pair(cpk v) {
  return {make_float2(v.re.x, v.im.x), make_float2(v.re.y, v.im.y)};
}

// a + (DIR i) d and a - (DIR i) d
template <int DIR, class V>
__device__ __forceinline__ V add_rot(V a, V d) {
  return cadd(a, rot90<DIR>(d));
}
template <int DIR, class V>
__device__ __forceinline__ V sub_rot(V a, V d) {
  return csub(a, rot90<DIR>(d));
}
template <int DIR>
__device__ __forceinline__ cpk add_rot(cpk a, cpk d) {
  return DIR < 0 ? cpk{f2add(a.re, d.im), f2sub(a.im, d.re)} : cpk{f2sub(a.re, d.im), f2add(a.im, d.re)};
}
template <int DIR>
__device__ __forceinline__ cpk sub_rot(cpk a, cpk d) {
  return DIR < 0 ? cpk{f2sub(a.re, d.im), f2add(a.im, d.re)} : cpk{f2add(a.re, d.im), f2sub(a.im, d.re)};
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

// butterfly of a radix-R combine: lo = e + W_R^K o, hi = e - W_R^K o
template <int R, int K, int DIR, class V>
__device__ __forceinline__ void bfly(V& lo, V& hi, V e, V o) {
  const V t = twc<R, K, DIR>(o);
  lo = cadd(e, t);
  hi = csub(e, t);
}
// packed pairs: products with +-1 and +-i fold into the additions, and the (+-1 +-i) / sqrt 2
// products into two fused multiply-adds per component
template <int R, int K, int DIR>
__device__ __forceinline__ void bfly(cpk& lo, cpk& hi, cpk e, cpk o) {
  constexpr int k = (K * (32 / R)) & 31;
  if constexpr (k == 0) {
    lo = cadd(e, o);
    hi = csub(e, o);
  } else if constexpr (k == 8) {
    lo = add_rot<DIR>(e, o);
    hi = sub_rot<DIR>(e, o);
  } else if constexpr (k == 16) {
    lo = csub(e, o);
    hi = cadd(e, o);
  } else if constexpr (k == 24) {
    lo = add_rot<-DIR>(e, o);
    hi = sub_rot<-DIR>(e, o);
  } else if constexpr (k == 4 || k == 12 || k == 20 || k == 28) {
    // W o = h (c o.re - s o.im, c o.im + s o.re) with c, s = +-1: each component is one sum
    // or difference u, times +-h
    constexpr float h = 0.70710678118654752440f;
    constexpr int c = cos32(k) > 0 ? 1 : -1, sn = (sin32(k) > 0 ? 1 : -1) * DIR;
    const float2 u = c == sn ? (c > 0 ? f2sub(o.re, o.im) : f2sub(o.im, o.re)) : f2add(o.re, o.im);
    const float2 w = c == sn ? f2add(o.im, o.re) : (c > 0 ? f2sub(o.im, o.re) : f2sub(o.re, o.im));
    constexpr float hu = (c != sn && c < 0) ? -h : h, hw = (c == sn && c < 0) ? -h : h;
    lo = {f2fma(u, f2dup(hu), e.re), f2fma(w, f2dup(hw), e.im)};
    hi = {f2fma(u, f2dup(-hu), e.re), f2fma(w, f2dup(-hw), e.im)};
  } else {
    constexpr float c = (float)cos32(k), sn = (float)(DIR * sin32(k));
    const cpk t = {f2fma(o.re, f2dup(c), f2mul(o.im, f2dup(-sn))), f2fma(o.im, f2dup(c), f2mul(o.re, f2dup(sn)))};
    lo = cadd(e, t);
    hi = csub(e, t);
  }
}

// v0 - t / 2 (radix 3)
__device__ __forceinline__ float2 sub_half(float2 v0, float2 t) {
  return make_float2(v0.x - 0.5f * t.x, v0.y - 0.5f * t.y);
}
__device__ __forceinline__ cpair sub_half(cpair v0, cpair t) { return {sub_half(v0.a, t.a), sub_half(v0.b, t.b)}; }
__device__ __forceinline__ cpk sub_half(cpk v0, cpk t) {
  return {f2fma(t.re, f2dup(-0.5f), v0.re), f2fma(t.im, f2dup(-0.5f), v0.im)};
}

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
      bfly<R, K, DIR>(v[K], v[K + R / 2], e[K], o[K]);
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
    V t2 = cadd(v[1], v[3]), d = csub(v[1], v[3]);
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = add_rot<DIR>(t1, d);
    v[3] = sub_rot<DIR>(t1, d);
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

// The padded exchange layout that stage s writes: output o goes to slot o + (o / G) Pd
// with G = xgroup(s), Pd = xpad(s).  A later stage pads span(s) per group of span(s + 1),
// its butterflies' outputs.  A first stage of radix 2, 4 or 8 pads 1 per 16 outputs where
// one transform spans 16 threads or more: with 1 per radix, two lanes of each half-warp of
// the next stage's 8-byte loads (elements t + (N / R) r) share a bank pair, while the
// stores (R t + r + (R t + r) / 16) stay apart as well.  Narrower transforms share a warp,
// where the pitch between transforms decides, and keep 1 per radix.
template <class P>
__host__ __device__ constexpr int xgroup(int s) {
  return (s == 0 && P::T >= 16 && (P::R0 == 2 || P::R0 == 4 || P::R0 == 8)) ? 16 : P::span(s + 1);
}
template <class P>
__host__ __device__ constexpr int xpad(int s) {
  return P::span(s);
}

// shared-memory elements of one transform's padded exchange buffer: the largest layout
// of a stage whose outputs go through shared memory (every stage but the last)
template <class P>
__host__ __device__ constexpr int pad_elems_p() {
  int m = 0;
  for (int s = 0; P::radix(s + 1) != 0; ++s) {
    const int e = P::N + (P::N / xgroup<P>(s)) * xpad<P>(s);
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

// packed pairs: both lanes share the twiddles, so the powers are formed once, as pairs
// with equal lanes, and each product with a pair of values is five two-lane instructions
template <int N, int E, int R, int NS, int DIR>
__device__ __forceinline__ void stage_twiddle(cpk (&b)[E], int t, const float2* __restrict__ tw) {
  constexpr int T = N / E;
  constexpr int STEP = N / (NS * R);
#pragma unroll
  for (int u = 0; u < E / R; ++u) {
    const int j = t + u * T;
    const int k1 = (j % NS) * STEP;
    cpk pw[6];
    int np = 0;
    {
      const float2 w1 = __ldg(&tw[k1 % N]);
      cpk w = {f2dup(w1.x), f2dup(DIR < 0 ? w1.y : -w1.y)};
#pragma unroll
      for (int q = 1; q < R; q <<= 1) {
        pw[np++] = w;
        w = cmul_b(w, w);
      }
    }
#pragma unroll
    for (int r = 1; r < R; ++r) {
      cpk w;
      bool have = false;
#pragma unroll
      for (int q = 0; q < 6; ++q)
        if ((r >> q) & 1) {
          w = have ? cmul_b(w, pw[q]) : pw[q];
          have = true;
        }
      b[u * R + r] = cmul_b(b[u * R + r], w);
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

// write the outputs of a stage (radix R, NS) in the exchange layout (PAD: groups of G
// outputs, PD slots of padding after each)
template <int N, int E, int R, int NS, bool PAD, int STRIDE, int G, int PD, class V>
__device__ __forceinline__ void stage_store(const V (&b)[E], V* sm, int t) {
  constexpr int T = N / E;
  // the butterfly's R outputs (base + r NS) lie in one group: G = NS R, or NS = 1 with R
  // dividing G
  static_assert(!PAD || G == NS * R || (NS == 1 && G % R == 0), "exchange groups");
#pragma unroll
  for (int u = 0; u < E / R; ++u) {
    const int j = t + u * T;
    const int o = (j / NS) * NS * R + (j % NS);
    const int base = PAD ? o + (o / G) * PD : o;
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
// stages S >= 1 of plan P: inputs from the layout of stage S - 1 (groups of xgroup(S - 1),
// padding xpad(S - 1)), twiddles, radix-R DFT; then the next stage through shared memory,
// or, after the last stage, the outputs into v
template <class P, int DIR, bool PAD, int STRIDE, bool TAIL, int S, class Sync, class V>
__device__ __forceinline__ void fft_stages(V (&v)[P::E], V (&b)[P::E], V* sm, int t, const float2* __restrict__ tw,
                                           const Sync& sync) {
  constexpr int N = P::N, E = P::E, R = P::radix(S), NS = P::span(S);
  constexpr bool LAST = P::radix(S + 1) == 0;
  stage_load<N, E, R, xgroup<P>(S - 1), xpad<P>(S - 1), PAD, STRIDE>(b, sm, t);
  if (TAIL || !LAST) sync();
  stage_tw<N, E, R, NS, DIR>(b, t, tw);
  stage_dft<N, E, R, DIR>(b);
  if constexpr (LAST) {
#pragma unroll
    for (int u = 0; u < E / R; ++u)
#pragma unroll
      for (int r = 0; r < R; ++r) v[u + r * (E / R)] = b[u * R + r];
  } else {
    stage_store<N, E, R, NS, PAD, STRIDE, xgroup<P>(S), xpad<P>(S)>(b, sm, t);
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
  stage_store<N, E, R0, 1, PAD, STRIDE, xgroup<P>(0), xpad<P>(0)>(b, sm, t);
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
