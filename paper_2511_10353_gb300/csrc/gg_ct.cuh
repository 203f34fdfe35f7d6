// Compile-time FFT codelets for the grid sizes of the named workloads.
//
// The run-time kernels in gg_kernels.cuh take N, the radix schedule and the
// tile width as parameters; every shared-memory access then needs its own
// index arithmetic. Here N, the tile width and the schedule are template
// constants: stage radices, spans, twiddle steps and butterfly positions fold
// into immediate offsets, and the stage loop unrolls. The data flow is the
// same as the run-time kernels' (same passes, same tiles, same rounding of
// the FP64-generated tables).
#pragma once

#include <cuda.h>

#include "gg_device.cuh"

namespace gg {
namespace ct {

// ------------------------------------------------------------ schedules
// A schedule is named by a key: the transform length n, plus kBig for the
// FP32 codelets. Those take a few large radices where a thread can hold a
// whole butterfly (n = 256: 16 x 16; n = 512: 32 x 16): each radix is one
// DFT in registers (constant twiddles inside it), so a transform makes one
// shared-memory round trip and one twiddle stage instead of two or three of
// each. Other lengths, and every FP64 codelet (whose bound is the FP64
// pipe, not the stage count), use radix 8 first, then 4 or 2, then the 3s.
constexpr int kBig = 1 << 20;
template <typename R> __host__ __device__ constexpr int skey(int n) {
  return sizeof(R) == 4 ? (n | kBig) : n;
}
__host__ __device__ constexpr int key_n(int key) { return key & (kBig - 1); }

struct Fac {
  int a, b;  // n = 2^a 3^b
};
__host__ __device__ constexpr Fac factor(int n) {
  Fac f{0, 0};
  while (n % 2 == 0) { n /= 2; ++f.a; }
  while (n % 3 == 0) { n /= 3; ++f.b; }
  return f;
}
// large-radix forward schedules of the FP32 codelets (0: none at this n / stage)
__host__ __device__ constexpr int big_radix(int n, int s) {
  switch (n) {
    case 256: return s < 2 ? 16 : 0;
    case 512: return s == 0 ? 32 : (s == 1 ? 16 : 0);
    case 768: return s < 2 ? 8 : (s == 2 ? 12 : 0);
    case 1536: return s < 2 ? 8 : (s == 2 ? 24 : 0);
    default: return 0;
  }
}
__host__ __device__ constexpr bool is_big(int key) {
  return (key & kBig) != 0 && big_radix(key_n(key), 0) != 0;
}
__host__ __device__ constexpr int nstages(int key) {
  if (is_big(key)) {
    int c = 0;
    while (big_radix(key_n(key), c)) ++c;
    return c;
  }
  const Fac f = factor(key_n(key));
  return f.a / 3 + (f.a % 3 ? 1 : 0) + f.b;
}
// forward schedule: radix 8 first, then 4 or 2, then the 3s (or the large radices)
__host__ __device__ constexpr int radix_fwd(int key, int s) {
  if (is_big(key)) return big_radix(key_n(key), s);
  const Fac f = factor(key_n(key));
  const int n8 = f.a / 3;
  if (s < n8) return 8;
  s -= n8;
  if (f.a % 3) {
    if (s == 0) return f.a % 3 == 2 ? 4 : 2;
    s -= 1;
  }
  return 3;
}
// the inverse transforms use the same radices in reverse order, so that the
// first inverse stage has the radix of the last forward stage
__host__ __device__ constexpr int radix_of(int key, int s, bool inv) {
  return inv ? radix_fwd(key, nstages(key) - 1 - s) : radix_fwd(key, s);
}
__host__ __device__ constexpr int ns_of(int key, int s, bool inv) {
  int p = 1;
  for (int i = 0; i < s; ++i) p *= radix_of(key, i, inv);
  return p;
}
__host__ __device__ constexpr int gcd_c(int a, int b) { return b ? gcd_c(b, a % b) : a; }
// elements per thread: the least common multiple of the radices
__host__ __device__ constexpr int elems(int key) {
  int e = 1;
  for (int s = 0; s < nstages(key); ++s) {
    const int r = radix_fwd(key, s);
    e = e / gcd_c(e, r) * r;
  }
  return e;
}

// ------------------------------------------------ in-register DFTs of composite length
// cos and sin of 2 pi m / r in FP64 at compile time: exact reduction to a
// quadrant, then the Taylor series on [0, pi/2) (terms to x^29: error below
// 1e-20), then the quadrant's exact rotation.
__host__ __device__ constexpr double taylor_cos(double x) {
  double t = 1.0, s = 1.0;
  for (int i = 1; i < 15; ++i) {
    t *= -x * x / ((2.0 * i - 1.0) * (2.0 * i));
    s += t;
  }
  return s;
}
__host__ __device__ constexpr double taylor_sin(double x) {
  double t = x, s = x;
  for (int i = 1; i < 15; ++i) {
    t *= -x * x / ((2.0 * i) * (2.0 * i + 1.0));
    s += t;
  }
  return s;
}
__host__ __device__ constexpr double cos_turn(int m, int r) {
  m = ((m % r) + r) % r;
  const int q = 4 * m / r, rem = 4 * m - q * r;  // angle = (q + rem / r) pi / 2
  const double x = 1.57079632679489661923132169163975 * (double)rem / (double)r;
  const double c = taylor_cos(x), s = taylor_sin(x);
  return q == 0 ? c : (q == 1 ? -s : (q == 2 ? -c : s));
}
__host__ __device__ constexpr double sin_turn(int m, int r) {
  m = ((m % r) + r) % r;
  const int q = 4 * m / r, rem = 4 * m - q * r;
  const double x = 1.57079632679489661923132169163975 * (double)rem / (double)r;
  const double c = taylor_cos(x), s = taylor_sin(x);
  return q == 0 ? s : (q == 1 ? c : (q == 2 ? -s : -c));
}

template <int I, int END, class F> __device__ __forceinline__ void static_for(const F &f) {
  if constexpr (I < END) {
    f(IntC<I>{});
    static_for<I + 1, END>(f);
  }
}

// a * w^E with w = exp(-2 pi i / RT) (forward) or its conjugate (INV), E a
// compile-time exponent: no arithmetic for w^E = 1, a swap for +-i, a sign
// for -1, two adds and two multiplies for the odd eighths, else a complex
// product with the FP64-computed constant rounded once.
template <int RT, int EXP, bool INV, typename T> __device__ __forceinline__ T tw_const(T a) {
  using R = decltype(a.x);
  constexpr int e = ((EXP % RT) + RT) % RT;
  if constexpr (e == 0) {
    return a;
  } else if constexpr (2 * e == RT) {
    return T{-a.x, -a.y};
  } else if constexpr (4 * e == RT) {
    return mul_wi<INV>(a);  // -i forward
  } else if constexpr (4 * e == 3 * RT) {
    return mul_wi<!INV>(a);  // +i forward
  } else if constexpr ((8 * e) % RT == 0) {  // (+-1 +- i) / sqrt 2
    constexpr R h = (R)0.70710678118654752440;
    constexpr int o = 8 * e / RT;  // 1, 3, 5, 7
    constexpr R c = (o == 1 || o == 7) ? h : -h;
    constexpr R sn = (o == 1 || o == 3) ? -h : h;  // imaginary part of w^e (forward)
    constexpr R si = INV ? -sn : sn;
    // a * (c + i si) with |c| = |si| = h: h * (+-a.x -+ a.y, ...)
    if constexpr (c > 0 && si < 0) return T{h * (a.x + a.y), h * (a.y - a.x)};
    else if constexpr (c > 0 && si > 0) return T{h * (a.x - a.y), h * (a.y + a.x)};
    else if constexpr (c < 0 && si < 0) return T{-h * (a.x - a.y), -h * (a.y + a.x)};
    else return T{-h * (a.x + a.y), h * (a.x - a.y)};
  } else {
    constexpr R c = (R)cos_turn(e, RT);
    constexpr R sn = (R)(INV ? sin_turn(e, RT) : -sin_turn(e, RT));
    return T{a.x * c - a.y * sn, a.x * sn + a.y * c};
  }
}

}  // namespace ct

// DFT of length R1 * R2 on registers in natural order (input n, output k):
// n = R2 n1 + n2, k = k1 + R1 k2; a length-R1 DFT over n1 for each n2, the
// twiddle w_R^(n2 k1), then a length-R2 DFT over n2 for each k1.
template <int R1, int R2, bool INV, typename T> struct ComposedDft {
  static __device__ __forceinline__ void run(T *v) {
    constexpr int RT = R1 * R2;
    T t[RT];
    ct::static_for<0, R2>([&](auto n2c) {
      constexpr int n2 = decltype(n2c)::value;
      T u[R1];
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) u[n1] = v[R2 * n1 + n2];
      Butterfly<R1, INV, T>::run(u);
      ct::static_for<0, R1>([&](auto k1c) {
        constexpr int k1 = decltype(k1c)::value;
        t[n2 * R1 + k1] = ct::tw_const<RT, n2 * k1, INV>(u[k1]);
      });
    });
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      T u[R2];
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) u[n2] = t[n2 * R1 + k1];
      Butterfly<R2, INV, T>::run(u);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) v[k1 + R1 * k2] = u[k2];
    }
  }
};
template <bool INV, typename T> struct Butterfly<6, INV, T> : ComposedDft<2, 3, INV, T> {};
template <bool INV, typename T> struct Butterfly<12, INV, T> : ComposedDft<4, 3, INV, T> {};
template <bool INV, typename T> struct Butterfly<16, INV, T> : ComposedDft<4, 4, INV, T> {};
template <bool INV, typename T> struct Butterfly<24, INV, T> : ComposedDft<8, 3, INV, T> {};
template <bool INV, typename T> struct Butterfly<32, INV, T> : ComposedDft<8, 4, INV, T> {};
template <bool INV, typename T> struct Butterfly<48, INV, T> : ComposedDft<16, 3, INV, T> {};

namespace ct {

// k = j mod NS for j = p + P*b, 0 <= p < P, 0 <= b < NB, folded at compile time
template <int NS, int P, int NB>
__device__ __forceinline__ int k_of(int p, int b) {
  if constexpr (NS == 1) {
    return 0;
  } else if constexpr (P % NS == 0) {
    return p % NS;
  } else if constexpr (P * NB <= NS) {
    return p + P * b;  // j < NS
  } else {
    return (p + P * b) % NS;
  }
}

// A twiddle table: in shared memory (SM: the strided passes of the
// large-radix schedules copy it there) or in global memory, read through the
// non-coherent cache.
template <typename T, bool SM> struct Tw {
  const T *p;
  __device__ __forceinline__ T operator[](int i) const {
    if constexpr (SM) return p[i];
    else return __ldg(p + i);
  }
};
template <typename T> __device__ __forceinline__ Tw<T, false> tw_global(const void *p) {
  return Tw<T, false>{reinterpret_cast<const T *>(p)};
}

// Twiddles of a stage with NS > 1: FP32 radices up to 8 load w^1 per
// butterfly (before the stage's shared-memory reads, to overlap their
// latency) and form the other powers by at most three products; FP64, and
// the large FP32 radices, read every power w^(k r) from the table (an FP32
// power chain over 15 or 31 steps would lose accuracy).
template <typename R, int RAD> __host__ __device__ constexpr bool powers_from_w1() {
  return sizeof(R) == 4 && (RAD == 2 || RAD == 3 || RAD == 4 || RAD == 8);
}
template <typename R, int RAD, bool INV, int TSTEP, class TwT>
__device__ __forceinline__ void stage_twiddles(Cx<R> *v, int k, Cx<R> w1, const TwT &tw) {
  if constexpr (powers_from_w1<R, RAD>()) {
    twiddle_powers<RAD, INV>(v, w1);
  } else {
#pragma unroll
    for (int r = 1; r < RAD; ++r) {
      const Cx<R> w = tw[k * TSTEP * r];
      v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
    }
  }
}

// Barrier of an in-place stage: none (the stage writes elsewhere), the whole
// CTA, or the warp (when every transform lies within one warp).
// kSyncCtaAsync: CTA barriers, the one after the stage's stores preceded by
// a proxy fence (the stage's output is then read by a TMA store)
enum Sync : int { kSyncNone = 0, kSyncCta = 1, kSyncWarp = 2, kSyncCtaAsync = 3 };
// OR-ed into a stage's SY: no thread-index range hint (the z inverse measured
// faster without it, 0.264 against 0.259 ms at 512^3)
constexpr int kNoRangeHint = 16;
template <int SY, bool AFTER_STORES = false> __device__ __forceinline__ void stage_barrier() {
  if constexpr (SY == kSyncCtaAsync && AFTER_STORES) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
  } else if constexpr (SY == kSyncCta || SY == kSyncCtaAsync) {
    __syncthreads();
  } else if constexpr (SY == kSyncWarp) {
    __syncwarp();
  }
}

// One Stockham stage of a length-N transform, stage index SI of the forward
// (INV = false) or inverse schedule, for the butterflies j = p + P*b of this
// thread. ld(n) reads element n of the stage input, st(n, v) writes element n
// of its output; with a barrier (SY) the stage runs in place in shared memory.
template <typename R, int N, int E, int SI, bool INV, int SY, class Ld, class St, class TwT>
__device__ __forceinline__ void stage(int p, const TwT &tw, const Ld &ld,
                                      const St &st) {
  constexpr int K = skey<R>(N);
  constexpr int RAD = radix_of(K, SI, INV);
  constexpr int NS = ns_of(K, SI, INV);
  constexpr int P = N / E, NB = E / RAD, SPAN = N / RAD, TSTEP = N / (NS * RAD);
  asm volatile("" : "+r"(p));
  if constexpr (!(SY & kNoRangeHint)) __builtin_assume(p >= 0 && p < P);
  Cx<R> w1[NB];
  if constexpr (NS > 1 && powers_from_w1<R, RAD>()) {
#pragma unroll
    for (int b = 0; b < NB; ++b) w1[b] = tw[k_of<NS, P, NB>(p, b) * TSTEP];
  }
  Cx<R> v[E];
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int r = 0; r < RAD; ++r) v[b * RAD + r] = ld(p + P * b + r * SPAN);
  stage_barrier<SY & 15>();
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    if constexpr (NS > 1)
      stage_twiddles<R, RAD, INV, TSTEP>(&v[b * RAD], k_of<NS, P, NB>(p, b), w1[b], tw);
    Butterfly<RAD, INV, Cx<R>>::run(&v[b * RAD]);
  }
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int k = k_of<NS, P, NB>(p, b);
    const int base = (p + P * b - k) * RAD + k;
#pragma unroll
    for (int r = 0; r < RAD; ++r) st(base + r * NS, v[b * RAD + r]);
  }
  stage_barrier<SY & 15, true>();
}

// Stages FIRST .. LAST-1 in place in shared memory, barrier SY.
template <typename R, int N, int E, bool INV, int FIRST, int LAST, int SY = kSyncCta, class Ld,
          class St, class TwT>
__device__ __forceinline__ void stages(int p, const TwT &tw, const Ld &ld,
                                       const St &st) {
  if constexpr (FIRST < LAST) {
    stage<R, N, E, FIRST, INV, SY>(p, tw, ld, st);
    stages<R, N, E, INV, FIRST + 1, LAST, SY>(p, tw, ld, st);
  }
}

// Stages FIRST .. LAST-1 alternating between two shared buffers (FIRST reads
// A and writes B, the next reads B and writes A, ...): one CTA barrier per
// stage instead of two. The caller leaves B free; an even count ends in A.
template <typename R, int N, int E, bool INV, int FIRST, int LAST, class LdA, class StA, class LdB,
          class StB, class TwT>
__device__ __forceinline__ void stages_pingpong(int p, const TwT &tw, const LdA &lda,
                                                const StA &sta, const LdB &ldb, const StB &stb) {
  if constexpr (FIRST < LAST) {
    stage<R, N, E, FIRST, INV, kSyncNone>(p, tw, lda, stb);
    __syncthreads();
    stages_pingpong<R, N, E, INV, FIRST + 1, LAST>(p, tw, ldb, stb, lda, sta);
  }
}

// The last stage of a schedule, outputs kept in registers: on return v holds
// element j + r*N/RAD at v[b*RAD + r] (j = p + P*b).
template <typename R, int N, int E, bool INV, bool HINT = true, class Ld, class TwT>
__device__ __forceinline__ void last_stage_regs(int p, const TwT &tw, const Ld &ld,
                                                Cx<R> *v) {
  constexpr int K = skey<R>(N);
  constexpr int S = nstages(K);
  constexpr int RAD = radix_of(K, S - 1, INV);
  constexpr int NS = ns_of(K, S - 1, INV);
  constexpr int P = N / E, NB = E / RAD, SPAN = N / RAD, TSTEP = N / (NS * RAD);
  static_assert(NS * RAD == N, "last stage");
  asm volatile("" : "+r"(p));
  if constexpr (HINT) __builtin_assume(p >= 0 && p < P);
  Cx<R> w1[NB];
  if constexpr (NS > 1 && powers_from_w1<R, RAD>()) {
#pragma unroll
    for (int b = 0; b < NB; ++b) w1[b] = tw[k_of<NS, P, NB>(p, b) * TSTEP];
  }
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int r = 0; r < RAD; ++r) v[b * RAD + r] = ld(p + P * b + r * SPAN);
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    if constexpr (NS > 1)
      stage_twiddles<R, RAD, INV, TSTEP>(&v[b * RAD], k_of<NS, P, NB>(p, b), w1[b], tw);
    Butterfly<RAD, INV, Cx<R>>::run(&v[b * RAD]);
  }
}

// ------------------------------------------------------------ register pairs
// A thread holds E elements: p + P*b + r*SPAN. Where E is a multiple of
// RA*RB for the last two radices of the forward schedule (the first two of
// the inverse), the thread's elements hold whole butterflies of both stages,
// so the pair runs in registers without a shared-memory round trip between
// them. Same twiddles, butterflies and order of operations as the two
// separate stages.
template <typename R, int N, int E> __host__ __device__ constexpr bool fuse_pair() {
  constexpr int K = skey<R>(N);
  return nstages(K) >= 3 && E % (radix_fwd(K, nstages(K) - 2) * radix_fwd(K, nstages(K) - 1)) == 0;
}

// Twiddles w^(k r), r = 1 .. RAD-1, on one butterfly's inputs; kt = k*TSTEP.
template <typename R, int RAD, bool INV, class TwT>
__device__ __forceinline__ void stage_twiddle(Cx<R> *v, const TwT &tw, int kt) {
  if constexpr (sizeof(R) == 4) {
    twiddle_powers<RAD, INV>(v, tw[kt]);
  } else {
#pragma unroll
    for (int r = 1; r < RAD; ++r) {
      const Cx<R> w = tw[kt * r];
      v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
    }
  }
}

// The forward schedule's last two stages (A, B), outputs in registers with
// the contract of last_stage_regs. Stage A's butterflies of this thread are
// j = p + P*b, b = g + G*q (k = p + P*g, q < RB); their outputs are the inputs
// of stage B's butterflies j' = p + P*(g + G*r), input q.
template <typename R, int N, int E, class Ld, class TwT>
__device__ __forceinline__ void last_two_stages_regs(int p, const TwT &tw,
                                                     const Ld &ld, Cx<R> *v) {
  constexpr int K = skey<R>(N);
  constexpr int S = nstages(K);
  constexpr int RA = radix_of(K, S - 2, false), RB = radix_of(K, S - 1, false);
  constexpr int NSA = ns_of(K, S - 2, false);
  constexpr int P = N / E, G = E / (RA * RB), NBA = E / RA, NBB = E / RB;
  constexpr int SPANA = N / RA, TSA = N / (NSA * RA);
  static_assert(NSA == P * G && NSA * RA * RB == N, "register pair");
  asm volatile("" : "+r"(p));
  __builtin_assume(p >= 0 && p < P);
  Cx<R> w1[NBA];
  if constexpr (sizeof(R) == 4) {
#pragma unroll
    for (int b = 0; b < NBA; ++b) w1[b] = tw[k_of<NSA, P, NBA>(p, b) * TSA];
  }
  Cx<R> a[E];
#pragma unroll
  for (int b = 0; b < NBA; ++b)
#pragma unroll
    for (int r = 0; r < RA; ++r) a[b * RA + r] = ld(p + P * b + r * SPANA);
#pragma unroll
  for (int b = 0; b < NBA; ++b) {
    if constexpr (NSA > 1) {
      if constexpr (sizeof(R) == 4) twiddle_powers<RA, false>(&a[b * RA], w1[b]);
      else stage_twiddle<R, RA, false>(&a[b * RA], tw, k_of<NSA, P, NBA>(p, b) * TSA);
    }
    Butterfly<RA, false, Cx<R>>::run(&a[b * RA]);
  }
#pragma unroll
  for (int g = 0; g < G; ++g)
#pragma unroll
    for (int q = 0; q < RB; ++q)
#pragma unroll
      for (int r = 0; r < RA; ++r) v[(g + G * r) * RB + q] = a[(g + G * q) * RA + r];
  // stage B: NS = N / RB, every j' < NS, so k = j' and TSTEP = 1
#pragma unroll
  for (int b = 0; b < NBB; ++b) {
    stage_twiddle<R, RB, false>(&v[b * RB], tw, p + P * b);
    Butterfly<RB, false, Cx<R>>::run(&v[b * RB]);
  }
}

// The inverse schedule's first two stages (A: NS = 1, B: NS = RA) on
// registers holding the hand-off layout (element p + P*b + r*N/RA at
// v[b*RA + r]). Stage A's butterfly b = g + G*q feeds input q of stage B's
// butterfly (g, r) = j' = p*RA + P*RA*g + r, whose k = r is known at compile
// time. On return v[(g*RA + r)*RB + s] holds stage B's output s of butterfly
// (g, r); inverse_head_store writes them.
template <typename R, int N, int E, class TwT>
__device__ __forceinline__ void inverse_head_regs(const TwT &tw, Cx<R> *v) {
  constexpr int RA = radix_of(skey<R>(N), 0, true), RB = radix_of(skey<R>(N), 1, true);
  constexpr int P = N / E, G = E / (RA * RB), NBA = E / RA;
  constexpr int TSB = N / (RA * RB);
#pragma unroll
  for (int b = 0; b < NBA; ++b) Butterfly<RA, true, Cx<R>>::run(&v[b * RA]);
  Cx<R> u[E];
#pragma unroll
  for (int g = 0; g < G; ++g)
#pragma unroll
    for (int r = 0; r < RA; ++r)
#pragma unroll
      for (int q = 0; q < RB; ++q) u[(g * RA + r) * RB + q] = v[(g + G * q) * RA + r];
#pragma unroll
  for (int g = 0; g < G; ++g)
#pragma unroll
    for (int r = 0; r < RA; ++r) {
      if (r > 0) stage_twiddle<R, RB, true>(&u[(g * RA + r) * RB], tw, r * TSB);
      Butterfly<RB, true, Cx<R>>::run(&u[(g * RA + r) * RB]);
    }
#pragma unroll
  for (int i = 0; i < E; ++i) v[i] = u[i];
  (void)P;
}
// Stage B's outputs: element s of butterfly j' goes to (j' - k)*RB + k + s*RA.
template <typename R, int N, int E, class St>
__device__ __forceinline__ void inverse_head_store(int p, const Cx<R> *v, const St &st) {
  constexpr int RA = radix_of(skey<R>(N), 0, true), RB = radix_of(skey<R>(N), 1, true);
  constexpr int P = N / E, G = E / (RA * RB);
#pragma unroll
  for (int g = 0; g < G; ++g)
#pragma unroll
    for (int r = 0; r < RA; ++r)
#pragma unroll
      for (int s = 0; s < RB; ++s)
        st(p * RA * RB + P * RA * RB * g + r + s * RA, v[(g * RA + r) * RB + s]);
}

// ------------------------------------------------------------ tile policy
// Tile variants the autotuner chooses between (V = 0, 1, 2 for the strided
// pass; V = 0 .. 3 for the z passes). An invalid variant for a size falls
// back to variant 0's shape.
//
// Strided pass, variant
//   0: E = lcm of the radices, rows of up to 128 bytes, <= 512 threads
//   1: E doubled (two butterflies per thread and stage), rows of up to 128 bytes
//   2: E doubled where it fits, rows halved (a smaller CTA: several share an
//      SM, or two outputs fit the register budget)
// Whether the handed-off spectrum may stay in registers while an inverse
// runs is estimated from the register budget; otherwise (SPILL) it is parked
// in shared memory and every output reads it from there.
// Tile variant of the persistent batched kernel (gg_persist.cu): exactly 256
// threads per CTA for every pass and size, two CTAs per SM.
constexpr int kPersistV = 4;

template <typename R, int N, int V> struct AxisPolicy {
  static constexpr int CB = 2 * (int)sizeof(R);
  static constexpr bool BIG = is_big(skey<R>(N));
  static constexpr int E0 = elems(skey<R>(N));
  static constexpr bool DOUBLE_OK = N % (2 * E0) == 0 && 2 * E0 * ((int)sizeof(R) / 4) <= 16;
  static constexpr int E = ((V == 1 || V == 2) && DOUBLE_OK) ? 2 * E0 : E0;
  static constexpr int P = N / E;
  // large-radix schedules (E cannot double): variant 1 is the small tile of
  // variant 2 with the handed-off spectrum parked in shared memory, so that
  // three CTAs' registers fit an SM
  static constexpr bool SMALL = V == 2 || (BIG && V == 1);
  static constexpr int pick() {
    if (V == kPersistV) return 256 / P;  // the persistent batched kernel: 256 threads
    int b = 128 / CB;
    while (b > 1 && ((N / 2) % b != 0 || P * b > 512 || 2 * (N * b * CB) > 200 * 1024)) b /= 2;
    if (SMALL && b * CB > 32) b /= 2;
    return b;
  }
  static constexpr int B = pick();
  static constexpr int THREADS = P * B;
  // variant 2 (small CTAs): register bound for two CTAs per SM where the
  // shared memory of two tiles lets two fit (the FP32 filter table of the x
  // pass may still keep that pass at one); variant 1 of the large radices:
  // as many CTAs as the tiles' shared memory allows, up to three
  static constexpr int SMEM_EST = 128 + 2 * N * B * CB;
  // variant 2 of the FP32 large radices from N = 512, where the two tiles
  // and the largest filter table of three CTAs fit an SM: three CTAs with
  // the spectrum in registers (the outputs leave by TMA from the tile buffer
  // itself, the twiddles stay in global memory). 512^3 x pass 0.454 ->
  // 0.421 ms; at N = 256 the two-CTA staging-tile form stays (the batched
  // workload measured 17.0 against 17.4 ms with three CTAs there too)
  static constexpr bool THREE = V == 2 && BIG && sizeof(R) == 4 && N >= 512 &&
                                3 * (SMEM_EST + 4 * kInterpExact + 16 * kMaxInterpCells(N) + 1024) <=
                                    228 * 1024;
  static constexpr int min_blocks() {
    if (V == kPersistV) return 2;
    if (THREE) return 3;
    if (BIG && V == 1) {  // the x pass's filter table (about 11 KB) may still cost one
      const int by_smem = (228 * 1024) / (SMEM_EST + 1024);
      return by_smem < 1 ? 1 : (by_smem > 3 ? 3 : by_smem);
    }
    return (V == 2 && THREADS <= 256 && 2 * SMEM_EST <= 227 * 1024) ? 2 : 1;
  }
  static constexpr int MINB = min_blocks();
  static constexpr int REG_BUDGET =
      65536 / (THREADS * MINB) < 255 ? 65536 / (THREADS * MINB) : 255;
  static constexpr int REG_NEED = 4 * E * ((int)sizeof(R) / 4) + 48;
  static constexpr bool SPILL = (BIG && V == 1) || (!THREE && REG_NEED > REG_BUDGET);
  static constexpr int ROWS_BOX = N <= 256 ? N : (N % 256 == 0 ? 256 : (N % 192 == 0 ? 192 : 128));
  static_assert(V != kPersistV || (THREADS == 256 && (N / 2) % B == 0), "persistent tile");
  // the large radices read their stage twiddles from a shared-memory copy
  // where it fits beside the tiles and the largest filter table
  static constexpr bool TW_SMEM = BIG && sizeof(R) == 4 && V != kPersistV && !THREE &&
                                  SMEM_EST + N * CB + 4 * kInterpExact + 16 * kMaxInterpCells(N) <= 227 * 1024;
  // The inverse outputs leave through a third (staging) tile and TMA stores
  // instead of per-thread global stores, where that tile fits beside the two
  // tiles, the twiddles and (filter: the x pass) the largest FP32 filter
  // table for MINB CTAs per SM. Not with the spectrum parked in shared
  // memory, nor in the persistent batched kernel.
  __host__ __device__ static constexpr bool tma_st(bool filter) {
    const int per_cta = SMEM_EST + N * B * CB + (TW_SMEM ? N * CB : 0) +
                        (filter ? 4 * kInterpExact + 16 * kMaxInterpCells(N) : 0) + 1024;
    return !SPILL && !THREE && V != kPersistV && nstages(skey<R>(N)) > 1 && MINB * per_cta <= 228 * 1024;
  }
};

// z passes: lines per tile, variant 0 ~256 threads (sized so that two dense
// tiles and a padded tile fit in 160 KB), variant 1 half as many lines,
// variant 2 the lines of variant 0 with warp instead of CTA barriers between
// the stages (where each line lies within one warp; warps then drift apart),
// variant 3 the lines of variant 1 with warp barriers.
template <typename R, int N, int V> struct ZPolicy {
  static constexpr int M = N / 2;
  static constexpr int E = elems(skey<R>(M));
  static constexpr int P = M / E;
  static constexpr int CB = 2 * (int)sizeof(R);
  static constexpr int LD = M + (M >> 4) + 1;  // tile sizing (the widest padding)
  // the forward's last two and the inverse's first two stages in registers
  static constexpr bool FUSE = fuse_pair<R, M, E>();
  // Padding of the work tile, per direction: one empty slot every PAD values
  // (0: none). Chosen by counting the shared-memory wavefronts of every
  // stage's stores and loads for each size; FP32 (FP64 keeps 1 in 16).
  static constexpr int pad_of(bool inv) {
    if (sizeof(R) != 4) return 16;
    if (inv && FUSE) {             // register pair first: its stores are 12-24 apart
      if (M == 768) return 32;         // 248 wavefronts a line instead of 360 unpadded
      if (M == 192 || M == 96) return 64;
    }
    if (M == 96) return 32;           // N = 192: 1.2x / 1.5x the minimum instead of 2x
    if (inv && M == 768) return 32;   // N = 1536 inverse (8 x 8 x 12, first stage in registers): 1.5x instead of 2x
    return 16;
  }
  static constexpr int PAD_INV = pad_of(true), PAD_FWD = pad_of(false);
  static constexpr int LD_INV = M + (PAD_INV ? M / PAD_INV : 0) + 1;
  static constexpr int LD_FWD = M + (PAD_FWD ? M / PAD_FWD : 0) + 1;
  static constexpr int pick() {
    if (V == kPersistV) return 256 / P;  // the persistent batched kernel: 256 threads
    int l = 1;
    while (l < 64 && P * l * 2 <= 256 && (2 * (2 * l) * M + 2 * l * LD) * CB <= 160 * 1024) l *= 2;
    if ((V == 1 || V == 3) && l > 1) l /= 2;
    return l;
  }
  static constexpr int L = pick();
  static constexpr int THREADS = P * L;
  // variant 2, and every line within one warp (P divides 32): the stages need
  // only warp barriers
  static constexpr int SY = ((V == 2 || V == 3) && P <= 32 && 32 % P == 0) ? kSyncWarp : kSyncCta;
  static constexpr int DENSE = L * M;        // complex values of one dense tile
  static constexpr int WORK_INV = L * LD_INV;  // complex values of the padded tiles
  static constexpr int WORK_FWD = L * LD_FWD;
  // CTAs per SM the register allocation must leave room for: enough for 16
  // warps, as far as the shared memory of the pass allows (inverse: a dense
  // staging tile and the padded tile; forward: the padded tile). FP64 lines
  // need twice the registers and run at the FP64 rate: no bound there.
  static constexpr int min_blocks(int smem) {
    if (V == kPersistV) return 2;
    const int by_smem = (228 * 1024) / smem, by_warps = 512 / THREADS;
    const int m = by_smem < by_warps ? by_smem : by_warps;
    return sizeof(R) == 4 && m > 0 ? m : 1;
  }
  static constexpr int MINB_INV = min_blocks(128 + DENSE * CB + WORK_INV * CB);
  static constexpr int MINB_FWD = min_blocks(WORK_FWD * CB);
};

}  // namespace ct
}  // namespace gg
