// Device building blocks of the sm_103a path: complex arithmetic, the
// Philox4x32-10 generator, the Box-Muller map, radix-2/3/4/8 butterflies and
// one Stockham stage of an in-CTA FFT held in shared memory.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gg_internal.h"

namespace gg {

template <typename R> struct CxOf;
template <> struct CxOf<float> { using T = float2; };
template <> struct CxOf<double> { using T = double2; };
template <typename R> using Cx = typename CxOf<R>::T;

template <typename T> __device__ __forceinline__ T cadd(T a, T b) { return {a.x + b.x, a.y + b.y}; }
template <typename T> __device__ __forceinline__ T csub(T a, T b) { return {a.x - b.x, a.y - b.y}; }
template <typename T> __device__ __forceinline__ T cmul(T a, T b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// a * conj(b)
template <typename T> __device__ __forceinline__ T cmulc(T a, T b) {
  return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
template <typename T> __device__ __forceinline__ T cconj(T a) { return {a.x, -a.y}; }
// a * (-i) and a * (+i)
template <typename T> __device__ __forceinline__ T mul_mi(T a) { return {a.y, -a.x}; }
template <typename T> __device__ __forceinline__ T mul_pi(T a) { return {-a.y, a.x}; }
// a * (-i) for the forward transform, a * (+i) for the inverse
template <bool INV, typename T> __device__ __forceinline__ T mul_wi(T a) {
  return INV ? mul_pi(a) : mul_mi(a);
}

template <typename T> __device__ __forceinline__ T ldg_c(const T *p) { return __ldg(p); }

template <int V> struct IntC { static constexpr int value = V; };

// ---------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3"
// (SC'11): ten rounds of the 4x32 Philox S-box/P-box with a Weyl key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return make_uint4(c0, c1, c2, c3);
}

// The four Philox words of the group holding cell `idx` (group = idx >> 2).
__device__ __forceinline__ uint4 noise_words(uint64_t seed, uint64_t group) {
  return philox4x32_10((uint32_t)group, (uint32_t)(group >> 32), 0u, 0u, (uint32_t)seed,
                       (uint32_t)(seed >> 32));
}
// The same for a group index below 2^32 (every group of a grid of N <= 2048
// points per axis): the counter's high word is a compile-time zero, which
// removes a wide multiply from each of the first two rounds. Same words.
__device__ __forceinline__ uint4 noise_words32(uint64_t seed, uint32_t group) {
  return philox4x32_10(group, 0u, 0u, 0u, (uint32_t)seed, (uint32_t)(seed >> 32));
}

// Two-output Box-Muller (Box & Muller 1958) on one word pair (r_a, r_b):
// u_a = (r_a + 1) 2^-32 in (0, 1], u_b = r_b 2^-32; rho = sqrt(-2 ln u_a);
// outputs rho cos(2 pi u_b), rho sin(2 pi u_b). gauss4 applies it to the
// pairs (r0, r1) and (r2, r3) of a group.
//
// FP32 form, built from the integer words so that each step keeps FP32
// accuracy where the value is small:
// * ln u_a: 1 - u_a = v = (2^32 - 1 - r_a) 2^-32 is exact in integers; for
//   v < 2^-8 the series ln(1 - v) = -(v + v^2/2 + v^3/3 + v^4/4) (next term
//   below 2^-34 v); otherwise log2 u_a from the hardware base-2 logarithm
//   (absolute error below 2^-22.6 on [1/2, 2], two ulp elsewhere) times ln 2;
// * rho = a rsqrt(a), a = -2 ln u_a (0 when u_a = 1);
// * the angle 2 pi u_b is reduced exactly in integers to the nearest
//   quarter turn q and a remainder x in [-pi/4, pi/4), sin x / x and cos x
//   are polynomials in x^2 of degrees 3 and 4 fitted by weighted least
//   squares on 20001 Chebyshev points of [-pi/4, pi/4] (relative error of
//   sin below 4e-9, absolute error of cos below 6e-11, both far below an
//   FP32 ulp), and the quarter turn is applied by swaps and signs.
// Against the FP64 form: relative L2 about 1e-7, largest difference about
// 1e-6 (the pair's cos/sin rounding, and near u_a = 1 the FP32 rounding of
// a tiny rho).
__device__ __forceinline__ float ln_u32(uint32_t ra) {
  const uint32_t nv = ~ra;  // (1 - u_a) 2^32
  if (nv < (1u << 24)) {
    const float v = __uint2float_rn(nv) * 0x1p-32f;  // exact: nv < 2^24
    return -v * fmaf(v, fmaf(v, fmaf(v, 0.25f, 0.333333333f), 0.5f), 1.0f);
  }
  return __log2f(fmaf(__uint2float_rn(ra), 0x1p-32f, 0x1p-32f)) * 0.693147180559945309f;
}
__device__ __forceinline__ void sincos_turn32(uint32_t rb, float &s, float &c) {
  const uint32_t q = (rb + (1u << 29)) >> 30;    // nearest quarter turn (mod 4)
  const int32_t t = (int32_t)(rb - (q << 30));   // remainder, |t| <= 2^29 (an eighth)
  const float x = (float)t * (6.28318530717958648f * 0x1p-32f);
  const float x2 = x * x;
  float sp = fmaf(x2, -1.9513928466e-4f, 8.3321482266e-3f);
  sp = fmaf(x2, sp, -1.6666654339e-1f);
  const float sn = fmaf(x * x2, sp, x);
  float cp = fmaf(x2, 2.4389199288e-5f, -1.3886747959e-3f);
  cp = fmaf(x2, cp, 4.1666622701e-2f);
  cp = fmaf(x2, cp, -4.9999999718e-1f);
  const float cs = fmaf(x2, cp, 1.0f);
  // sin(x + q pi/2), cos(x + q pi/2)
  const float a = (q & 1) ? cs : sn, b = (q & 1) ? sn : cs;
  s = (q & 2) ? -a : a;
  c = ((q + 1) & 2) ? -b : b;
}
__device__ __forceinline__ void gauss2(uint32_t ra, uint32_t rb, float &c, float &s) {
  const float a = -2.0f * ln_u32(ra);
  const float rho = a > 0.0f ? a * rsqrtf(a) : 0.0f;
  float sn, cs;
  sincos_turn32(rb, sn, cs);
  c = rho * cs;
  s = rho * sn;
}
__device__ __forceinline__ void gauss2(uint32_t ra, uint32_t rb, double &c, double &s) {
  const double ua = ((double)ra + 1.0) * 0x1p-32;
  const double rho = sqrt(-2.0 * log(ua));
  double sn, cs;
  sincospi(2.0 * ((double)rb * 0x1p-32), &sn, &cs);
  c = rho * cs;
  s = rho * sn;
}
template <typename R> __device__ __forceinline__ void gauss4(uint4 w, R out[4]) {
  gauss2(w.x, w.y, out[0], out[1]);
  gauss2(w.z, w.w, out[2], out[3]);
}

// W at one cell (used where a line does not start on a group boundary).
template <typename R> __device__ __forceinline__ R noise_cell(uint64_t seed, uint64_t idx) {
  R v[4];
  gauss4(noise_words(seed, idx >> 2), v);
  const int lane = (int)(idx & 3);
  return lane == 0 ? v[0] : lane == 1 ? v[1] : lane == 2 ? v[2] : v[3];
}

// A product rounded on its own, never fused into an FMA with a later add.
// Used where the kernels' instantiations differ only in which branches are
// fixed at compile time (a fused multiply-add in one and not in another
// would round differently): the lattice coordinates (i + offset) * cell of
// Eq. 3 and the i m_z factor of the z inverse pass.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// Periodic wrap of a coordinate into [0, L) (Eq. 3 positions).
template <typename R>
__device__ __forceinline__ R wrap_box(R x, R box) {
  if (x < (R)0) x += box;
  else if (x >= box) x -= box;
  if (!(x >= (R)0 && x < box)) {
    x = x - box * floor(x / box);
    if (x >= box) x -= box;
    if (x < (R)0) x = (R)0;
  }
  return x;
}

// Cloud-in-cell (trilinear) interpolation between the cell centres of a
// periodic coarse grid of nl points per axis, evaluated at the centre of
// fine cell i of a grid of nh points: in coarse cell-centre units the centre
// is u = (i + 1/2) nl / nh - 1/2 = ((2i + 1) nl - nh) / (2 nh), taken as an
// exact fraction (floor by integer division, weight of the upper cell t).
template <typename R> struct CicAxis {
  int i0, i1;
  R t;
};
template <typename R> __device__ __forceinline__ CicAxis<R> cic_axis(int i, int nl, int nh) {
  const int num = (2 * i + 1) * nl - nh, den = 2 * nh;
  const int q = num >= 0 ? num / den : -((den - 1 - num) / den);  // floor(num / den) >= -1
  CicAxis<R> c;
  c.t = (R)(num - q * den) / (R)den;
  c.i0 = q < 0 ? q + nl : q;
  c.i1 = c.i0 + 1 == nl ? 0 : c.i0 + 1;
  return c;
}
// Both fine cells 2n and 2n + 1 of a z line at once (nl <= nh): their
// numerators differ by 2 nl < 2 nh, so one division serves both, and their
// z taps lie in the three consecutive coarse cells q, q + 1, q + 2; each of
// the four (x, y) coarse lines is read at those three points, combined
// bilinearly in x and y, then linearly in z per cell.
template <typename R>
__device__ __forceinline__ void cic_pair(const R *__restrict__ g, int nl, int nh, const CicAxis<R> &x,
                                         const CicAxis<R> &y, int n, R &a0, R &a1) {
  const int den = 2 * nh;
  const int num0 = (4 * n + 1) * nl - nh;
  const int q = num0 >= 0 ? num0 / den : -((den - 1 - num0) / den);  // floor, >= -1
  const int r0 = num0 - q * den;
  const int step = r0 + 2 * nl >= den ? 1 : 0;  // cell 2n + 1 starts one coarse cell later
  const int r1 = r0 + 2 * nl - step * den;
  const int z0 = q < 0 ? q + nl : q;
  const int z1 = z0 + 1 == nl ? 0 : z0 + 1;
  const int z2 = z1 + 1 == nl ? 0 : z1 + 1;
  const R wx[2] = {(R)1 - x.t, x.t}, wy[2] = {(R)1 - y.t, y.t};
  const int ix[2] = {x.i0, x.i1}, iy[2] = {y.i0, y.i1};
  R c0 = (R)0, c1 = (R)0, c2 = (R)0;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const R *line = g + ((int64_t)ix[a] * nl + iy[b]) * nl;
      const R w = wx[a] * wy[b];
      c0 += w * __ldg(line + z0);
      c1 += w * __ldg(line + z1);
      c2 += w * __ldg(line + z2);
    }
  const R t0 = (R)r0 / (R)den, t1 = (R)r1 / (R)den;
  a0 = ((R)1 - t0) * c0 + t0 * c1;
  a1 = step ? ((R)1 - t1) * c1 + t1 * c2 : ((R)1 - t1) * c0 + t1 * c1;
}

// ------------------------------------------------------------------ butterflies
// In-register DFT of length RAD: y_k = sum_n x_n exp(-+2 pi i n k / RAD)
// (minus sign forward, plus sign for INV).
template <int RAD, bool INV, typename T> struct Butterfly;

template <bool INV, typename T> struct Butterfly<2, INV, T> {
  static __device__ __forceinline__ void run(T *v) {
    const T a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <bool INV, typename T> struct Butterfly<3, INV, T> {
  static __device__ __forceinline__ void run(T *v) {
    using R = decltype(v[0].x);
    const R h = (R)0.86602540378443864676;  // sqrt(3)/2
    const T s = cadd(v[1], v[2]);
    const T d = csub(v[1], v[2]);
    const T t = {v[0].x - (R)0.5 * s.x, v[0].y - (R)0.5 * s.y};
    const T hd = {h * d.x, h * d.y};
    v[0] = cadd(v[0], s);
    v[1] = cadd(t, mul_wi<INV>(hd));
    v[2] = csub(t, mul_wi<INV>(hd));
  }
};

template <bool INV, typename T> struct Butterfly<4, INV, T> {
  static __device__ __forceinline__ void run(T *v) {
    const T t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    const T t2 = cadd(v[1], v[3]), t3 = mul_wi<INV>(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
  }
};

template <bool INV, typename T> struct Butterfly<8, INV, T> {
  static __device__ __forceinline__ void run(T *v) {
    using R = decltype(v[0].x);
    const R r2 = (R)0.70710678118654752440;  // 1/sqrt(2)
    T e[4] = {v[0], v[2], v[4], v[6]};
    T o[4] = {v[1], v[3], v[5], v[7]};
    Butterfly<4, INV, T>::run(e);
    Butterfly<4, INV, T>::run(o);
    // o_k *= w8^k, w8 = exp(-+2 pi i / 8)
    T o1, o3;
    if (INV) {
      o1 = {r2 * (o[1].x - o[1].y), r2 * (o[1].x + o[1].y)};
      o3 = {-r2 * (o[3].x + o[3].y), r2 * (o[3].x - o[3].y)};
    } else {
      o1 = {r2 * (o[1].x + o[1].y), r2 * (o[1].y - o[1].x)};
      o3 = {r2 * (o[3].y - o[3].x), -r2 * (o[3].x + o[3].y)};
    }
    const T o2 = mul_wi<INV>(o[2]);
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);
    v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);
    v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);
    v[7] = csub(e[3], o3);
  }
};

// ---------------------------------------------------------------- smem layouts
// Contiguous lines (z passes): element n of line l at l * ld + n + n / 16.
struct LineLayout {
  int ld;
  __device__ __forceinline__ int operator()(int l, int n) const { return l * ld + n + (n >> 4); }
};
__host__ __device__ inline int line_ld(int half_len) { return half_len + (half_len >> 4) + 1; }

// ------------------------------------------------ TMA and mbarrier helpers
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// Before the barrier's shared memory is used for anything else.
__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Orders this thread's (and, after a CTA barrier, the CTA's) generic-proxy
// shared-memory accesses before later async-proxy (TMA) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait for the phase with the given parity: gives up after limit_us
// microseconds of the global timer (0: two seconds, far beyond any tile
// copy), then returns false and sets *err = 2 (GG_ETIMEOUT on the host).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *err,
                                          uint32_t limit_us = 0) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  const uint64_t lim = 1000ull * (limit_us ? limit_us : 2000000u);
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > lim) {
      if (err) atomicExch(err, 2);
      return false;
    }
  return true;
}
// 3-D tiled TMA load global -> shared, completion counted on `bar`.
__device__ __forceinline__ void tma_load_3d(void *dst, const void *map, uint64_t *bar, int c0, int c1,
                                            int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_addr(dst)),
      "l"(map), "r"(smem_addr(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}
__device__ __forceinline__ void prefetch_l1(const void *p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}
// 4-D tiled TMA load (the strided passes: kz reals, y, x, realization).
__device__ __forceinline__ void tma_load_4d(void *dst, const void *map, uint64_t *bar, int c0, int c1,
                                            int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(smem_addr(dst)),
      "l"(map), "r"(smem_addr(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
      : "memory");
}
// 5-D tiled TMA load (chunk-major spectra: reals of a chunk, y, x, chunk, realization).
__device__ __forceinline__ void tma_load_5d(void *dst, const void *map, uint64_t *bar, int c0, int c1,
                                            int c2, int c3, int c4) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6, %7}], [%2];" ::"r"(smem_addr(dst)),
      "l"(map), "r"(smem_addr(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
      : "memory");
}
// Tiled TMA stores shared -> global (the strided passes' output tiles, same
// coordinates as the loads), tracked by the issuing thread's bulk group.
__device__ __forceinline__ void tma_store_4d(const void *map, const void *src, int c0, int c1, int c2,
                                             int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4, %5}], [%1];" ::"l"(
          map),
      "r"(smem_addr(src)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
      : "memory");
}
__device__ __forceinline__ void tma_store_5d(const void *map, const void *src, int c0, int c1, int c2,
                                             int c3, int c4) {
  asm volatile(
      "cp.async.bulk.tensor.5d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4, %5, %6}], [%1];" ::"l"(
          map),
      "r"(smem_addr(src)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
      : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// This thread's committed bulk stores have read their shared memory (it may
// be rewritten).
__device__ __forceinline__ void bulk_wait_read0() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// This thread's committed bulk stores are complete.
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// Plain bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// ------------------------------------------------------------- Stockham stage
// Multiplies v[r] (r = 1 .. RAD-1) by w^r (conjugated for INV), the powers
// formed from w = w^1 by at most three products (FP32, where a table load
// costs more than four FMAs) or read from the table (FP64, whose arithmetic
// is the scarce resource on this GPU).
template <int RAD, bool INV, typename T>
__device__ __forceinline__ void twiddle_powers(T *v, T w1) {
  auto mul = [](T x, T w) { return INV ? cmulc(x, w) : cmul(x, w); };
  if constexpr (RAD == 2) {
    v[1] = mul(v[1], w1);
  } else if constexpr (RAD == 3) {
    const T w2 = cmul(w1, w1);
    v[1] = mul(v[1], w1);
    v[2] = mul(v[2], w2);
  } else if constexpr (RAD == 4) {
    const T w2 = cmul(w1, w1), w3 = cmul(w2, w1);
    v[1] = mul(v[1], w1);
    v[2] = mul(v[2], w2);
    v[3] = mul(v[3], w3);
  } else {
    const T w2 = cmul(w1, w1), w3 = cmul(w2, w1), w4 = cmul(w2, w2);
    const T w5 = cmul(w4, w1), w6 = cmul(w4, w2), w7 = cmul(w4, w3);
    v[1] = mul(v[1], w1);
    v[2] = mul(v[2], w2);
    v[3] = mul(v[3], w3);
    v[4] = mul(v[4], w4);
    v[5] = mul(v[5], w5);
    v[6] = mul(v[6], w6);
    v[7] = mul(v[7], w7);
  }
}

// Twiddles of one stage for this thread's butterflies j = p + P*b (FP32):
// w^1 per butterfly, loaded before the stage's shared-memory reads so that the
// load latency overlaps them. FP64 reads each power from the table at use:
// FP64 arithmetic, not load latency, is the scarce resource on this GPU.
template <typename R, int E, int RAD> struct StageTw {
  static constexpr int kCount = sizeof(R) == 4 ? E / RAD : 1;
  Cx<R> w[kCount];
};

template <typename R, int E, int RAD>
__device__ __forceinline__ void load_twiddles(StageTw<R, E, RAD> &t, int p, int P, int ns,
                                              int ns_shift, int tstep, const Cx<R> *__restrict__ tw) {
  if constexpr (sizeof(R) == 4) {
    if (ns <= 1) return;
#pragma unroll
    for (int b = 0; b < E / RAD; ++b) {
      const int j = p + P * b;
      const int k = ns_shift >= 0 ? (j & ((1 << ns_shift) - 1)) : (j % ns);
      t.w[b] = ldg_c(tw + k * tstep);
    }
  }
}

// Butterflies of one Stockham decimation-in-time stage on registers: v holds,
// for each butterfly j = p + P*b of this thread, the RAD inputs at positions
// j + r*len/RAD; on return it holds the outputs for positions
// (j - k)*RAD + k + r*ns, k = j mod ns.
template <typename R, int E, int RAD, bool INV>
__device__ __forceinline__ void stage_compute(Cx<R> *v, int p, int P, int ns, int ns_shift, int tstep,
                                              const StageTw<R, E, RAD> &t,
                                              const Cx<R> *__restrict__ tw) {
  constexpr int NB = E / RAD;
  if (ns > 1) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      if constexpr (sizeof(R) == 4) {
        twiddle_powers<RAD, INV>(&v[b * RAD], t.w[b]);
      } else {
        const int j = p + P * b;
        const int k = ns_shift >= 0 ? (j & ((1 << ns_shift) - 1)) : (j % ns);
#pragma unroll
        for (int r = 1; r < RAD; ++r) {
          const Cx<R> w = ldg_c(tw + k * tstep * r);
          v[b * RAD + r] = INV ? cmulc(v[b * RAD + r], w) : cmul(v[b * RAD + r], w);
        }
      }
    }
  }
#pragma unroll
  for (int b = 0; b < NB; ++b) Butterfly<RAD, INV, Cx<R>>::run(&v[b * RAD]);
}

// Output position of element r of butterfly j in a stage with ns.
__device__ __forceinline__ int stage_out_pos(int j, int r, int ns, int ns_shift, int rad) {
  const int k = ns_shift >= 0 ? (j & ((1 << ns_shift) - 1)) : (j % ns);
  return (j - k) * rad + k + r * ns;
}

// One whole stage with caller-supplied element access: ld(n) returns element
// n of the stage input, st(n, v) stores element n of its output. With SYNC the
// stage runs in place in shared memory (barrier between all reads and all
// writes, and after the writes).
template <typename R, int E, int RAD, bool INV, bool SYNC, class Ld, class St>
__device__ __forceinline__ void stage_io(int p, int P, int len, int ns, int ns_shift, int tstep,
                                         const Cx<R> *__restrict__ tw, const Ld &ld, const St &st) {
  constexpr int NB = E / RAD;
  // opaque to the optimiser: keeps this stage's index arithmetic inside the
  // stage instead of hoisted (and live) across the whole kernel
  asm volatile("" : "+r"(p));
  StageTw<R, E, RAD> t;
  load_twiddles<R, E, RAD>(t, p, P, ns, ns_shift, tstep, tw);
  Cx<R> v[E];
  const int span = len / RAD;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int j = p + P * b;
#pragma unroll
    for (int r = 0; r < RAD; ++r) v[b * RAD + r] = ld(j + r * span);
  }
  if (SYNC) __syncthreads();
  stage_compute<R, E, RAD, INV>(v, p, P, ns, ns_shift, tstep, t, tw);
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int j = p + P * b;
#pragma unroll
    for (int r = 0; r < RAD; ++r) st(stage_out_pos(j, r, ns, ns_shift, RAD), v[b * RAD + r]);
  }
  if (SYNC) __syncthreads();
}

// Calls f(std::integral_constant<int, RAD>) for the run-time radix `rad`.
template <int E, class F>
__device__ __forceinline__ void with_radix(int rad, const F &f) {
  if constexpr (E % 8 == 0) {
    if (rad == 8) { f(IntC<8>{}); return; }
  }
  if constexpr (E % 4 == 0) {
    if (rad == 4) { f(IntC<4>{}); return; }
  }
  if constexpr (E % 2 == 0) {
    if (rad == 2) { f(IntC<2>{}); return; }
  }
  if constexpr (E % 3 == 0) {
    if (rad == 3) { f(IntC<3>{}); return; }
  }
}

// Stage s of st with the radix dispatched at run time.
template <typename R, int E, bool INV, bool SYNC, class Ld, class St>
__device__ __forceinline__ void stage_dispatch(const FftStages &st, int s, int p, int P,
                                               const Cx<R> *__restrict__ tw, const Ld &ld,
                                               const St &sto) {
  const int ns = st.ns[s], sh = st.ns_shift[s], ts = st.tstep[s];
  with_radix<E>(st.radix[s], [&](auto rc) {
    stage_io<R, E, decltype(rc)::value, INV, SYNC>(p, P, st.len, ns, sh, ts, tw, ld, sto);
  });
}

// All stages of st on line l of a LineLayout tile (every thread of the CTA
// must call this).
template <typename R, int E, bool INV, class Lay>
__device__ __forceinline__ void fft_smem(Cx<R> *buf, const Lay &lay, int l, int p, int P,
                                         const FftStages &st, const Cx<R> *__restrict__ tw) {
  auto ld = [&](int n) { return buf[lay(l, n)]; };
  auto sto = [&](int n, Cx<R> v) { buf[lay(l, n)] = v; };
  for (int s = 0; s < st.nstages; ++s) stage_dispatch<R, E, INV, true>(st, s, p, P, tw, ld, sto);
}

}  // namespace gg
