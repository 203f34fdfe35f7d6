// White-noise refinement (Appendix A) on sm_103a.
//
// One thread owns one parent patch (N_L^3 parent cells -> N_H^3 child cells):
//   1. the parent coefficients a_ijk = sum F_i F_j F_k V (i, j, k < N_L),
//      three separable passes over the patch in registers;
//   2. the new coefficients: the child grid's white noise at the child cell
//      of each coefficient position, one Philox group per child z-run;
//   3. the child values W = sum a_ijk E_i E_j E_k (Eqs. A.14, A.28), three
//      separable passes, stored as z-runs (one 16-byte store per run for
//      FP32 doubling; a warp's runs are contiguous, 512 bytes per store).
// The work is local and every child value is written once: HBM traffic is
// the parent read once plus the child written once; the Philox and
// Box-Muller arithmetic for the new coefficients is the larger cost.
#include <cmath>
#include <cstdint>
#include <cstdio>

#include <cuda_runtime.h>

#include "gg.h"
#include "gg_device.cuh"
#include "gg_internal.h"

namespace gg {
namespace {

template <typename R> struct Basis {
  R f[3][3];  // f[i][m] = F_i(m), i, m < N_L
  R e[4][4];  // e[j][k] = E_j(k), j, k < N_H
};

struct RefineBox {
  int64_t n;         // parent points per axis
  int64_t nc;        // points per axis of the whole refined grid
  int64_t np;        // parent patches per axis, n / N_L
  int64_t o[3];      // first parent patch of the box, per axis
  int64_t pp[3];     // patches of the box, per axis
  int64_t dims[3];   // child box, per axis
  int64_t patches;   // pp[0] * pp[1] * pp[2]
};

// N_H consecutive child-noise values starting at global child cell idx0
// (they lie in one or two Philox groups). HI_ONLY (runs of four): only the
// last two values are used, so only the second Box-Muller pair is formed.
template <typename R, int NH, bool HI_ONLY>
__device__ __forceinline__ void noise_run(uint64_t seed, uint64_t idx0, R out[NH]) {
  if constexpr (NH == 4) {  // runs of four start on a group (the host checks nc % 4 == 0)
    const uint4 g = noise_words(seed, idx0 >> 2);
    if (!HI_ONLY) gauss2(g.x, g.y, out[0], out[1]);
    gauss2(g.z, g.w, out[2], out[3]);
  } else {
    R w[8];
    gauss4(noise_words(seed, idx0 >> 2), w);
    const int s = (int)(idx0 & 3);
    if (s + NH > 4) {
      gauss4(noise_words(seed, (idx0 >> 2) + 1), w + 4);
    } else {
#pragma unroll
      for (int k = 4; k < 8; ++k) w[k] = (R)0;
    }
#pragma unroll
    for (int k = 0; k < NH; ++k)
      out[k] = s == 0 ? w[k] : s == 1 ? w[k + 1] : s == 2 ? w[k + 2] : w[k + 3];
  }
}

template <typename R, int NH> __device__ __forceinline__ void store_run(R *p, const R *v) {
  if constexpr (NH == 4 && sizeof(R) == 4) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else if constexpr (NH == 2 && sizeof(R) == 4) {
    *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
  } else if constexpr (NH % 2 == 0 && sizeof(R) == 8) {
#pragma unroll
    for (int k = 0; k < NH; k += 2) *reinterpret_cast<double2 *>(p + k) = make_double2(v[k], v[k + 1]);
  } else {
#pragma unroll
    for (int k = 0; k < NH; ++k) p[k] = v[k];
  }
}

template <typename R, int NL, int NH>
__global__ void __launch_bounds__(256) k_refine(const R *__restrict__ parent, R *__restrict__ child,
                                                const Basis<R> bs, const RefineBox b, uint64_t seed) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < b.patches; t += step) {
    const int64_t pz = t % b.pp[2], rest = t / b.pp[2];
    const int64_t py = rest % b.pp[1], px = rest / b.pp[1];
    // the patch in the whole grid (periodic)
    const int64_t gx = (b.o[0] + px) % b.np, gy = (b.o[1] + py) % b.np, gz = (b.o[2] + pz) % b.np;
    R a[NH][NH][NH];
    // 1. parent coefficients
    {
      R v[NL][NL][NL];
#pragma unroll
      for (int m = 0; m < NL; ++m)
#pragma unroll
        for (int q = 0; q < NL; ++q) {
          const R *row = parent + ((gx * NL + m) * b.n + gy * NL + q) * b.n + gz * NL;
#pragma unroll
          for (int l = 0; l < NL; ++l) v[m][q][l] = row[l];
        }
      R u[NL][NL][NL], w[NL][NL][NL];
#pragma unroll
      for (int m = 0; m < NL; ++m)  // along z: u[m][q][k] = sum_l F_k(l) v[m][q][l]
#pragma unroll
        for (int q = 0; q < NL; ++q)
#pragma unroll
          for (int k = 0; k < NL; ++k) {
            R s = (R)0;
#pragma unroll
            for (int l = 0; l < NL; ++l) s = fma(bs.f[k][l], v[m][q][l], s);
            u[m][q][k] = s;
          }
#pragma unroll
      for (int m = 0; m < NL; ++m)  // along y
#pragma unroll
        for (int j = 0; j < NL; ++j)
#pragma unroll
          for (int k = 0; k < NL; ++k) {
            R s = (R)0;
#pragma unroll
            for (int q = 0; q < NL; ++q) s = fma(bs.f[j][q], u[m][q][k], s);
            w[m][j][k] = s;
          }
#pragma unroll
      for (int i = 0; i < NL; ++i)  // along x
#pragma unroll
        for (int j = 0; j < NL; ++j)
#pragma unroll
          for (int k = 0; k < NL; ++k) {
            R s = (R)0;
#pragma unroll
            for (int m = 0; m < NL; ++m) s = fma(bs.f[i][m], w[m][j][k], s);
            a[i][j][k] = s;
          }
    }
    // 2. new coefficients: child noise at the coefficient's child cell
#pragma unroll
    for (int i = 0; i < NH; ++i)
#pragma unroll
      for (int j = 0; j < NH; ++j) {
        const uint64_t idx0 =
            ((uint64_t)(gx * NH + i) * (uint64_t)b.nc + (uint64_t)(gy * NH + j)) * (uint64_t)b.nc +
            (uint64_t)(gz * NH);
        R r[NH];
        if (i < NL && j < NL) noise_run<R, NH, NL >= 2>(seed, idx0, r);  // k < N_L: parent's
        else noise_run<R, NH, false>(seed, idx0, r);
#pragma unroll
        for (int k = 0; k < NH; ++k)
          if (i >= NL || j >= NL || k >= NL) a[i][j][k] = r[k];
      }
    // 3. W(m, q, l) = sum_ijk a_ijk E_i(m) E_j(q) E_k(l), in place
#pragma unroll
    for (int i = 0; i < NH; ++i)  // along z
#pragma unroll
      for (int j = 0; j < NH; ++j) {
        R s[NH];
#pragma unroll
        for (int l = 0; l < NH; ++l) {
          s[l] = (R)0;
#pragma unroll
          for (int k = 0; k < NH; ++k) s[l] = fma(a[i][j][k], bs.e[k][l], s[l]);
        }
#pragma unroll
        for (int l = 0; l < NH; ++l) a[i][j][l] = s[l];
      }
#pragma unroll
    for (int i = 0; i < NH; ++i)  // along y
#pragma unroll
      for (int l = 0; l < NH; ++l) {
        R s[NH];
#pragma unroll
        for (int q = 0; q < NH; ++q) {
          s[q] = (R)0;
#pragma unroll
          for (int j = 0; j < NH; ++j) s[q] = fma(a[i][j][l], bs.e[j][q], s[q]);
        }
#pragma unroll
        for (int q = 0; q < NH; ++q) a[i][q][l] = s[q];
      }
#pragma unroll
    for (int q = 0; q < NH; ++q)  // along x
#pragma unroll
      for (int l = 0; l < NH; ++l) {
        R s[NH];
#pragma unroll
        for (int m = 0; m < NH; ++m) {
          s[m] = (R)0;
#pragma unroll
          for (int i = 0; i < NH; ++i) s[m] = fma(a[i][q][l], bs.e[i][m], s[m]);
        }
#pragma unroll
        for (int m = 0; m < NH; ++m) a[m][q][l] = s[m];
      }
    // child box coordinates of the patch's first cell
#pragma unroll
    for (int m = 0; m < NH; ++m)
#pragma unroll
      for (int q = 0; q < NH; ++q)
        store_run<R, NH>(child + ((px * NH + m) * b.dims[1] + py * NH + q) * b.dims[2] + pz * NH,
                         a[m][q]);
  }
}

// ------------------------------------------------------------ host side
struct KindInfo {
  int nl, nh;
};

bool kind_info(gg_refine_kind k, KindInfo *out) {
  switch (k) {
    case GG_REFINE_HR: *out = {1, 2}; return true;
    case GG_REFINE_3_2: *out = {2, 3}; return true;
    case GG_REFINE_2:
    case GG_REFINE_2_LINEAR:
    case GG_REFINE_2_SINE: *out = {2, 4}; return true;
    case GG_REFINE_4_3: *out = {3, 4}; return true;
  }
  return false;
}

// The bases of Appendix A in FP64 (rows are basis functions).
void bases(gg_refine_kind k, double f[3][3], double e[4][4]) {
  const double r2 = std::sqrt(2.0), r3 = std::sqrt(3.0), r6 = std::sqrt(6.0), r7 = std::sqrt(7.0),
               r20 = std::sqrt(20.0);
  const double two[2][2] = {{1 / r2, 1 / r2}, {-1 / r2, 1 / r2}};               // Eqs. A.2-A.3, A.5-A.6
  const double three[3][3] = {{1 / r3, 1 / r3, 1 / r3}, {-1 / r2, 0.0, 1 / r2},  // Eqs. A.7-A.9
                              {-1 / r6, 2 / r6, -1 / r6}};
  const double four[4][4] = {{0.5, 0.5, 0.5, 0.5},  // Eqs. A.10-A.13
                             {-r7 / 4, -0.25, 0.25, r7 / 4},
                             {-0.5, 0.5, 0.5, -0.5},
                             {0.25, -r7 / 4, r7 / 4, -0.25}};
  const double four_lin[4][4] = {{0.5, 0.5, 0.5, 0.5},  // Eqs. A.20-A.23
                                 {-3 / r20, -1 / r20, 1 / r20, 3 / r20},
                                 {-0.5, 0.5, 0.5, -0.5},
                                 {1 / r20, -3 / r20, 3 / r20, -1 / r20}};
  const double four_sine[4][4] = {{0.5, 0.5, 0.5, 0.5},  // Eqs. A.24-A.27
                                  {-0.5, -0.5, 0.5, 0.5},
                                  {-0.5, 0.5, 0.5, -0.5},
                                  {0.5, -0.5, 0.5, -0.5}};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) f[i][j] = 0.0;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) e[i][j] = 0.0;
  auto put_f = [&](const double *src, int n) {
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) f[i][j] = src[i * n + j];
  };
  auto put_e = [&](const double *src, int n) {
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) e[i][j] = src[i * n + j];
  };
  switch (k) {
    case GG_REFINE_HR: f[0][0] = 1.0; put_e(&two[0][0], 2); break;
    case GG_REFINE_3_2: put_f(&two[0][0], 2); put_e(&three[0][0], 3); break;
    case GG_REFINE_2: put_f(&two[0][0], 2); put_e(&four[0][0], 4); break;
    case GG_REFINE_2_LINEAR: put_f(&two[0][0], 2); put_e(&four_lin[0][0], 4); break;
    case GG_REFINE_2_SINE: put_f(&two[0][0], 2); put_e(&four_sine[0][0], 4); break;
    case GG_REFINE_4_3: put_f(&three[0][0], 3); put_e(&four[0][0], 4); break;
  }
}

gg_status fail(const char *msg) {
  set_thread_error(msg);
  return GG_EINVAL;
}

// Checks *p and fills the box; no device calls.
gg_status make_box(const gg_refine_params *p, KindInfo *ki, RefineBox *b) {
  if (!p) return fail("gg_refine: params is NULL");
  if (!kind_info(p->kind, ki)) return fail("gg_refine: unknown refinement kind");
  if (p->prec != GG_F32 && p->prec != GG_F64) return fail("gg_refine: prec must be GG_F32 or GG_F64");
  if (p->n <= 0 || p->n > (int64_t)1 << 20 || p->n % ki->nl)
    return fail("gg_refine: n must be a positive multiple of the parent patch (<= 2^20)");
  b->n = p->n;
  b->np = p->n / ki->nl;
  b->nc = b->np * ki->nh;
  b->patches = 1;
  for (int j = 0; j < 3; ++j) {
    const int64_t ext = p->extent[j] == 0 ? p->n : p->extent[j];
    if (p->origin[j] < 0 || p->origin[j] >= p->n || p->origin[j] % ki->nl)
      return fail("gg_refine: origin must be a multiple of the parent patch in [0, n)");
    if (ext < 0 || ext > p->n || ext % ki->nl)
      return fail("gg_refine: extent must be a multiple of the parent patch in (0, n]");
    b->o[j] = p->origin[j] / ki->nl;
    b->pp[j] = ext / ki->nl;
    b->dims[j] = b->pp[j] * ki->nh;
    b->patches *= b->pp[j];
  }
  if (ki->nh == 4 && b->nc % 4)  // z-runs of four start on a Philox group
    return fail("gg_refine: internal: refined grid not a multiple of 4");
  return GG_OK;
}

template <typename R>
gg_status launch(const gg_refine_params *p, const KindInfo &ki, const RefineBox &b, const void *parent,
                 uint64_t seed, void *child, cudaStream_t st) {
  double f[3][3], e[4][4];
  bases(p->kind, f, e);
  Basis<R> bs;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) bs.f[i][j] = (R)f[i][j];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) bs.e[i][j] = (R)e[i][j];
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 1;
  const int threads = 256;
  const int64_t want = (b.patches + threads - 1) / threads;
  const int blocks = (int)(want < (int64_t)sms * 32 ? want : (int64_t)sms * 32);
  const R *src = static_cast<const R *>(parent);
  R *dst = static_cast<R *>(child);
  if (ki.nl == 1) k_refine<R, 1, 2><<<blocks, threads, 0, st>>>(src, dst, bs, b, seed);
  else if (ki.nl == 2 && ki.nh == 3) k_refine<R, 2, 3><<<blocks, threads, 0, st>>>(src, dst, bs, b, seed);
  else if (ki.nl == 2) k_refine<R, 2, 4><<<blocks, threads, 0, st>>>(src, dst, bs, b, seed);
  else k_refine<R, 3, 4><<<blocks, threads, 0, st>>>(src, dst, bs, b, seed);
  const cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) {
    set_thread_error(cudaGetErrorString(err));
    return GG_ECUDA;
  }
  return GG_OK;
}

}  // namespace
}  // namespace gg

extern "C" gg_status gg_refine_dims(const gg_refine_params *p, int64_t dims[3]) {
  gg::KindInfo ki;
  gg::RefineBox b;
  const gg_status st = gg::make_box(p, &ki, &b);
  if (st != GG_OK) return st;
  if (!dims) return gg::fail("gg_refine_dims: dims is NULL");
  for (int j = 0; j < 3; ++j) dims[j] = b.dims[j];
  return GG_OK;
}

extern "C" gg_status gg_refine_noise(const gg_refine_params *p, const void *parent_dev,
                                     uint64_t seed_child, void *child_dev, void *stream) {
  gg::KindInfo ki;
  gg::RefineBox b;
  const gg_status st = gg::make_box(p, &ki, &b);
  if (st != GG_OK) return st;
  if (!parent_dev || !child_dev || ((uintptr_t)parent_dev & 15u) || ((uintptr_t)child_dev & 15u))
    return gg::fail("gg_refine_noise: parent_dev / child_dev NULL or not 16-byte aligned");
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  return p->prec == GG_F64 ? gg::launch<double>(p, ki, b, parent_dev, seed_child, child_dev, s)
                           : gg::launch<float>(p, ki, b, parent_dev, seed_child, child_dev, s);
}
