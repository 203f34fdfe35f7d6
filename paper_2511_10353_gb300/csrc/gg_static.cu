// gg_gaussian_field_static: the density field of gg_gaussian_field for small
// grids, without any device allocation.
//
// Who needs this: a caller that cannot call cudaMalloc. For example, an
// application whose device memory is entirely owned by its own pool
// allocator (so cudaMalloc would fail or break its accounting), or code that
// must not pay cudaMalloc's implicit device-wide synchronisation in the middle
// of latency-critical work. gg_plan allocates a transform workspace and its
// tables; this entry point instead uses fixed arrays that live in the
// library's own device image (file-scope __device__ storage below), sized for
// grids of at most GG_STATIC_MAX_N points per axis.
//
// Costs of that choice, which callers must accept:
//  * every GPU that loads the library holds the arrays (about 2.2 MB) until
//    the process exits, used or not;
//  * every call on a device, from any stream or host thread of this process,
//    shares them: calls whose work overlaps on that GPU race and corrupt each
//    other's results; serialise them (one stream, or events). (Each process
//    has its own copy of the arrays in its own CUDA context.);
//  * the first call on each device looks the arrays' device addresses up
//    with cudaGetSymbolAddress (which may load the module) and keeps them for
//    the life of the process: cudaDeviceReset between calls is not supported
//    (the kept addresses would be stale);
//  * every call copies its host-made tables with cudaMemcpyAsync from host
//    stack arrays and ends with cudaStreamSynchronize, so no call can be made
//    while its stream is being captured into a CUDA graph.
// The host side computes the FP64 cosmology and tables with ordinary host
// code (as gg_plan does), evaluating the cosmology model once per call;
// nothing here allocates device memory or calls an allocating CUDA or
// PyTorch routine.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "gg.h"
#include "gg_internal.h"

namespace {

constexpr int kMaxN = GG_STATIC_MAX_N;
constexpr int kMaxHalf = kMaxN / 2;
constexpr int kMaxTable = 3 * kMaxHalf * kMaxHalf + 1;  // S(m2), m2 <= 3 (N/2)^2
constexpr double kPi = 3.14159265358979323846;

// Device-side scratch, shared by every call on a device. Sized in bytes for
// FP64; FP32 calls use the first half of each.
static __device__ __align__(256) double g_work[(size_t)kMaxN * kMaxN * kMaxN];
static __device__ __align__(256) double g_tw_n[2 * kMaxN];
static __device__ __align__(256) double g_tw_half[2 * kMaxHalf];
static __device__ __align__(256) double g_table[kMaxTable];
static __device__ __align__(256) int g_err[64];

struct Scratch {
  void *work = nullptr, *tw_n = nullptr, *tw_half = nullptr, *table = nullptr;
  int *err = nullptr;
  bool ready = false;
};
constexpr int kMaxDevices = 64;
Scratch g_scratch[kMaxDevices];
std::mutex g_scratch_mu;

// failures are reported through gg_last_error(NULL), like every plan-less call
gg_status fail(gg_status st, const char *msg) {
  gg::set_thread_error(msg);
  return st;
}

// Once per device, with that device current: the device addresses of the
// scratch arrays (host code may not use the symbols themselves as pointers).
gg_status scratch_for_current_device(Scratch **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(GG_ECUDA, "gg_gaussian_field_static: no usable current device");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  Scratch &s = g_scratch[dev];
  if (!s.ready) {
    if (cudaGetSymbolAddress(&s.work, g_work) != cudaSuccess ||
        cudaGetSymbolAddress(&s.tw_n, g_tw_n) != cudaSuccess ||
        cudaGetSymbolAddress(&s.tw_half, g_tw_half) != cudaSuccess ||
        cudaGetSymbolAddress(&s.table, g_table) != cudaSuccess ||
        cudaGetSymbolAddress((void **)&s.err, g_err) != cudaSuccess)
      return fail(GG_ECUDA, "gg_gaussian_field_static: cudaGetSymbolAddress failed");
    s.ready = true;
  }
  *out = &s;
  return GG_OK;
}

template <typename R>
gg_status run(const gg_params *p, const gg_info &info, const double *sd, uint64_t seed,
              const void *noise, void *delta, cudaStream_t st, const Scratch &s) {
  const int n = (int)p->n, half = n / 2;
  // tables in FP64 on the host, rounded once, copied into the scratch arrays
  R tw_n[2 * kMaxN], tw_half[2 * kMaxHalf], tab[kMaxTable];
  for (int i = 0; i < n; ++i) {
    tw_n[2 * i] = (R)std::cos(-2.0 * kPi * i / n);
    tw_n[2 * i + 1] = (R)std::sin(-2.0 * kPi * i / n);
  }
  for (int i = 0; i < half; ++i) {
    tw_half[2 * i] = (R)std::cos(-2.0 * kPi * i / half);
    tw_half[2 * i + 1] = (R)std::sin(-2.0 * kPi * i / half);
  }
  const int count = 3 * half * half + 1;
  const double norm = 1.0 / std::pow((double)n, 1.5);
  for (int i = 0; i < count; ++i) tab[i] = (R)(sd[i] * norm);
  cudaError_t e;
  if ((e = cudaMemsetAsync(s.err, 0, sizeof(int), st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(s.tw_n, tw_n, sizeof(R) * 2 * n, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(s.tw_half, tw_half, sizeof(R) * 2 * half, cudaMemcpyHostToDevice, st)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(s.table, tab, sizeof(R) * count, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return fail(GG_ECUDA, cudaGetErrorString(e));
  gg::FftStages st_n, st_half;
  if (!gg::make_stages(n, &st_n) || !gg::make_stages(half, &st_half))
    return fail(GG_EINVAL, "gg_gaussian_field_static: no FFT schedule");
  const gg::FftStages st_inv = gg::reversed_stages(st_n);
  const bool spec = gg::spec_has<R>(n);
  // z forward: noise (generated or read) -> half spectrum in the scratch grid
  gg::ZFwdArgs z{};
  z.noise = noise;
  z.out = s.work;
  z.seed = seed;
  z.nlines = (int64_t)n * n;
  z.n = n;
  z.st = st_half;
  z.tw_half = s.tw_half;
  z.tw_full = s.tw_n;
  const int lines = gg::z_lines_per_cta<R>(st_half);  // the rule gg_plan uses
  z.lines_per_cta = lines;
  e = spec ? gg::spec_zfwd<R>(z, st) : gg::launch_zfwd<R>(z, st);
  if (e != cudaSuccess) return fail(GG_ECUDA, cudaGetErrorString(e));
  // strided passes: plain (non-TMA) tiles of one column for the run-time kernel
  gg::AxisArgs a{};
  a.src = s.work;
  a.cols = 1;
  a.inner_chunks = half;
  a.n = n;
  a.st_fwd = st_n;
  a.st_inv = st_inv;
  a.tw = s.tw_n;
  a.table = s.table;
  a.e = st_n.e;
  a.rows_box = 0;
  a.err = s.err;
  auto axis = [&](int axis_id, int fwd, int inv, int pre) {
    gg::AxisArgs c = a;
    c.axis = axis_id;
    c.stride = axis_id == 1 ? half : (int64_t)n * half;
    c.outer_stride = axis_id == 1 ? (int64_t)n * half : half;
    c.fwd = fwd;
    c.inv = inv;
    c.pre = pre;
    c.nout = 1;
    c.dst[0] = s.work;
    c.mul[0] = gg::kMulNone;
    return spec ? gg::spec_axis<R>(c, st) : gg::launch_axis<R>(c, st);
  };
  if ((e = axis(1, 1, 0, 0)) != cudaSuccess || (e = axis(0, 1, 1, 1)) != cudaSuccess ||
      (e = axis(1, 0, 1, 0)) != cudaSuccess)
    return fail(GG_ECUDA, cudaGetErrorString(e));
  gg::ZInvArgs zi{};
  zi.src = s.work;
  zi.psi = delta;
  zi.nlines = (int64_t)n * n;
  zi.n = n;
  zi.lines_per_cta = lines;
  zi.box = p->box;
  zi.cell = p->box / n;
  zi.q_offset = 0.5;
  zi.vfac = info.vfac;
  zi.st = st_half;
  zi.tw_half = s.tw_half;
  zi.tw_full = s.tw_n;
  zi.err = s.err;
  e = spec ? gg::spec_zinv<R>(zi, st) : gg::launch_zinv<R>(zi, st);
  if (e != cudaSuccess) return fail(GG_ECUDA, cudaGetErrorString(e));
  int word = 0;
  if ((e = cudaMemcpyAsync(&word, s.err, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)  // also keeps the host tables alive until used
    return fail(GG_ECUDA, cudaGetErrorString(e));
  if (word) return fail(word == 2 ? GG_ETIMEOUT : GG_ECUDA, "device reported an error");
  return GG_OK;
}

}  // namespace

extern "C" gg_status gg_gaussian_field_static(const gg_params *p, uint64_t seed,
                                              const void *noise_dev, void *delta_dev, void *stream) {
  if (!p) return fail(GG_EINVAL, "gg_gaussian_field_static: params is NULL");
  if (p->n > kMaxN) {
    char msg[200];
    std::snprintf(msg, sizeof msg,
                  "gg_gaussian_field_static: n = %lld exceeds the static scratch limit of %d "
                  "(use gg_plan + gg_gaussian_field for larger grids)",
                  (long long)p->n, kMaxN);
    return fail(GG_EINVAL, msg);
  }
  // the cosmology and the Eq. 1 filter from one evaluation of the model
  // (also the parameter check: invalid parameters as in gg_plan)
  gg_info info{};
  double sd[kMaxTable];
  const int half = p->n > 0 ? (int)(p->n / 2) : 0;
  const char *why = nullptr;
  if (!gg::info_and_filter(p, &info, sd, 3 * (int64_t)half * half + 1, &why))
    return fail(GG_EINVAL, why ? why : "invalid parameters");
  if (!delta_dev || ((uintptr_t)delta_dev & 15u) || ((uintptr_t)noise_dev & 15u))
    return fail(GG_EINVAL, "gg_gaussian_field_static: delta_dev NULL or a buffer unaligned");
  Scratch *s = nullptr;
  gg_status stt = scratch_for_current_device(&s);
  if (stt != GG_OK) return stt;
  const cudaStream_t st = (cudaStream_t)stream;
  return p->prec == GG_F64 ? run<double>(p, info, sd, seed, noise_dev, delta_dev, st, *s)
                           : run<float>(p, info, sd, seed, noise_dev, delta_dev, st, *s);
}
