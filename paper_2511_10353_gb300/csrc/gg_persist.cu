// The batched form as one persistent launch: every pass of every realization
// of a batch (FP32, grid sizes 64 to 384) in a single kernel.
//
// Work items are (pass, group, run of tiles), numbered pass-major: all z forward
// tiles of every group, then all y forward tiles, and so on. A CTA takes the
// next number from a device counter, waits until the realization owning the
// tile has completed every tile of the pass the tile reads (per-realization
// pass counters; the wait is bounded by the global timer and by an abort
// flag), runs the tile with the size-specialised codelet bodies of
// gg_ct_kernels.cuh in their 256-thread shape, then counts it done. Numbers
// are taken in increasing order and a CTA holds one item at a time, so every
// item a CTA waits on is held by a running CTA whose own waits point further
// back: the schedule cannot deadlock, with or without every CTA resident.
#include "gg_ct_kernels.cuh"

namespace gg {
namespace {

constexpr int kPV = ct::kPersistV;
constexpr int kThreads = 256;
// the pass each pass reads: y forward reads the z forward's output, the x
// pass the y forward's, both y inverse passes the x pass's outputs, the z
// inverse passes the y inverse passes' outputs
__device__ __constant__ int kDep[kPersistPasses] = {-1, 0, 1, 2, 2, 3, 4, 4};
constexpr int kCounterBase = 64;  // words before the pass counters: [0] queue, [1] abort
constexpr int kChunk = 64;        // default tiles per work item, where a realization's tiles divide

// A work item is `chunk` consecutive tiles of one pass and realization (the
// codelet bodies double-buffer their copies across them).
struct PersistParams {
  CUtensorMap maps[kPersistMaxGroups][4];
  PersistPlan p;
  int64_t items[kPersistPasses][kPersistMaxGroups];     // items of a pass over the group's realizations
  int64_t per_real[kPersistPasses][kPersistMaxGroups];  // items of a pass for one realization
  int64_t base[kPersistPasses][kPersistMaxGroups];      // number of its first work item
  int chunk[kPersistPasses][kPersistMaxGroups];         // tiles per item
  int64_t total;
};
static_assert(sizeof(PersistParams) <= 32000, "kernel parameter space");

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Tiles t .. t + c - 1 of one pass of group gi.
template <int N>
__device__ __noinline__ bool persist_item(const PersistParams &P, int gi, int pass, int64_t t, int c) {
  const PersistGroupArgs &g = P.p.g[gi];
  const int64_t e = t + c;
  switch (pass) {
    case 0:
      zfwd_body<float, N, kPV>(g.zf, t, 1, e);
      return true;
    case 1:
      return axis_body<float, N, kPV, kAxisFwd, false, kFiltNone>(P.maps[gi][0], g.ax[0], t, 1, e);
    case 2:
      return axis_body<float, N, kPV, kAxisFwdInv, false, kFiltInterp>(P.maps[gi][1], g.ax[1], t, 1, e);
    case 3:
    case 4:
      return axis_body<float, N, kPV, kAxisInv>(P.maps[gi][pass - 1], g.ax[pass - 1], t, 1, e);
    case 5:
    case 6:
      return g.plain ? zinv_body<float, N, kPV, false, kZPosVel>(g.zi[pass - 5], t, 1, e)
                     : zinv_body<float, N, kPV>(g.zi[pass - 5], t, 1, e);
    default:
      return g.plain ? zinv_body<float, N, kPV, false, kZPosVelZ>(g.zi[2], t, 1, e)
                     : zinv_body<float, N, kPV>(g.zi[2], t, 1, e);
  }
}

__global__ void __launch_bounds__(kThreads, 2) k_persist(const __grid_constant__ PersistParams P) {
  __shared__ int s_pass, s_group;
  __shared__ long long s_tile;
  const int tid = threadIdx.x;
  unsigned *counters = P.p.counters;
  unsigned *done = counters + kCounterBase;
  for (;;) {
    if (tid == 0) {
      int pass = -1, gi = 0;
      int64_t t = 0;
      const int64_t item = (int64_t)atomicAdd(&counters[0], 1u);
      if (item < P.total && !ld_acquire(&counters[1])) {
        for (int s = 0; s < kPersistPasses; ++s)
          for (int g = 0; g < P.p.ngroups; ++g)
            if (item >= P.base[s][g] && item < P.base[s][g] + P.items[s][g]) {
              pass = s;
              gi = g;
            }
        t = item - P.base[pass][gi];
        const int dp = kDep[pass];
        if (dp >= 0) {  // the realization's previous pass must be complete
          const int64_t rr = t / P.per_real[pass][gi];
          const unsigned need = (unsigned)P.per_real[dp][gi];
          const unsigned *c = done + (size_t)(P.p.g[gi].first + rr) * kPersistPasses + dp;
          if (ld_acquire(c) < need) {
            const uint64_t t0 = global_ns();
            const uint64_t lim = 1000ull * (P.p.wait_us ? P.p.wait_us : 2000000u);
            while (ld_acquire(c) < need) {
              if (ld_acquire(&counters[1])) {
                pass = -1;
                break;
              }
              if (global_ns() - t0 > lim) {
                atomicExch(P.p.err, 2);
                atomicExch(&counters[1], 1u);
                pass = -1;
                break;
              }
              __nanosleep(128);
            }
          }
          // the tile's copies (async proxy) read what other CTAs stored
          asm volatile("fence.proxy.async.global;" ::: "memory");
        }
      }
      s_pass = pass;
      s_group = gi;
      s_tile = t;
    }
    __syncthreads();
    const int pass = s_pass, gi = s_group;
    const int64_t t = s_tile;  // the item's number within its pass and group
    if (pass < 0) break;
    const int c = P.chunk[pass][gi];
    bool ok = true;
    switch (P.p.g[gi].n) {
      case 64: ok = persist_item<64>(P, gi, pass, t * c, c); break;
      case 128: ok = persist_item<128>(P, gi, pass, t * c, c); break;
      case 192: ok = persist_item<192>(P, gi, pass, t * c, c); break;
      case 256: ok = persist_item<256>(P, gi, pass, t * c, c); break;
      default: ok = persist_item<384>(P, gi, pass, t * c, c); break;
    }
    __threadfence();  // this thread's stores of the tile, before the count
    __syncthreads();
    if (tid == 0) {
      if (!ok) {
        atomicExch(&counters[1], 1u);
      } else if (!(P.p.test_stall && pass == 1 && gi == 0 && t == 0)) {  // fault test: stall
        __threadfence();
        const int64_t rr = t / P.per_real[pass][gi];
        atomicAdd(&done[(size_t)(P.p.g[gi].first + rr) * kPersistPasses + pass], 1u);
      }
    }
  }
}

// Tile shapes, tile counts and shared memory of one group (size N).
template <int N>
void shape_group(PersistGroupArgs &g, int64_t tiles[kPersistPasses], size_t *smem) {
  using AP = ct::AxisPolicy<float, N, kPV>;
  using ZP = ct::ZPolicy<float, N, kPV>;
  for (auto &a : g.ax) {
    a.cols = AP::B;
    a.inner_chunks = (N / 2) / AP::B;
    a.rows_box = AP::ROWS_BOX;
    a.e = AP::E;
    a.variant = kPV;
  }
  g.zf.lines_per_cta = ZP::L;
  g.zf.variant = kPV;
  for (auto &z : g.zi) {
    z.lines_per_cta = ZP::L;
    z.variant = kPV;
  }
  const int64_t lines = (int64_t)g.nb * N * N;
  const int64_t axis_tiles = (int64_t)g.nb * N * ((N / 2) / AP::B);
  tiles[0] = lines / ZP::L;
  for (int s = 1; s < 5; ++s) tiles[s] = axis_tiles;
  for (int j = 0; j < 3; ++j) tiles[5 + j] = g.zi_on[j] ? lines / ZP::L : 0;
  const size_t tile = ((size_t)N * AP::B * 8 + 127) & ~(size_t)127;
  const size_t axis = 128 + 2 * tile + kInterpExact * 4 + (size_t)g.ax[1].interp_cells * 16;
  const size_t zinv = 128 + (((size_t)ZP::DENSE * 8 + 127) & ~(size_t)127) + (size_t)ZP::WORK_INV * 8;
  const size_t zfwd = (size_t)ZP::WORK_FWD * 8;
  size_t m = axis > zinv ? axis : zinv;
  m = m > zfwd ? m : zfwd;
  *smem = *smem > m ? *smem : m;
}

}  // namespace

bool persist_has(int n) { return n == 64 || n == 128 || n == 192 || n == 256 || n == 384; }

cudaError_t launch_persist(PersistPlan p, cudaStream_t s, int *launched_blocks) {
  static PersistParams P;  // host staging of the kernel parameters (large: kept off the stack)
  std::memset(&P, 0, sizeof P);
  if (p.ngroups < 1 || p.ngroups > kPersistMaxGroups) return cudaErrorInvalidValue;
  size_t smem = 0;
  for (int gi = 0; gi < p.ngroups; ++gi) {
    PersistGroupArgs &g = p.g[gi];
    int64_t tiles[kPersistPasses];
    switch (g.n) {
      case 64: shape_group<64>(g, tiles, &smem); break;
      case 128: shape_group<128>(g, tiles, &smem); break;
      case 192: shape_group<192>(g, tiles, &smem); break;
      case 256: shape_group<256>(g, tiles, &smem); break;
      case 384: shape_group<384>(g, tiles, &smem); break;
      default: return cudaErrorInvalidValue;
    }
    for (int k = 0; k < 4; ++k) {
      const cudaError_t e = make_map<float>(&P.maps[gi][k], g.ax[k]);
      if (e != cudaSuccess) return e;
    }
    for (int ps = 0; ps < kPersistPasses; ++ps) {
      const int64_t per = tiles[ps] / g.nb;  // tiles of one realization
      int c = p.chunk > 0 ? p.chunk : kChunk;
      while (c > 1 && per % c) c /= 2;
      P.chunk[ps][gi] = c;
      P.items[ps][gi] = tiles[ps] / c;
      P.per_real[ps][gi] = per / c;
    }
  }
  int64_t item = 0;
  for (int ps = 0; ps < kPersistPasses; ++ps)
    for (int gi = 0; gi < p.ngroups; ++gi) {
      P.base[ps][gi] = item;
      item += P.items[ps][gi];
    }
  if (item >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;
  P.total = item;
  P.p = p;
  cudaError_t e = set_smem(k_persist, smem);
  if (e != cudaSuccess) return e;
  const int blocks = persistent_blocks(k_persist, kThreads, smem, item);
  if (launched_blocks) *launched_blocks = blocks;
  k_persist<<<blocks, kThreads, smem, s>>>(P);
  return cudaGetLastError();
}

}  // namespace gg
