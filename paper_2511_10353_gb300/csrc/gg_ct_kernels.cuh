// Size-specialised kernels of the three transform passes (see gg_ct.cuh).
// Included by gg_ct_f32.cu / gg_ct_f64.cu, which instantiate them for the
// grid sizes of the named workloads; every other size runs the run-time
// kernels of gg_kernels.cuh.
#pragma once

#include "gg_ct.cuh"
#include "gg_launch.cuh"

namespace gg {

__device__ __forceinline__ int ct_freq(int n, int N) { return n < (N >> 1) ? n : n - N; }

// ------------------------------------------------------------ strided pass
// The pass of k_axis (gg_kernels.cuh) with N and the tile width fixed:
// persistent CTAs, TMA double buffering, forward stages in place in shared
// memory, the spectrum handed to the inverse stages in registers, each
// inverse's last stage storing straight to HBM.
// Where the handed-off spectrum and an inverse do not both fit the register
// budget (Pol::SPILL), the spectrum is parked in the tile buffer at its
// natural positions (each thread reads back only what it wrote) and every
// output reads it from there. With several outputs the second buffer is then
// the inverse work buffer, and the next tile's copy is issued into the first
// once the last output has read the spectrum, overlapping that output's
// inverse stages: all outputs come from one launch.
// MODE (kAxisFwd, kAxisInv, kAxisFwdInv) fixes at compile time which halves
// run (the flags a.fwd, a.inv are not read): each kernel holds only its path.
// FILT: how the handed-off spectrum is filtered: kFiltArgs as a.pre and
// a.interp say, kFiltNone never (the forward y pass), kFiltInterp always by the
// interpolated FP32 table at a.interp (the fused x pass of the plain path).
constexpr int kAxisFwd = 1, kAxisInv = 2, kAxisFwdInv = 3;
constexpr int kFiltArgs = 0, kFiltNone = 1, kFiltInterp = 2;
// The body processes tiles t0, t0 + tstep, ... below tlimit (the kernel: its
// CTA's share of all tiles; the persistent batched kernel: one tile). It
// returns false when a copy wait gave up (the error word then holds
// GG_ETIMEOUT). `map` must live in parameter (grid-constant) memory.
// TST: the inverse outputs go through the staging tile and TMA stores
// (smap0 / smap1: the tensor maps of dst[0] / dst[1], in parameter memory).
template <typename R, int N, int V, int MODE, bool CUT = false, int FILT = kFiltArgs>
__host__ __device__ constexpr bool axis_tma_store() {
  return MODE != kAxisFwd && ct::AxisPolicy<R, N, V>::tma_st(FILT != kFiltNone && sizeof(R) == 4);
}
// (only where the register budget is tight, Pol::SPILL: at 512 the plain
// stores measured faster, 0.170 against 0.178 ms)
template <typename R, int N, int V, int MODE>
__host__ __device__ constexpr bool axis_tma_store_fwd() {
  return MODE == kAxisFwd && V != ct::kPersistV && ct::nstages(ct::skey<R>(N)) > 1 &&
         ct::AxisPolicy<R, N, V>::SPILL;
}
template <typename R, int N, int V, int MODE, bool CUT = false, int FILT = kFiltArgs>
__host__ __device__ constexpr bool axis_tma_store_inplace() {
  using Pol = ct::AxisPolicy<R, N, V>;
  return MODE != kAxisFwd && (Pol::SPILL || Pol::THREE) && V != ct::kPersistV &&
         ct::nstages(ct::skey<R>(N)) > 1 &&
         !ct::fuse_pair<R, N, Pol::E>() && !axis_tma_store<R, N, V, MODE, CUT, FILT>();
}
template <typename R, int N, int V, int MODE, bool CUT = false, int FILT = kFiltArgs>
__device__ __forceinline__ bool axis_body(const CUtensorMap &map, const AxisArgs &a, int64_t t0,
                                          int64_t tstep, int64_t tlimit,
                                          const CUtensorMap *smap0 = nullptr,
                                          const CUtensorMap *smap1 = nullptr) {
  using C = Cx<R>;
  constexpr bool FWD = MODE != kAxisInv, INV = MODE != kAxisFwd;
  using Pol = ct::AxisPolicy<R, N, V>;
  constexpr bool TST = axis_tma_store<R, N, V, MODE, CUT, FILT>();
  constexpr int K = ct::skey<R>(N);
  constexpr int B = Pol::B, E = Pol::E, P = Pol::P, HALF = N / 2, S = ct::nstages(K);
  constexpr int TILE = N * B;
  constexpr int TILE_STRIDE = (int)(((TILE * sizeof(C) + 127) / 128) * 128 / sizeof(C));
  constexpr int INNER = HALF / B;
  constexpr int RH = ct::radix_of(K, 0, true);  // radix at the register hand-off
  static_assert(RH == ct::radix_of(K, S - 1, false), "hand-off radix");
  constexpr int SPAN = N / RH, NB = E / RH;
  constexpr bool SPILL = Pol::SPILL;
  constexpr bool FUSE = ct::fuse_pair<R, N, E>();  // stage pairs around the hand-off in registers
  // TSI: with the spectrum parked (no room for a staging tile), each inverse
  // output's last stage runs in place in the work buffer and a TMA store
  // copies it out; the buffer is rewritten once that store has read it
  constexpr bool TSI = axis_tma_store_inplace<R, N, V, MODE, CUT, FILT>();
  // TSF: forward only, the spectrum back into the tile buffer and out by TMA
  constexpr bool TSF = axis_tma_store_fwd<R, N, V, MODE>();
  constexpr bool TMA_OUT = TST || TSI || TSF;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw);
  C *bufs = reinterpret_cast<C *>(smem_raw + 128);
  // TST: the staging tile after the two tiles; then the interpolated filter
  // (FP32): exact values, then Hermite cells
  constexpr int NT = TST ? 3 : 2;
  C *stg = bufs + 2 * TILE_STRIDE;
  float *f_exact = reinterpret_cast<float *>(bufs + NT * TILE_STRIDE);
  float4 *f_cells = reinterpret_cast<float4 *>(f_exact + kInterpExact);
  const int tid = threadIdx.x;
  const int64_t per_real = (int64_t)N * INNER;
  const int64_t ntiles = per_real * (a.nbatch > 0 ? a.nbatch : 1);
  const R *table = reinterpret_cast<const R *>(a.table);
  static_assert(FILT != kFiltInterp || sizeof(R) == 4, "interpolated filter: FP32");
  const bool pre = FILT == kFiltArgs ? a.pre != 0 : FILT == kFiltInterp;
  const bool interp = FILT == kFiltArgs ? sizeof(R) == 4 && a.pre && a.interp : FILT == kFiltInterp;
  // large radices: the N twiddles in shared memory (15-31 loads a butterfly),
  // after the tiles and the filter table
  constexpr bool TW_SMEM = ct::AxisPolicy<R, N, V>::TW_SMEM;
  C *tw_s = bufs + NT * TILE_STRIDE + (interp ? (kInterpExact + 4 * kMaxInterpCells(N)) / 2 : 0);
  if constexpr (TW_SMEM) {
    const C *src = reinterpret_cast<const C *>(a.tw);
    for (int i = tid; i < N; i += blockDim.x) tw_s[i] = src[i];
  }
  const ct::Tw<C, TW_SMEM> tw{TW_SMEM ? tw_s : reinterpret_cast<const C *>(a.tw)};
  if (interp) {
    const float *src = reinterpret_cast<const float *>(a.interp);
    for (int i = tid; i < kInterpExact; i += blockDim.x) f_exact[i] = src[i];
    const float4 *cs = reinterpret_cast<const float4 *>(src + kInterpExact);
    for (int i = tid; i < a.interp_cells; i += blockDim.x) f_cells[i] = cs[i];
  }
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  // tile t -> (realization, outer index, chunk of columns). The x pass walks
  // a chunk-major source chunk-outer, so that concurrent tiles share pages;
  // the y passes keep the outer-major order, in which concurrent tiles write
  // adjacent columns of the plain layout.
  const bool cin = a.chunked_in != 0;
  const bool chunk_outer = cin && a.axis == 0;
  auto decode = [&](int64_t t, int64_t &rr, int64_t &outer, int &chunk) {
    rr = t / per_real;
    const int64_t tt = t - rr * per_real;
    if (chunk_outer) {
      chunk = (int)(tt / N);
      outer = tt - (int64_t)chunk * N;
    } else {
      outer = tt / INNER;
      chunk = (int)(tt - outer * INNER);
    }
  };
  auto issue = [&](int64_t t, int sb) {
    int64_t rr, outer;
    int chunk;
    decode(t, rr, outer, chunk);
    C *dst = bufs + sb * TILE_STRIDE;
    if (a.test_skip_copy) return;  // fault test: the wait for this tile runs out
    mbar_arrive_expect_tx(&bars[sb], (uint32_t)(TILE * sizeof(C)));
#pragma unroll
    for (int i = 0; i < N; i += Pol::ROWS_BOX) {
      if (cin) {
        if (a.axis == 1) tma_load_5d(dst + i * B, &map, &bars[sb], 0, i, (int)outer, chunk, (int)rr);
        else tma_load_5d(dst + i * B, &map, &bars[sb], 0, (int)outer, i, chunk, (int)rr);
      } else if (a.axis == 1) {
        tma_load_4d(dst + i * B, &map, &bars[sb], chunk * B * 2, i, (int)outer, (int)rr);
      } else {
        tma_load_4d(dst + i * B, &map, &bars[sb], chunk * B * 2, (int)outer, i, (int)rr);
      }
    }
  };
  // late: one input buffer (0) and one work buffer (1); the copy of the next
  // tile is issued during the last output
  const bool late = SPILL && INV && a.nout > 1;
  if (tlimit > ntiles) tlimit = ntiles;
  int64_t t = t0;
  if (tid == 0 && t < tlimit) issue(t, 0);
  for (int it = 0; t < tlimit; t += tstep, ++it) {
    const int sb = late ? 0 : it & 1;
    const uint32_t phase = late ? (uint32_t)(it & 1) : (uint32_t)((it >> 1) & 1);
    const int64_t tn = t + tstep;
    // the next tile's copy, into the other buffer; TSI with one output: later,
    // once the previous tile's output store (from that buffer) has read it
    const bool ahead = !late && !TSI && !TSF;
    if (tid == 0 && tn < tlimit && ahead) {
      fence_proxy_async_smem();
      issue(tn, sb ^ 1);
    }
    int c = tid & (B - 1), p = tid / B;
    asm volatile("" : "+r"(c), "+r"(p));
    __builtin_assume(c >= 0 && c < B && p >= 0 && p < P);
    int64_t rr, outer;
    int chunk;
    decode(t, rr, outer, chunk);
    const int kz = chunk * B + c;
    C *buf = bufs + sb * TILE_STRIDE;
    C *wb = late ? bufs + TILE_STRIDE : buf;  // the inverse work buffer
    // outputs: the plain layout, or chunk-major (rows B apart along y, N B along x)
    const int64_t gbase =
        a.chunked_out ? rr * a.batch_stride + (a.axis == 1 ? ((int64_t)chunk * N + outer) * N * B
                                                           : ((int64_t)chunk * N * N + outer) * B) + c
                      : rr * a.batch_stride + outer * a.outer_stride + kz;
    const int64_t ostride = a.chunked_out ? (a.axis == 1 ? (int64_t)B : (int64_t)N * B) : a.stride;
    const int m_outer = a.axis == 0 ? ct_freq((int)outer, N) : 0;
    const bool nyq_outer = a.axis == 0 && (int)outer == HALF;
    auto tab_index = [&](int n) {
      const int m = ct_freq(n, N);
      return (n == HALF || nyq_outer) ? -1 : m * m + m_outer * m_outer + kz * kz;
    };
    if (pre && !interp) {
#pragma unroll
      for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int r = 0; r < RH; ++r) {
          const int q = tab_index(p + P * b + r * SPAN);
          if (q >= 0) prefetch_l1(table + q);
        }
    }
    const bool ok = __syncthreads_and(mbar_wait(&bars[sb], phase, a.err, a.wait_us));
    if (!ok) {  // late: no other copy is in flight
      if (tid == 0 && tn < tlimit && ahead && !a.test_skip_copy)
        mbar_wait(&bars[sb ^ 1], (uint32_t)(((it + 1) >> 1) & 1), nullptr, a.wait_us);
      if constexpr (TMA_OUT) {
        if (tid == 0) bulk_wait0();  // the output stores, before the CTA exits
      }
      return false;
    }
    auto ld_smem = [&](int n) { return buf[n * B + c]; };
    auto st_smem = [&](int n, C v) { buf[n * B + c] = v; };
    auto ld_work = [&](int n) { return wb[n * B + c]; };
    auto st_work = [&](int n, C v) { wb[n * B + c] = v; };
    // SPILL, inverse only, no filter: the spectrum is already parked
    const bool x_regs = !SPILL || FWD || pre || !INV;
    // the outputs by TMA: tile rows at the load's coordinates, from src_t
    auto tma_out = [&](const C *src_t, int o) {
      const CUtensorMap *sm = o == 0 ? smap0 : smap1;
#pragma unroll
      for (int i = 0; i < N; i += Pol::ROWS_BOX) {
        if (a.chunked_out) {
          if (a.axis == 1) tma_store_5d(sm, src_t + i * B, 0, i, (int)outer, chunk, (int)rr);
          else tma_store_5d(sm, src_t + i * B, 0, (int)outer, i, chunk, (int)rr);
        } else if (a.axis == 1) {
          tma_store_4d(sm, src_t + i * B, chunk * B * 2, i, (int)outer, (int)rr);
        } else {
          tma_store_4d(sm, src_t + i * B, chunk * B * 2, (int)outer, i, (int)rr);
        }
      }
      bulk_commit();
    };
    // TSF: the next tile's copy once the forward's first stages have run (the
    // previous tile's store has read that buffer by then)
    auto issue_after_stages = [&]() {
      if constexpr (TSF) {
        if (tid == 0 && tn < tlimit) {
          bulk_wait_read0();
          fence_proxy_async_smem();
          issue(tn, sb ^ 1);
        }
      }
    };
    C X[E];
    if constexpr (FWD) {
      if constexpr (FUSE) {
        if ((S - 2) % 2 == 0 && late)  // the work buffer is free: ping-pong, ending in buf
          ct::stages_pingpong<R, N, E, false, 0, S - 2>(p, tw, ld_smem, st_smem, ld_work, st_work);
        else
          ct::stages<R, N, E, false, 0, S - 2>(p, tw, ld_smem, st_smem);
        issue_after_stages();
        ct::last_two_stages_regs<R, N, E>(p, tw, ld_smem, X);
      } else {
        ct::stages<R, N, E, false, 0, S - 1>(p, tw, ld_smem, st_smem);
        issue_after_stages();
        ct::last_stage_regs<R, N, E, false>(p, tw, ld_smem, X);
      }
    } else if (x_regs) {
#pragma unroll
      for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int r = 0; r < RH; ++r) X[b * RH + r] = buf[(p + P * b + r * SPAN) * B + c];
    }
    if (pre) {
#pragma unroll
      for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int r = 0; r < RH; ++r) {
          const int q = tab_index(p + P * b + r * SPAN);
          R f;
          if (q < 0) {
            f = (R)0;
          } else if (!interp) {
            f = __ldg(table + q);
          } else if (q < kInterpExact) {
            f = (R)f_exact[q];
          } else {  // cubic Hermite in m = sqrt(m2), unit cells, Horner form
            const float mf = (float)q;
            const float m = mf * rsqrtf(mf);
            const int j = (int)m;
            const float t = m - (float)j;
            const float4 cc = f_cells[j - kInterpFirstCell];
            f = (R)fmaf(t, fmaf(t, fmaf(t, cc.w, cc.z), cc.y), cc.x);
          }
          if constexpr (CUT) {
            if (q < a.qmin) f = (R)0;  // Eq. 4: large scales removed
          }
          X[b * RH + r] = C{f * X[b * RH + r].x, f * X[b * RH + r].y};
        }
    }
    if constexpr (!INV) {  // forward only: the spectrum to dst[0]
      if constexpr (TSF) {
        __syncthreads();  // the last stage has read the tile: it becomes the output tile
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
          for (int r = 0; r < RH; ++r) buf[(p + P * b + r * SPAN) * B + c] = X[b * RH + r];
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) tma_out(buf, 0);
      } else {
        C *d = reinterpret_cast<C *>(a.dst[0]) + gbase;
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
          for (int r = 0; r < RH; ++r) d[(int64_t)(p + P * b + r * SPAN) * ostride] = X[b * RH + r];
        __syncthreads();
      }
      continue;
    }
    if constexpr (SPILL) {
      if constexpr (FWD) __syncthreads();  // the forward's last stage has read the tile
      if (x_regs) {
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
          for (int r = 0; r < RH; ++r) buf[(p + P * b + r * SPAN) * B + c] = X[b * RH + r];
      }
    } else {
      __syncthreads();  // the tile is in registers: buf becomes the inverse work buffer
    }
    for (int o = 0; o < a.nout; ++o) {
      asm volatile("" : "+r"(c), "+r"(p));
      __builtin_assume(c >= 0 && c < B && p >= 0 && p < P);
      C *d = reinterpret_cast<C *>(a.dst[o]) + gbase;
      auto st_glob = [&](int n, C v) { d[(int64_t)n * ostride] = v; };
      C W[E];
      const bool im = a.mul[o] == kMulIm;
#pragma unroll
      for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int r = 0; r < RH; ++r) {
          const int n = p + P * b + r * SPAN;
          const C v = SPILL ? buf[n * B + c] : X[b * RH + r];
          const R f = n == HALF ? (R)0 : (R)ct_freq(n, N);
          W[b * RH + r] = im ? C{-f * v.y, f * v.x} : v;
        }
      if constexpr (FUSE) {
        ct::inverse_head_regs<R, N, E>(tw, W);  // inverse stages 0 and 1
      } else {
#pragma unroll
        for (int b = 0; b < NB; ++b) Butterfly<RH, true, C>::run(&W[b * RH]);  // inverse stage 0
      }
      // the previous output's last stage has read the work buffer; SPILL with
      // one buffer: every thread has read its parked spectrum; TSI: the
      // previous output's store has read the work buffer
      if constexpr (TSI) {
        if (tid == 0) bulk_wait_read0();
        __syncthreads();
        if (!late && o == 0 && tid == 0 && tn < tlimit) {  // the other buffer is free now
          fence_proxy_async_smem();
          issue(tn, sb ^ 1);
        }
      } else {
        // (TST: the previous output ended with a barrier after its last stage)
        if (!TST && (o > 0 || (SPILL && !late))) __syncthreads();
      }
      if (late && o == a.nout - 1 && tid == 0 && tn < tlimit) {  // the input buffer is free
        fence_proxy_async_smem();
        issue(tn, 0);
      }
      // TST: the last stage writes the staging tile, which the previous
      // output's stores must have finished reading (checked by their issuing
      // thread before the barrier ahead of the remaining stages)
      auto st_stg = [&](int n, C v) { stg[n * B + c] = v; };
      if constexpr (S == 1) {
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
          for (int r = 0; r < RH; ++r) st_glob((p + P * b) * RH + r, W[b * RH + r]);
      } else if constexpr (FUSE) {
        ct::inverse_head_store<R, N, E>(p, W, st_work);
        if constexpr (TST) {
          if (tid == 0) bulk_wait_read0();
        }
        __syncthreads();
        ct::stages<R, N, E, true, 2, S - 1>(p, tw, ld_work, st_work);
        if constexpr (TST) ct::stage<R, N, E, S - 1, true, ct::kSyncNone>(p, tw, ld_work, st_stg);
        else ct::stage<R, N, E, S - 1, true, ct::kSyncNone>(p, tw, ld_work, st_glob);
      } else {
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
          for (int r = 0; r < RH; ++r) wb[((p + P * b) * RH + r) * B + c] = W[b * RH + r];
        if constexpr (TST) {
          if (tid == 0) bulk_wait_read0();
        }
        __syncthreads();
        ct::stages<R, N, E, true, 1, S - 1>(p, tw, ld_work, st_work);
        if constexpr (TST) {
          ct::stage<R, N, E, S - 1, true, ct::kSyncNone>(p, tw, ld_work, st_stg);
        } else if constexpr (TSI) {  // in place: loads, barrier, stores, fence, barrier
          ct::stage<R, N, E, S - 1, true, ct::kSyncCtaAsync>(p, tw, ld_work, st_work);
        } else {
          ct::stage<R, N, E, S - 1, true, ct::kSyncNone>(p, tw, ld_work, st_glob);
        }
      }
      if constexpr (TMA_OUT) {  // the tile to dst[o] by TMA, once every thread's values are in
        const C *src_t = TST ? stg : wb;
        if constexpr (TST) {
          fence_proxy_async_smem();
          __syncthreads();
        }
        if (tid == 0) tma_out(src_t, o);
      }
    }
    // (TST: the last output's barrier after its last stage already ordered
    // every access to the tile buffers before the next copy into them)
    if constexpr (!TST) __syncthreads();
  }
  if constexpr (TMA_OUT) {
    if (tid == 0) bulk_wait0();  // the output stores, before the CTA exits
  }
  __syncthreads();
  if (tid == 0) {  // the caller may reuse the shared memory
    mbar_inval(&bars[0]);
    mbar_inval(&bars[1]);
  }
  return true;
}

template <typename R, int N, int V, int MODE, bool CUT = false, int FILT = kFiltArgs>
__global__ void __launch_bounds__(ct::AxisPolicy<R, N, V>::THREADS, ct::AxisPolicy<R, N, V>::MINB)
    k_axis_ct(const __grid_constant__ CUtensorMap map, const __grid_constant__ CUtensorMap smap0,
              const __grid_constant__ CUtensorMap smap1, const AxisArgs a) {
  axis_body<R, N, V, MODE, CUT, FILT>(map, a, blockIdx.x, gridDim.x, INT64_MAX, &smap0, &smap1);
}

// ------------------------------------------------------------ z passes
// Padded line layout of the z-pass work tile: element n of line l at
// l * LD + n + n / PAD (PAD a power of two or 0: no padding; pairs
// (2q, 2q+1) never straddle a pad).
template <int LD, int PAD> __device__ __forceinline__ int zpad(int l, int n) {
  if constexpr (PAD == 0) return l * LD + n;
  else return l * LD + n + (int)((unsigned)n / PAD);
}

// Inverse z pass (c2r) + Eq. 3 epilogue, persistent: one thread bulk-copies
// a block of L contiguous half-spectrum lines into a dense shared buffer. The
// c2r pre-processing moves it into the padded work tile (where the first two
// inverse stages pair up, through them in registers: the pre-processing
// yields exactly the first stage's inputs), after which the buffer is free
// and the copy of the CTA's next block starts; it lands while the transform
// and the epilogue of the current block run. The last stage's outputs
// (natural order) feed the epilogue from registers.
// EXT: the Sec. 2.4 merge (large) and the Sec. 2.2 particle options (shift,
// pos2), compiled only into the extended instantiation.
// OUT: 0 reads the outputs and the component from the arguments; kZPosVel
// (x or y component) and kZPosVelZ (z component, i m_z) fix the plain
// path's pos + vel outputs at compile time (no psi, no accumulation; with
// per-realization lists, every entry set).
constexpr int kZPosVel = 1, kZPosVelZ = 2;
template <typename R, int N, int V, bool EXT = false, int OUT = 0>
__device__ __forceinline__ bool zinv_body(const ZInvArgs &a, int64_t t0, int64_t tstep,
                                          int64_t tlimit) {
  using C = Cx<R>;
  using Pol = ct::ZPolicy<R, N, V>;
  constexpr int M = Pol::M, E = Pol::E, P = Pol::P, L = Pol::L, LD = Pol::LD_INV, PAD = Pol::PAD_INV;
  constexpr int KM = ct::skey<R>(M);
  constexpr int S = ct::nstages(KM);
  constexpr int RL = ct::radix_of(KM, S - 1, true), SPANL = M / RL, NBL = E / RL;
  // stages of the inverse done in registers straight from the c2r
  // pre-processing (which yields exactly the first stage's inputs): two
  // where a thread holds whole butterflies of both, one for the 768-point
  // lines (8 x 8 x 12: measured 8.35 -> 7.27 ms at N = 1536; at M = 256 the
  // register-resident first stage was slower, 0.262 -> 0.282 ms)
  constexpr int HEAD = Pol::FUSE ? 2 : (S >= 3 && M >= 768 ? 1 : 0);
  constexpr int DENSE_STRIDE = (int)(((Pol::DENSE * sizeof(C) + 127) / 128) * 128 / sizeof(C));
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
  C *dense = reinterpret_cast<C *>(smem_raw + 128);
  C *work = dense + DENSE_STRIDE;
  const int tid = threadIdx.x;
  const int64_t ntiles = a.nlines / L;
  const ct::Tw<C, false> tw_half{reinterpret_cast<const C *>(a.tw_half)};
  const C *twf = reinterpret_cast<const C *>(a.tw_full);
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  auto issue = [&](int64_t t) {
    mbar_arrive_expect_tx(bar, (uint32_t)(Pol::DENSE * sizeof(C)));
    bulk_load(dense, reinterpret_cast<const C *>(a.src) + t * Pol::DENSE,
              (uint32_t)(Pol::DENSE * sizeof(C)), bar);
  };
  const R box = (R)a.box, cell = (R)a.cell, qo = (R)a.q_offset, vfac = (R)a.vfac;
  if (tlimit > ntiles) tlimit = ntiles;
  int64_t t = t0;
  if (tid == 0 && t < tlimit) issue(t);
  for (int it = 0; t < tlimit; t += tstep, ++it) {
    const int64_t tn = t + tstep;
    int l = tid / P, p = tid - (tid / P) * P;
    asm volatile("" : "+r"(l), "+r"(p));
    const bool ok = __syncthreads_and(mbar_wait(bar, (uint32_t)(it & 1), a.err));
    if (!ok) return false;  // nothing else in flight: the next copy is issued after this wait
    const C *dl = dense + l * M;
    const R pf = (R)p;  // (R)(p + c) == pf + (R)c exactly: small integers
    auto ld_w = [&](int n) { return work[zpad<LD, PAD>(l, n)]; };
    auto st_w = [&](int n, C v) { work[zpad<LD, PAD>(l, n)] = v; };
    C v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int k = p + P * i;
      C xk = dl[k];
      C xm = k ? dl[M - k] : C{(R)0, (R)0};
      if (OUT == 0 ? a.mul_kz != 0 : OUT == kZPosVelZ) {  // i m_z on both members of the pair
        const R kf = pf + (R)(P * i), mf = (R)M - kf;
        xk = C{mul_rn(-kf, xk.y), mul_rn(kf, xk.x)};
        xm = C{mul_rn(-mf, xm.y), mul_rn(mf, xm.x)};
      }
      const C s = {xk.x + xm.x, xk.y - xm.y};  // X_k + conj X_{M-k}
      const C d = {xk.x - xm.x, xk.y + xm.y};  // X_k - conj X_{M-k}
      const C z = cadd(s, mul_pi(cmulc(d, ldg_c(twf + k))));
      if constexpr (HEAD > 0) {  // k = p + P*(b + (E/RA)*r): the first stage's layout
        constexpr int RA = ct::radix_of(KM, 0, true), NBA = E / RA;
        v[(i % NBA) * RA + i / NBA] = z;
      } else {
        st_w(k, z);
      }
    }
    if constexpr (HEAD == 2) {  // the inverse's first two stages in registers
      ct::inverse_head_regs<R, M, E>(tw_half, v);
      ct::inverse_head_store<R, M, E>(p, v, st_w);
    } else if constexpr (HEAD == 1) {  // the first stage (no twiddles: NS = 1) in registers
      constexpr int RA = ct::radix_of(KM, 0, true), NBA = E / RA;
#pragma unroll
      for (int b = 0; b < NBA; ++b) {
        Butterfly<RA, true, C>::run(&v[b * RA]);
#pragma unroll
        for (int r = 0; r < RA; ++r) st_w((p + P * b) * RA + r, v[b * RA + r]);
      }
    }
    __syncthreads();
    if (tid == 0 && tn < tlimit) {  // the dense buffer has been read: fetch the next block
      fence_proxy_async_smem();
      issue(tn);
    }
    ct::stages<R, M, E, true, HEAD, S - 1, Pol::SY | ct::kNoRangeHint>(p, tw_half, ld_w, st_w);
    ct::last_stage_regs<R, M, E, true, false>(p, tw_half, ld_w, v);
    // line -> (realization, x, y): line counts stay below 2^32 (N <= 4096, the
    // host bounds the batch), so 32-bit divisions suffice
    const uint32_t line = (uint32_t)(t * L + l);
    const uint32_t lpr = (uint32_t)(a.lines_per_real > 0 ? a.lines_per_real : a.nlines);
    const uint32_t rr = line / lpr, local = line - rr * lpr;
    const uint32_t ix = local / (uint32_t)a.n, iy = local - ix * (uint32_t)a.n;
    const int comp = OUT == 0 ? a.comp : (OUT == kZPosVelZ ? 2 : a.comp);
    const R qline = mul_rn(comp == 0 ? (R)ix + qo : (R)iy + qo, cell);
    const R q2p = (R)(2 * p);  // (R)(2n) == q2p + (R)(2n - 2p) exactly
    void *psi_b = OUT ? nullptr : (a.psi_list ? a.psi_list[rr] : a.psi);
    void *pos_b = a.pos_list ? a.pos_list[rr] : a.pos;
    void *vel_b = a.vel_list ? a.vel_list[rr] : a.vel;
    const int64_t off = (int64_t)(((!OUT && a.psi_list) || a.pos_list || a.vel_list) ? local : line) * M;
    C *psi = psi_b ? reinterpret_cast<C *>(psi_b) + off : nullptr;
    C *pos = pos_b ? reinterpret_cast<C *>(pos_b) + off : nullptr;
    C *vel = vel_b ? reinterpret_cast<C *>(vel_b) + off : nullptr;
    const R *large = EXT ? reinterpret_cast<const R *>(a.large) : nullptr;
    C *pos2 = EXT && a.pos2 ? reinterpret_cast<C *>(a.pos2) + off : nullptr;
    const R sh1 = EXT ? (R)a.shift : (R)0, sh2 = EXT ? (R)a.shift2 : (R)0;
    CicAxis<R> cx{}, cy{};
    if (EXT && large) {
      cx = cic_axis<R>((int)ix, a.n_low, N);
      cy = cic_axis<R>((int)iy, a.n_low, N);
    }
#pragma unroll
    for (int b = 0; b < NBL; ++b)
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        const int n = p + P * b + r * SPANL;
        C z = v[b * RL + r];
        if constexpr (EXT) {  // Sec. 2.4: the interpolated coarse large scales
          if (large) {
            R l0, l1;
            cic_pair<R>(large, a.n_low, N, cx, cy, n, l0, l1);
            z.x += l0;
            z.y += l1;
          }
        }
        if (!OUT && psi) {
          if (a.accumulate) {
            const C o = psi[n];
            psi[n] = C{o.x + (R)a.alpha * z.x, o.y + (R)a.alpha * z.y};
          } else {
            psi[n] = z;
          }
        }
        if (OUT || pos) {
          R q0 = qline, q1 = qline;
          if (comp == 2) {
            q0 = mul_rn(q2p + (R)(2 * (n - p)) + qo, cell);
            q1 = mul_rn(q2p + (R)(2 * (n - p) + 1) + qo, cell);
          }
          if constexpr (EXT) {  // Sec. 2.2: periodic shift; gas partners
            pos[n] = C{wrap_box<R>(q0 + sh1 + z.x, box), wrap_box<R>(q1 + sh1 + z.y, box)};
            if (pos2) pos2[n] = C{wrap_box<R>(q0 + sh2 + z.x, box), wrap_box<R>(q1 + sh2 + z.y, box)};
          } else {
            pos[n] = C{wrap_box<R>(q0 + z.x, box), wrap_box<R>(q1 + z.y, box)};
          }
        }
        if (OUT || vel) vel[n] = C{vfac * z.x, vfac * z.y};
      }
    ct::stage_barrier<Pol::SY>();  // the work tile's lines are rewritten next tile
  }
  __syncthreads();
  if (tid == 0) mbar_inval(bar);  // the caller may reuse the shared memory
  return true;
}

template <typename R, int N, int V, bool EXT = false, int OUT = 0>
__global__ void __launch_bounds__(ct::ZPolicy<R, N, V>::THREADS, ct::ZPolicy<R, N, V>::MINB_INV)
    k_zinv_ct(const ZInvArgs a) {
  zinv_body<R, N, V, EXT, OUT>(a, blockIdx.x, gridDim.x, INT64_MAX);
}

// Forward z pass: Philox noise (or caller noise) of L lines into the padded
// work tile, the length-N/2 transform in place, then the real-input unpacking
// X_k = (Z_k + conj Z_{M-k})/2 - i/2 e^{-2 pi i k/N} (Z_k - conj Z_{M-k}).
template <typename R, int N, int V>
__device__ __forceinline__ void zfwd_body(const ZFwdArgs &a, int64_t t0, int64_t tstep,
                                          int64_t tlimit) {
  using C = Cx<R>;
  using Pol = ct::ZPolicy<R, N, V>;
  constexpr int M = Pol::M, E = Pol::E, P = Pol::P, L = Pol::L, LD = Pol::LD_FWD, PAD = Pol::PAD_FWD;
  constexpr int KM = ct::skey<R>(M);
  constexpr int S = ct::nstages(KM);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C *work = reinterpret_cast<C *>(smem_raw);
  const int tid = threadIdx.x;
  const int64_t ntiles = a.nlines / L;
  const ct::Tw<C, false> tw_half{reinterpret_cast<const C *>(a.tw_half)};
  const C *twf = reinterpret_cast<const C *>(a.tw_full);
  if (tlimit > ntiles) tlimit = ntiles;
  for (int64_t t = t0; t < tlimit; t += tstep) {
    int l = tid / P, p = tid - (tid / P) * P;
    asm volatile("" : "+r"(l), "+r"(p));
    __builtin_assume(l >= 0 && l < L && p >= 0 && p < P);
    const int64_t line = t * L + l;
    // line counts stay below 2^32 (N <= 4096, the host bounds the batch)
    const uint32_t lpr = (uint32_t)(a.lines_per_real > 0 ? a.lines_per_real : a.nlines);
    const uint32_t rr = (uint32_t)line / lpr, local = (uint32_t)line - rr * lpr;
    static_assert(N % 4 == 0, "lines start on a Philox group");
    const uint64_t g0 = (uint64_t)local * (uint64_t)(N / 4);
    auto gen = [&](uint64_t seed) {
#pragma unroll
      for (int i = 0; i < E / 2; ++i) {
        const int q = p + P * i;
        R w[4];
        if constexpr ((int64_t)N * N * N / 4 <= 0xFFFFFFFFll)  // group indices fit 32 bits
          gauss4(noise_words32(seed, (uint32_t)(g0 + q)), w);
        else
          gauss4(noise_words(seed, g0 + q), w);
        work[zpad<LD, PAD>(l, 2 * q)] = C{w[0], w[1]};
        work[zpad<LD, PAD>(l, 2 * q + 1)] = C{w[2], w[3]};
      }
    };
    if (a.noise) {
      const C *src = reinterpret_cast<const C *>(a.noise) + line * M;
#pragma unroll
      for (int i = 0; i < E; ++i) work[zpad<LD, PAD>(l, p + P * i)] = src[p + P * i];
    } else if (!a.seeds) {  // one seed for the launch: its key schedule is uniform
      gen(a.seed);
    } else {
      gen(a.seeds[rr]);
    }
    ct::stage_barrier<Pol::SY>();
    auto ld_w = [&](int n) { return work[zpad<LD, PAD>(l, n)]; };
    auto st_w = [&](int n, C v) { work[zpad<LD, PAD>(l, n)] = v; };
    if constexpr (Pol::FUSE) {  // the last two stages in registers, stored in natural order
      ct::stages<R, M, E, false, 0, S - 2, Pol::SY>(p, tw_half, ld_w, st_w);
      constexpr int RB = ct::radix_of(KM, S - 1, false), NBB = E / RB, SPANB = M / RB;
      C v[E];
      ct::last_two_stages_regs<R, M, E>(p, tw_half, ld_w, v);
      ct::stage_barrier<Pol::SY>();
#pragma unroll
      for (int b = 0; b < NBB; ++b)
#pragma unroll
        for (int r = 0; r < RB; ++r) st_w(p + P * b + r * SPANB, v[b * RB + r]);
      ct::stage_barrier<Pol::SY>();
    } else {
      ct::stages<R, M, E, false, 0, S, Pol::SY>(p, tw_half, ld_w, st_w);
    }
    // X_k = S/2 + D u_k with S = Z_k + conj Z_{M-k}, D = Z_k - conj Z_{M-k},
    // u_k = -(i/2) w_k; the partner X_{M-k} = conj(S/2 - D u_k) (w_{M-k} =
    // -conj w_k), so each thread takes the pairs k = p + P i < M/2 and both
    // members from one pair of loads. k = 0: X_0 = Re Z_0 + Im Z_0 (real), and
    // the self-paired X_{M/2} = conj Z_{M/2}.
    static_assert(P * (E / 2) == M / 2, "r2c pairs");
    C *dst = reinterpret_cast<C *>(a.out) + line * M;
#pragma unroll
    for (int i = 0; i < E / 2; ++i) {
      const int k = p + P * i;
      const C zk = work[zpad<LD, PAD>(l, k)];
      if (k == 0) {
        const C zh = work[zpad<LD, PAD>(l, M / 2)];
        dst[0] = C{zk.x + zk.y, (R)0};
        dst[M / 2] = C{zh.x, -zh.y};
      } else {
        const C zm = work[zpad<LD, PAD>(l, M - k)];
        const C w = ldg_c(twf + k);
        const C u = {(R)0.5 * w.y, (R)-0.5 * w.x};  // exact: a halving and a swap
        const C sm = {zk.x + zm.x, zk.y - zm.y};
        const C df = {zk.x - zm.x, zk.y + zm.y};
        const C t = cmul(df, u);
        dst[k] = C{fma_rn((R)0.5, sm.x, t.x), fma_rn((R)0.5, sm.y, t.y)};
        dst[M - k] = C{fma_rn((R)0.5, sm.x, -t.x), -fma_rn((R)0.5, sm.y, -t.y)};
      }
    }
    ct::stage_barrier<Pol::SY>();  // the work tile's lines are rewritten next tile
  }
}

template <typename R, int N, int V>
__global__ void __launch_bounds__(ct::ZPolicy<R, N, V>::THREADS, ct::ZPolicy<R, N, V>::MINB_FWD)
    k_zfwd_ct(const ZFwdArgs a) {
  zfwd_body<R, N, V>(a, blockIdx.x, gridDim.x, INT64_MAX);
}

// ------------------------------------------------------------ launchers
template <typename R, int N, int V, int MODE, bool CUT = false, int FILT = kFiltArgs>
cudaError_t ct_launch_axis(const AxisArgs &in, cudaStream_t s) {
  using Pol = ct::AxisPolicy<R, N, V>;
  AxisArgs a = in;
  if ((a.chunked_in || a.chunked_out) && a.cols != Pol::B) return cudaErrorInvalidValue;
  a.cols = Pol::B;
  a.inner_chunks = (N / 2) / Pol::B;
  a.rows_box = Pol::ROWS_BOX;
  a.e = Pol::E;
  CUtensorMap map;
  cudaError_t e = make_map<R>(&map, a);
  if (e != cudaSuccess) return e;
  // TMA stores: the maps of the outputs (same geometry, their own layout)
  constexpr bool TST = axis_tma_store<R, N, V, MODE, CUT, FILT>() ||
                       axis_tma_store_inplace<R, N, V, MODE, CUT, FILT>() ||
                       axis_tma_store_fwd<R, N, V, MODE>();
  CUtensorMap smap[2] = {map, map};
  if constexpr (TST) {
    if (a.nout > 2) return cudaErrorInvalidValue;
    for (int o = 0; o < a.nout; ++o) {
      AxisArgs b = a;
      b.src = a.dst[o];
      b.chunked_in = a.chunked_out;
      if ((e = make_map<R>(&smap[o], b)) != cudaSuccess) return e;
    }
  }
  const size_t tile = ((size_t)N * Pol::B * 2 * sizeof(R) + 127) & ~(size_t)127;
  const bool interp = sizeof(R) == 4 && a.pre && a.interp;
  const size_t filt = interp ? (Pol::TW_SMEM ? kInterpExact * sizeof(float) + (size_t)kMaxInterpCells(N) * 16
                                              : kInterpExact * sizeof(float) + (size_t)a.interp_cells * 16)
                             : 0;
  constexpr bool STAGING = axis_tma_store<R, N, V, MODE, CUT, FILT>();  // a third tile
  const size_t smem = 128 + (STAGING ? 3 : 2) * tile + filt + (Pol::TW_SMEM ? (size_t)N * 2 * sizeof(R) : 0);
  if (interp && a.interp_cells > kMaxInterpCells(N)) return cudaErrorInvalidValue;
  auto kern = k_axis_ct<R, N, V, MODE, CUT, FILT>;
  if ((e = set_smem(kern, smem)) != cudaSuccess) return e;
  const int64_t tiles = (int64_t)N * a.inner_chunks * (a.nbatch > 0 ? a.nbatch : 1);
  kern<<<persistent_blocks(kern, Pol::THREADS, smem, tiles), Pol::THREADS, smem, s>>>(map, smap[0], smap[1], a);
  return cudaGetLastError();
}

template <typename R, int N, int V, bool EXT = false, int OUT = 0>
cudaError_t ct_launch_zinv(const ZInvArgs &a, cudaStream_t s) {
  using Pol = ct::ZPolicy<R, N, V>;
  const size_t dense = (Pol::DENSE * 2 * sizeof(R) + 127) & ~(size_t)127;
  const size_t smem = 128 + dense + (size_t)Pol::WORK_INV * 2 * sizeof(R);
  auto kern = k_zinv_ct<R, N, V, EXT, OUT>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  kern<<<persistent_blocks(kern, Pol::THREADS, smem, a.nlines / Pol::L), Pol::THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename R, int N, int V>
cudaError_t ct_launch_zfwd(const ZFwdArgs &a, cudaStream_t s) {
  using Pol = ct::ZPolicy<R, N, V>;
  const size_t smem = (size_t)Pol::WORK_FWD * 2 * sizeof(R);
  auto kern = k_zfwd_ct<R, N, V>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  kern<<<persistent_blocks(kern, Pol::THREADS, smem, a.nlines / Pol::L), Pol::THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

constexpr int kAxisVariants = 3;
constexpr int kZVariants = 4;

// Run-time dispatch over the specialised sizes and their tile variants.
template <typename R, int... NS> struct CtTable {
  static bool has(int n) { return ((n == NS) || ...); }
  template <int N> static int cols_n(int v) {
    return v == 1 ? ct::AxisPolicy<R, N, 1>::B : (v == 2 ? ct::AxisPolicy<R, N, 2>::B : ct::AxisPolicy<R, N, 0>::B);
  }
  static int cols(int n, int v) {
    int c = 0;
    ((n == NS ? (c = cols_n<NS>(v), 0) : 0), ...);
    return c;
  }
  template <int N, int V> static cudaError_t axis_v(const AxisArgs &a, cudaStream_t s) {
    if (a.fwd && a.inv) {
      if constexpr (sizeof(R) == 4)
        if (a.pre && a.interp) return ct_launch_axis<R, N, V, kAxisFwdInv, false, kFiltInterp>(a, s);
      return ct_launch_axis<R, N, V, kAxisFwdInv>(a, s);
    }
    if (a.fwd) {
      return a.pre ? ct_launch_axis<R, N, V, kAxisFwd>(a, s)
                   : ct_launch_axis<R, N, V, kAxisFwd, false, kFiltNone>(a, s);
    }
    // inverse only: the run-time flags measured faster at N = 1536 than the
    // filter-free instantiation (11.0 against 11.5 ms for the y/z branches)
    return ct_launch_axis<R, N, V, kAxisInv>(a, s);
  }
  template <int N> static cudaError_t axis_n(const AxisArgs &a, cudaStream_t s) {
    if (!a.fwd && !a.inv) return cudaErrorInvalidValue;
    if (a.pre && a.qmin > 0) {  // the Sec. 2.4 cut (the fused x pass only): variant 0
      if (!(a.fwd && a.inv)) return cudaErrorInvalidValue;
      return ct_launch_axis<R, N, 0, kAxisFwdInv, true>(a, s);
    }
    return a.variant == 1 ? axis_v<N, 1>(a, s) : (a.variant == 2 ? axis_v<N, 2>(a, s) : axis_v<N, 0>(a, s));
  }
  static cudaError_t axis(const AxisArgs &a, cudaStream_t s) {
    cudaError_t e = cudaErrorInvalidValue;
    ((a.n == NS ? (e = axis_n<NS>(a, s), 0) : 0), ...);
    return e;
  }
  template <int N, int V> static cudaError_t zinv_v(const ZInvArgs &a, cudaStream_t s) {
    const bool lists = a.pos_list || a.vel_list;
    const bool outs = lists ? a.pos_list && a.vel_list && a.lists_full && !a.pos && !a.vel
                            : a.pos && a.vel;
    const bool plain = !a.psi && !a.psi_list && !a.accumulate && outs &&
                       (a.mul_kz != 0) == (a.comp == 2);
    if (!plain) return ct_launch_zinv<R, N, V>(a, s);
    return a.comp == 2 ? ct_launch_zinv<R, N, V, false, kZPosVelZ>(a, s)
                       : ct_launch_zinv<R, N, V, false, kZPosVel>(a, s);
  }
  template <int N> static cudaError_t zinv_n(const ZInvArgs &a, cudaStream_t s) {
    if (a.large || a.pos2 || a.shift != 0.0 || a.shift2 != 0.0)  // Secs. 2.2, 2.4 options: variant 0
      return ct_launch_zinv<R, N, 0, true>(a, s);
    switch (a.variant) {
      case 1: return zinv_v<N, 1>(a, s);
      case 2: return zinv_v<N, 2>(a, s);
      case 3: return zinv_v<N, 3>(a, s);
      default: return zinv_v<N, 0>(a, s);
    }
  }
  template <int N> static cudaError_t zfwd_n(const ZFwdArgs &a, cudaStream_t s) {
    switch (a.variant) {
      case 1: return ct_launch_zfwd<R, N, 1>(a, s);
      case 2: return ct_launch_zfwd<R, N, 2>(a, s);
      case 3: return ct_launch_zfwd<R, N, 3>(a, s);
      default: return ct_launch_zfwd<R, N, 0>(a, s);
    }
  }
  static cudaError_t zinv(const ZInvArgs &a, cudaStream_t s) {
    cudaError_t e = cudaErrorInvalidValue;
    ((a.n == NS ? (e = zinv_n<NS>(a, s), 0) : 0), ...);
    return e;
  }
  static cudaError_t zfwd(const ZFwdArgs &a, cudaStream_t s) {
    cudaError_t e = cudaErrorInvalidValue;
    ((a.n == NS ? (e = zfwd_n<NS>(a, s), 0) : 0), ...);
    return e;
  }
};

}  // namespace gg
