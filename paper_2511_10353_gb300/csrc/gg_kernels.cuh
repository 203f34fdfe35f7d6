// Kernels of the noise -> Zel'dovich path (Secs. 2.1-2.2, Eqs. 1-3) and their
// launchers. Included once per real type by gg_kernels_f32.cu / _f64.cu.
//
// Data layout in HBM: the half spectrum [N][N][N/2] complex (x, y, kz with kz
// fastest) overlays exactly one real N^3 grid: the z-Nyquist plane is never
// stored because the filter zeroes it (every mode with |m_j| = N/2 is dropped).
#pragma once

#include <cstring>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "gg_device.cuh"
#include "gg_launch.cuh"

namespace gg {

// ------------------------------------------------------------------ noise
template <typename R>
__global__ void k_noise(NoiseArgs a) {
  const int64_t groups = (a.cells + 3) >> 2;
  R *out = reinterpret_cast<R *>(a.out);
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < groups;
       g += (int64_t)gridDim.x * blockDim.x) {
    R v[4];
    gauss4(noise_words(a.seed, (uint64_t)g), v);
    const int64_t c = g << 2;
    if (c + 3 < a.cells) {
      if constexpr (sizeof(R) == 4) {
        *reinterpret_cast<float4 *>(out + c) = make_float4(v[0], v[1], v[2], v[3]);
      } else {
        *reinterpret_cast<double2 *>(out + c) = make_double2(v[0], v[1]);
        *reinterpret_cast<double2 *>(out + c + 2) = make_double2(v[2], v[3]);
      }
    } else {
      for (int i = 0; i < 4 && c + i < a.cells; ++i) out[c + i] = v[i];
    }
  }
}


// ---------------------------------------------------------- forward z pass
// One CTA: `lines_per_cta` z-lines. Each line of N reals (noise made in place
// from (seed, cell index), or read) is packed as N/2 complex values
// z_n = W_2n + i W_2n+1, transformed with the length-N/2 FFT and unpacked into
// X_k = (Z_k + conj Z_{M-k})/2 - i/2 e^{-2 pi i k/N} (Z_k - conj Z_{M-k}),
// k < N/2 (the real-input DFT).
template <typename R, int E>
__global__ void k_zfwd(const ZFwdArgs a) {
  using C = Cx<R>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C *buf = reinterpret_cast<C *>(smem_raw);
  const int M = a.st.len, P = M / E;
  const LineLayout lay{line_ld(M)};
  const int l = threadIdx.x / P, p = threadIdx.x - l * P;
  const int64_t line = (int64_t)blockIdx.x * a.lines_per_cta + l;
  const bool live = line < a.nlines;
  const int64_t lpr = a.lines_per_real > 0 ? a.lines_per_real : a.nlines;
  const int64_t rr = line / lpr, local = line - rr * lpr;  // realization, line within it
  const uint64_t seed = (a.seeds && live) ? a.seeds[rr] : a.seed;
  if (live) {
    if (a.noise) {
      const C *src = reinterpret_cast<const C *>(a.noise) + line * M;
#pragma unroll
      for (int i = 0; i < E; ++i) buf[lay(l, p + P * i)] = src[p + P * i];
    } else if ((a.n & 3) == 0) {
      if constexpr (E % 2 == 0) {
        const uint64_t g0 = (uint64_t)local * (uint64_t)(a.n >> 2);
#pragma unroll
        for (int i = 0; i < E / 2; ++i) {
          const int q = p + P * i;
          R v[4];
          gauss4(noise_words(seed, g0 + q), v);
          buf[lay(l, 2 * q)] = C{v[0], v[1]};
          buf[lay(l, 2 * q + 1)] = C{v[2], v[3]};
        }
      }
    } else {
      const uint64_t c0 = (uint64_t)local * (uint64_t)a.n;
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const int k = p + P * i;
        buf[lay(l, k)] = C{noise_cell<R>(seed, c0 + 2 * k), noise_cell<R>(seed, c0 + 2 * k + 1)};
      }
    }
  }
  __syncthreads();
  fft_smem<R, E, false>(buf, lay, l, p, P, a.st, reinterpret_cast<const C *>(a.tw_half));
  if (live) {
    C *dst = reinterpret_cast<C *>(a.out) + line * M;
    const C *twf = reinterpret_cast<const C *>(a.tw_full);
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int k = p + P * i;
      const C zk = buf[lay(l, k)];
      const C zm = buf[lay(l, k ? M - k : 0)];
      const C fe = {(R)0.5 * (zk.x + zm.x), (R)0.5 * (zk.y - zm.y)};
      const C fo = {(R)0.5 * (zk.y + zm.y), (R)-0.5 * (zk.x - zm.x)};
      dst[k] = cadd(fe, cmul(fo, ldg_c(twf + k)));
    }
  }
}

// ------------------------------------------------------- strided passes
__device__ __forceinline__ int freq_of(int n, int N) { return n < (N >> 1) ? n : n - N; }

template <typename R>
__device__ __forceinline__ Cx<R> apply_mul(int kind, Cx<R> v, int n, int N) {
  if (kind == kMulIm) {
    const R f = n == (N >> 1) ? (R)0 : (R)freq_of(n, N);
    return Cx<R>{-f * v.y, f * v.x};
  }
  return v;
}

// Persistent strided pass (see AxisArgs). Each CTA walks the tiles
// t = blockIdx.x, blockIdx.x + gridDim.x, ...; one thread issues the TMA loads
// of tile t+1 (3-D tensor map over [x][y][kz], box of `cols` kz columns by
// rows_box points) into the second shared buffer while the CTA transforms
// tile t. Forward stages run in place in shared memory except the last, whose
// outputs stay in registers: they sit at the positions the first inverse stage
// reads (same radix, inverse radices in reverse order), so the filter
// multiplies registers and no shared round trip separates the two transforms.
// Each inverse's last stage stores straight to HBM. Rows of `cols` complex
// values are 64 or 128 bytes, so a half-warp (FP32) or quarter-warp (FP64)
// access covers whole rows. Table values of the filter are read before the
// wait for the tile (an L1 prefetch, no registers held).
template <typename R, int E>
__global__ void __launch_bounds__(E >= 24 ? 256 : 512, 1)
    k_axis(const __grid_constant__ CUtensorMap map, const AxisArgs a) {
  using C = Cx<R>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw);
  const int N = a.n, P = N / E, B = a.cols, half = N >> 1;
  const int tile_elems = N * B;
  const int stride_elems = ((tile_elems * (int)sizeof(C) + 127) & ~127) / (int)sizeof(C);
  C *bufs = reinterpret_cast<C *>(smem_raw + 128);
  const int tid = threadIdx.x;
  const int64_t per_real = (int64_t)N * a.inner_chunks;
  const int64_t ntiles = per_real * (a.nbatch > 0 ? a.nbatch : 1);
  const uint32_t tile_bytes = (uint32_t)(tile_elems * sizeof(C));
  const C *tw = reinterpret_cast<const C *>(a.tw);
  const R *table = reinterpret_cast<const R *>(a.table);
  const bool use_tma = a.rows_box > 0;
  const FftStages &sf = a.st_fwd;
  const FftStages &si = a.st_inv;
  const int S = sf.nstages;
  const int r0 = a.inv ? si.radix[0] : sf.radix[S - 1];
  if (use_tma && tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  auto issue = [&](int64_t t, int sb) {
    const int rr = (int)(t / per_real);
    const int64_t tt = t - rr * per_real;
    const int64_t outer = tt / a.inner_chunks;
    const int chunk = (int)(tt - outer * a.inner_chunks);
    C *dst = bufs + sb * stride_elems;
    if (a.test_skip_copy) return;  // fault test: the wait for this tile runs out
    mbar_arrive_expect_tx(&bars[sb], tile_bytes);
    const int c0 = chunk * B * 2;  // innermost coordinate in reals
    for (int i = 0; i < N; i += a.rows_box) {
      if (a.axis == 1) tma_load_4d(dst + i * B, &map, &bars[sb], c0, i, (int)outer, rr);
      else tma_load_4d(dst + i * B, &map, &bars[sb], c0, (int)outer, i, rr);
    }
  };
  int64_t t = blockIdx.x;
  if (use_tma && tid == 0 && t < ntiles) issue(t, 0);
  bool abort = false;
  for (int it = 0; t < ntiles && !abort; t += gridDim.x, ++it) {
    const int sb = use_tma ? (it & 1) : 0;
    const int64_t tn = t + gridDim.x;
    if (use_tma && tid == 0 && tn < ntiles) {
      fence_proxy_async_smem();
      issue(tn, sb ^ 1);
    }
    // thread coordinates, opaque to the optimiser so that the addresses of
    // every stage variant are not hoisted out of the tile loop (they would
    // stay live for the whole kernel)
    int c = tid & (B - 1), p = tid / B;
    asm volatile("" : "+r"(c), "+r"(p));
    const int64_t rr = t / per_real;
    const int64_t tt = t - rr * per_real;
    const int64_t outer = tt / a.inner_chunks;
    const int chunk = (int)(tt - outer * a.inner_chunks);
    const int kz = chunk * B + c;
    C *buf = bufs + sb * stride_elems;
    const int64_t gbase = rr * a.batch_stride + outer * a.outer_stride + kz;
    const int m_outer = a.axis == 0 ? freq_of((int)outer, N) : 0;
    const bool nyq_outer = a.axis == 0 && (int)outer == half;
    auto ld_smem = [&](int n) { return buf[n * B + c]; };
    auto st_smem = [&](int n, C v) { buf[n * B + c] = v; };
    // V: this thread's elements at the hand-off positions p + P*b + r*N/r0
    C V[E];
    auto tab_index = [&](int n) {
      const int m = freq_of(n, N);
      return (n == half || nyq_outer) ? -1 : m * m + m_outer * m_outer + kz * kz;
    };
    if (a.pre) {
      with_radix<E>(r0, [&](auto rc) {
        constexpr int RH = decltype(rc)::value;
        const int span = N / RH;
#pragma unroll
        for (int b = 0; b < E / RH; ++b)
#pragma unroll
          for (int r = 0; r < RH; ++r) {
            const int q = tab_index(p + P * b + r * span);
            if (q >= 0) prefetch_l1(table + q);
          }
      });
    }
    if (use_tma) {
      const bool ok =
          __syncthreads_and(mbar_wait(&bars[sb], (uint32_t)((it >> 1) & 1), a.err, a.wait_us));
      if (!ok) {
        if (tid == 0 && tn < ntiles && !a.test_skip_copy)
          mbar_wait(&bars[sb ^ 1], (uint32_t)(((it + 1) >> 1) & 1), nullptr, a.wait_us);
        abort = true;
        break;
      }
    } else {
      const C *src = reinterpret_cast<const C *>(a.src) + rr * a.batch_stride +
                     outer * a.outer_stride + chunk * B;
      for (int q = tid; q < tile_elems; q += blockDim.x) {
        const int n = q / B;
        buf[q] = src[(int64_t)n * a.stride + (q - n * B)];
      }
      __syncthreads();
    }
    if (a.fwd)
      for (int s2 = 0; s2 < S - 1; ++s2)
        stage_dispatch<R, E, false, true>(sf, s2, p, P, tw, ld_smem, st_smem);
    with_radix<E>(r0, [&](auto rc) {
      constexpr int RH = decltype(rc)::value;
      const int span = N / RH;
#pragma unroll
      for (int b = 0; b < E / RH; ++b)
#pragma unroll
        for (int r = 0; r < RH; ++r) V[b * RH + r] = buf[(p + P * b + r * span) * B + c];
      if (a.fwd) {
        StageTw<R, E, RH> tt;
        load_twiddles<R, E, RH>(tt, p, P, sf.ns[S - 1], sf.ns_shift[S - 1], sf.tstep[S - 1], tw);
        stage_compute<R, E, RH, false>(V, p, P, sf.ns[S - 1], sf.ns_shift[S - 1], sf.tstep[S - 1],
                                       tt, tw);
      }
      if (a.pre) {
#pragma unroll
        for (int b = 0; b < E / RH; ++b)
#pragma unroll
          for (int r = 0; r < RH; ++r) {
            const int q = tab_index(p + P * b + r * span);
            const R f = (q >= 0 && q >= a.qmin) ? __ldg(table + q) : (R)0;  // qmin: Eq. 4
            V[b * RH + r] = Cx<R>{f * V[b * RH + r].x, f * V[b * RH + r].y};
          }
      }
      if (!a.inv) {  // forward only: the spectrum to dst[0]
        C *d = reinterpret_cast<C *>(a.dst[0]) + gbase;
#pragma unroll
        for (int b = 0; b < E / RH; ++b)
#pragma unroll
          for (int r = 0; r < RH; ++r)
            d[(int64_t)(p + P * b + r * span) * a.stride] = V[b * RH + r];
      }
    });
    __syncthreads();  // the tile is in registers: buf becomes the inverse work buffer
    if (!a.inv) continue;
    for (int o = 0; o < a.nout; ++o) {
      asm volatile("" : "+r"(c), "+r"(p));
      C *d = reinterpret_cast<C *>(a.dst[o]) + gbase;
      auto st_glob = [&](int n, C v) { d[(int64_t)n * a.stride] = v; };
      if (o > 0) __syncthreads();  // the previous output's last stage has read buf
      with_radix<E>(r0, [&](auto rc) {
        constexpr int RH = decltype(rc)::value;
        const int span = N / RH;
        C W[E];
#pragma unroll
        for (int b = 0; b < E / RH; ++b)
#pragma unroll
          for (int r = 0; r < RH; ++r) {
            const int n = p + P * b + r * span;
            W[b * RH + r] = apply_mul<R>(a.mul[o], V[b * RH + r], n, N);
          }
        StageTw<R, E, RH> none;
        stage_compute<R, E, RH, true>(W, p, P, 1, 0, 0, none, tw);  // first inverse stage: ns = 1
#pragma unroll
        for (int b = 0; b < E / RH; ++b)
#pragma unroll
          for (int r = 0; r < RH; ++r) {
            const int q = (p + P * b) * RH + r;
            if (S == 1) st_glob(q, W[b * RH + r]);
            else buf[q * B + c] = W[b * RH + r];
          }
      });
      if (S == 1) continue;
      __syncthreads();
      for (int s2 = 1; s2 < S - 1; ++s2)
        stage_dispatch<R, E, true, true>(si, s2, p, P, tw, ld_smem, st_smem);
      stage_dispatch<R, E, true, false>(si, S - 1, p, P, tw, ld_smem, st_glob);
    }
    __syncthreads();
  }
}

// ---------------------------------------------- inverse z pass + epilogue
// c2r of each half-spectrum line (X_{N/2} = 0): Z_k = (X_k + conj X_{M-k})
// + i e^{+2 pi i k/N} (X_k - conj X_{M-k}), inverse FFT of length M = N/2,
// x_2n = Re z_n, x_2n+1 = Im z_n. Then Eq. 3 per cell: psi, pos = (q + psi)
// mod L, vel = vfac psi; or the plain real field when pos and vel are null.
template <typename R, int E>
__global__ void k_zinv(const ZInvArgs a) {
  using C = Cx<R>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C *buf = reinterpret_cast<C *>(smem_raw);
  const int M = a.st.len, P = M / E;
  const LineLayout lay{line_ld(M)};
  const int l = threadIdx.x / P, p = threadIdx.x - l * P;
  const int64_t line = (int64_t)blockIdx.x * a.lines_per_cta + l;
  const bool live = line < a.nlines;
  if (live) {
    const C *src = reinterpret_cast<const C *>(a.src) + line * M;
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int k = p + P * i;
      C v = src[k];
      if (a.mul_kz) v = C{mul_rn(-(R)k, v.y), mul_rn((R)k, v.x)};  // i m_z, m_z = k for k < N/2
      buf[lay(l, k)] = v;
    }
  }
  __syncthreads();
  C z[E];
  const C *twf = reinterpret_cast<const C *>(a.tw_full);
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int k = p + P * i;
    const C xk = buf[lay(l, k)];
    const C xm = k ? buf[lay(l, M - k)] : C{(R)0, (R)0};
    const C s = {xk.x + xm.x, xk.y - xm.y};  // X_k + conj X_{M-k}
    const C d = {xk.x - xm.x, xk.y + xm.y};  // X_k - conj X_{M-k}
    z[i] = cadd(s, mul_pi(cmulc(d, ldg_c(twf + k))));
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < E; ++i) buf[lay(l, p + P * i)] = z[i];
  __syncthreads();
  fft_smem<R, E, true>(buf, lay, l, p, P, a.st, reinterpret_cast<const C *>(a.tw_half));
  if (!live) return;
  const int64_t lpr = a.lines_per_real > 0 ? a.lines_per_real : a.nlines;
  const int64_t rr = line / lpr, local = line - rr * lpr;
  const int64_t ix = local / a.n, iy = local - ix * a.n;
  const R box = (R)a.box, cell = (R)a.cell, qo = (R)a.q_offset, vfac = (R)a.vfac;
  const R qline = mul_rn(a.comp == 0 ? (R)ix + qo : (R)iy + qo, cell);
  void *psi_b = a.psi_list ? a.psi_list[rr] : a.psi;
  void *pos_b = a.pos_list ? a.pos_list[rr] : a.pos;
  void *vel_b = a.vel_list ? a.vel_list[rr] : a.vel;
  const int64_t off = (a.psi_list || a.pos_list || a.vel_list) ? local * M : line * M;
  C *psi = psi_b ? reinterpret_cast<C *>(psi_b) + off : nullptr;
  C *pos = pos_b ? reinterpret_cast<C *>(pos_b) + off : nullptr;
  C *vel = vel_b ? reinterpret_cast<C *>(vel_b) + off : nullptr;
  const R *large = reinterpret_cast<const R *>(a.large);
  CicAxis<R> cx{}, cy{};
  if (large) {
    cx = cic_axis<R>((int)ix, a.n_low, a.n);
    cy = cic_axis<R>((int)iy, a.n_low, a.n);
  }
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int n = p + P * i;
    C v = buf[lay(l, n)];
    if (large) {  // Sec. 2.4: the interpolated coarse large scales
      R l0, l1;
      cic_pair<R>(large, a.n_low, a.n, cx, cy, n, l0, l1);
      v.x += l0;
      v.y += l1;
    }
    if (psi) {
      if (a.accumulate) {
        const C o = psi[n];
        psi[n] = C{o.x + (R)a.alpha * v.x, o.y + (R)a.alpha * v.y};
      } else {
        psi[n] = v;
      }
    }
    if (pos) {
      R q0 = qline, q1 = qline;
      if (a.comp == 2) {
        q0 = mul_rn((R)(2 * n) + qo, cell);
        q1 = mul_rn((R)(2 * n + 1) + qo, cell);
      }
      const R sh1 = (R)a.shift, sh2 = (R)a.shift2;  // Sec. 2.2: periodic shift, gas partners
      pos[n] = C{wrap_box<R>(q0 + sh1 + v.x, box), wrap_box<R>(q1 + sh1 + v.y, box)};
      if (a.pos2)
        reinterpret_cast<C *>(a.pos2)[off + n] =
            C{wrap_box<R>(q0 + sh2 + v.x, box), wrap_box<R>(q1 + sh2 + v.y, box)};
    }
    if (vel) vel[n] = C{vfac * v.x, vfac * v.y};
  }
}

// ----------------------------------------------------------------- launchers
#define GG_DISPATCH_E(E_, ...)                 \
  switch (E_) {                                 \
    case 2: { constexpr int EE = 2; __VA_ARGS__; } break;  \
    case 3: { constexpr int EE = 3; __VA_ARGS__; } break;  \
    case 4: { constexpr int EE = 4; __VA_ARGS__; } break;  \
    case 6: { constexpr int EE = 6; __VA_ARGS__; } break;  \
    case 8: { constexpr int EE = 8; __VA_ARGS__; } break;  \
    case 12: { constexpr int EE = 12; __VA_ARGS__; } break; \
    case 16: { constexpr int EE = 16; __VA_ARGS__; } break; \
    case 24: { constexpr int EE = 24; __VA_ARGS__; } break; \
    default: return cudaErrorInvalidValue;      \
  }

template <typename R>
cudaError_t launch_noise(const NoiseArgs &a, cudaStream_t s) {
  const int64_t groups = (a.cells + 3) >> 2;
  if (groups == 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 256;
  int64_t blocks = (groups + threads - 1) / threads;
  const int64_t cap = (int64_t)sms * 8;
  if (blocks > cap) blocks = cap;
  k_noise<R><<<(unsigned)blocks, threads, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_zfwd(const ZFwdArgs &a, cudaStream_t s) {
  const int P = a.st.len / a.st.e;
  const size_t smem = zpass_smem_bytes(a.st.len, a.lines_per_cta, sizeof(Cx<R>));
  const unsigned blocks = (unsigned)((a.nlines + a.lines_per_cta - 1) / a.lines_per_cta);
  const unsigned threads = (unsigned)(P * a.lines_per_cta);
  GG_DISPATCH_E(a.st.e, {
    auto kern = k_zfwd<R, EE>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<blocks, threads, smem, s>>>(a);
  });
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_axis(const AxisArgs &a, cudaStream_t s) {
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  cudaError_t e;
  if (a.rows_box > 0 && (e = make_map<R>(&map, a)) != cudaSuccess) return e;
  const int P = a.n / a.e;
  const unsigned threads = (unsigned)(P * a.cols);
  const size_t smem = axis_smem_bytes(a.n, a.cols, sizeof(Cx<R>));
  const int64_t tiles = (int64_t)a.n * a.inner_chunks * (a.nbatch > 0 ? a.nbatch : 1);
  GG_DISPATCH_E(a.e, {
    auto kern = k_axis<R, EE>;
    if ((e = set_smem(kern, smem)) != cudaSuccess) return e;
    kern<<<persistent_blocks(kern, threads, smem, tiles), threads, smem, s>>>(map, a);
  });
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_zinv(const ZInvArgs &a, cudaStream_t s) {
  const int P = a.st.len / a.st.e;
  const size_t smem = zpass_smem_bytes(a.st.len, a.lines_per_cta, sizeof(Cx<R>));
  const unsigned blocks = (unsigned)((a.nlines + a.lines_per_cta - 1) / a.lines_per_cta);
  const unsigned threads = (unsigned)(P * a.lines_per_cta);
  GG_DISPATCH_E(a.st.e, {
    auto kern = k_zinv<R, EE>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<blocks, threads, smem, s>>>(a);
  });
  return cudaGetLastError();
}

// Largest block each kernel can launch with (registers bound it), so the host
// can size tiles: kind 0 = forward z, 2 = inverse z, 3 = strided.
template <typename R>
int max_block_threads(int kind, int e) {
  cudaFuncAttributes fa{};
  cudaError_t err = cudaErrorInvalidValue;
  GG_DISPATCH_E(e, {
#ifdef GG_AXIS_TU
    if (kind == 3) err = cudaFuncGetAttributes(&fa, k_axis<R, EE>);
#else
    if (kind == 0) err = cudaFuncGetAttributes(&fa, k_zfwd<R, EE>);
    else if (kind == 2) err = cudaFuncGetAttributes(&fa, k_zinv<R, EE>);
#endif
  });
  return err == cudaSuccess ? fa.maxThreadsPerBlock : -1;
}

#define GG_INSTANTIATE_Z(R)                                                       \
  template cudaError_t launch_noise<R>(const NoiseArgs &, cudaStream_t);          \
  template cudaError_t launch_zfwd<R>(const ZFwdArgs &, cudaStream_t);            \
  template cudaError_t launch_zinv<R>(const ZInvArgs &, cudaStream_t);            \
  template <> int max_block_threads_z<R>(int kind, int e) { return max_block_threads<R>(kind, e); }

#define GG_INSTANTIATE_AXIS(R)                                                    \
  template cudaError_t launch_axis<R>(const AxisArgs &, cudaStream_t);            \
  template <> int max_block_threads_axis<R>(int e) { return max_block_threads<R>(3, e); }

}  // namespace gg
