// Internal interface between the host runtime (gg_api.cpp, gg_cosmo.cpp) and
// the sm_103a kernels (gg_kernels_*.cu). Plain C++: no device code here.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "gg.h"

namespace gg {

constexpr int kMaxStages = 16;
constexpr int kInterpExact = 1024;  // m2 below this: exact table values in shared memory
// first stored unit cell in m = sqrt(m2) of the interpolated filter: m2 >= 1024
// gives m >= 32 (31 for an FP32 square root just below 32)
constexpr int kInterpFirstCell = 31;
// most stored cells (j = kInterpFirstCell ...) for grids of n points
__host__ __device__ constexpr int kMaxInterpCells(int n) {
  return (int)(1.7320508075688772 * (n / 2)) + 3 - kInterpFirstCell > 0
             ? (int)(1.7320508075688772 * (n / 2)) + 3 - kInterpFirstCell
             : 0;
}

// Radix schedule of one complex transform of length `len` done inside a CTA
// (Stockham autosort, decimation in time). Stage s combines radix[s] partial
// transforms of length ns[s]; every thread holds `e` elements of its line and
// runs e / radix[s] butterflies per stage.
struct FftStages {
  int len;
  int nstages;
  int e;                      // elements per thread: a multiple of every radix
  int radix[kMaxStages];
  int ns[kMaxStages];         // product of the radices of earlier stages
  int ns_shift[kMaxStages];   // log2(ns) when ns is a power of two, else -1
  int tstep[kMaxStages];      // len / (ns * radix): twiddle index step
};

// Builds the schedule for len = 2^a 3^b (radix 8 first, then 4 / 2, then 3).
bool make_stages(int len, FftStages *st);
// The same radices in reverse order (the inverse transforms start with the
// radix the forward ones end with).
FftStages reversed_stages(const FftStages &f);

// Multipliers of the strided passes. The spectrum handed from the forward to
// the inverse transforms is first multiplied by T(m2) when `pre` is set (x
// pass only: m2 = m_x^2 + m_y^2 + m_z^2 with the outer index ky; modes with
// m_x or m_y = -N/2 give 0), then each output by its own factor.
enum Mul : int {
  kMulNone = 0,  // v
  kMulIm = 1,    // i m v, m = integer frequency along the pass axis (0 at -N/2)
};

// A strided pass over the half spectrum [N][N][N/2] complex along y (axis 1:
// outer index x) or x (axis 0: outer index ky). A CTA owns `cols` adjacent kz
// columns of one outer index, all N points. Modes:
//   fwd && !inv : forward transform, write the spectrum (x T if pre) to dst[0]
//   fwd &&  inv : forward transform, x T if pre, then for each output o:
//                 x mul[o], inverse transform, write to dst[o]
//  !fwd &&  inv : for each output o: x mul[o], inverse transform -> dst[o]
struct AxisArgs {
  const void *src;
  void *dst[3];
  int nout;
  int mul[3];
  int fwd, inv;
  int64_t stride;         // complex elements between points along the axis
  int64_t outer_stride;   // complex elements between outer indices
  int inner_chunks;       // (N/2) / cols
  int cols;
  int n;                  // N
  int axis;               // 0: x, 1: y
  FftStages st_fwd;       // forward schedule (radix 8 first, 3 last)
  FftStages st_inv;       // inverse schedule: the same radices in reverse order
  const void *tw;         // exp(-2 pi i t / N)
  int pre;                // 1: multiply the handed-off spectrum by table[m2]
  const void *table;      // T(m2)
  // FP32 size-specialised kernels: T from shared memory instead of a gather
  // from the global table: exact values for m2 < kInterpExact, above that a
  // cubic Hermite interpolation in m = sqrt(m2) over unit cells (float4:
  // the interpolant's coefficients a0..a3 in t = m - j, from F_j, F'_j,
  // F_j+1, F'_j+1). nullptr: gather from `table`.
  const void *interp;
  int interp_cells;
  int e;                  // elements per thread (multiple of every radix)
  int rows_box;           // TMA box height (divisor of N, <= 256); 0: plain loads
  int *err;               // device error word
  int variant;            // tile variant of the size-specialised kernel
  int nbatch;             // realizations in the buffers (<= 0 means 1), outermost
  int64_t batch_stride;   // complex elements between realizations
  int qmin;               // with pre: modes with m2 < qmin get 0 (Eq. 4 top hat; 0: none)
  // Chunk-major spectra [realization][k_z chunk][x][y][cols] (cols complex
  // columns per chunk, the codelet's tile width): a tile of either strided
  // axis then spans few memory pages. chunked_in: src has that layout (tiles
  // taken chunk-outer); chunked_out: every dst has it.
  int chunked_in, chunked_out;
  // fault test (gg_test_arm_fault): no tile copy is issued, so every CTA's
  // first wait gives up after wait_us and reports GG_ETIMEOUT; 0 normally
  int test_skip_copy;
  uint32_t wait_us;       // limit of the copy waits in microseconds (0: the default)
};

// Forward z pass: real lines of N (generated noise or caller noise) -> half
// spectra of N/2 complex (the z-Nyquist term is not kept).
struct ZFwdArgs {
  const void *noise;      // N^3 reals or nullptr: generate from seed
  void *out;              // nlines * (N/2) complex
  uint64_t seed;
  int64_t nlines;         // N^2
  int n;                  // N
  int lines_per_cta;
  FftStages st;           // length N/2
  const void *tw_half;    // exp(-2 pi i t / (N/2)), t < N/2
  const void *tw_full;    // exp(-2 pi i t / N), t < N
  int variant;            // tile variant of the size-specialised kernel
  const uint64_t *seeds;  // batched form: device array, one seed per realization (else seed)
  int64_t lines_per_real; // lines of one realization (<= 0: nlines)
};

// Inverse z pass (c2r) with the Zel'dovich epilogue (Eq. 3) or a plain real
// output (density).
struct ZInvArgs {
  const void *src;        // nlines * (N/2) complex
  void *psi;              // N^3 reals or nullptr
  void *pos;
  void *vel;
  int64_t nlines;
  int n;
  int lines_per_cta;
  int comp;               // 0, 1, 2: axis of the component (lattice coordinate)
  int mul_kz;             // 1: multiply the half spectrum by i m_z before the c2r
  double box;
  double cell;            // L / N
  double q_offset;        // 0.5 (cell centres) or 0 (corners)
  double vfac;
  FftStages st;           // length N/2
  const void *tw_half;
  const void *tw_full;
  int *err;               // device error word
  int variant;            // tile variant of the size-specialised kernel
  int64_t lines_per_real; // lines of one realization (<= 0: nlines)
  int accumulate;         // psi output: psi += alpha * result instead of psi = result
  double alpha;
  void *const *psi_list;  // batched form: device arrays of per-realization outputs
  void *const *pos_list;  // (entries may be null); when set they replace psi/pos/vel
  void *const *vel_list;
  int lists_full;         // every entry of pos_list and vel_list is set (batched form)
  // Sec. 2.4 merge: a coarse periodic grid of n_low^3 reals (cell-centred)
  // whose cloud-in-cell interpolation to this grid's cell centres is added to
  // the transform's output before the epilogue; nullptr: none
  const void *large;
  int n_low;
  // Sec. 2.2 particle options: shift added to q for pos (periodic shift, and
  // the dark-matter offset of gas pairs); pos2: a second position output
  // (the gas partners) with its own shift2; nullptr: none
  double shift;
  void *pos2;
  double shift2;
};

// Cloud-in-cell density of the Zel'dovich particles and its adjoint. Particle
// p sits at u_j = i_j + q_offset - 1/2 + psi_j[p] / cell (grid units, nodes at
// cell centres); it adds prod_j w_j to the 8 nodes around it with linear
// weights (1 - f, f), periodic.
struct CicArgs {
  const void *psi[3];     // N^3 reals each
  void *delta;            // deposit: N^3 reals (set to -1 first, then += weights)
  const void *g_delta;    // adjoint: N^3 reals
  void *g_psi[3];         // adjoint: d/dpsi_j of sum_c g(c) delta(c)
  int n;
  double cell;            // L / N
  double q_offset;        // 0.5 or 0
};
template <typename R> cudaError_t launch_cic_deposit(const CicArgs &a, cudaStream_t s);
template <typename R> cudaError_t launch_cic_adjoint(const CicArgs &a, cudaStream_t s);

// Eq. 5 with the cloud-in-cell deconvolution on a half spectrum (gg_merge.cu).
struct SpecScaleArgs {
  void *spec;               // N x N x N/2 complex, in place
  int n;
  int64_t qmax;             // modes with m2 >= qmax become 0
  const void *axis_factor;  // N reals: 1 / sinc^2(pi m_i / N) per array index (0 at N/2)
  double scale;             // 1 / N^3 (unnormalised forward and inverse transforms)
};
template <typename R> cudaError_t launch_spectrum_scale(const SpecScaleArgs &a, cudaStream_t s);
// Sec. 2.4 degrading: multiply a half spectrum by phase[x] phase[y] phase[k_z]
// (complex, N entries, 0 at N/2) and scale.
struct SpecPhaseArgs {
  void *spec;
  int n;
  const void *phase;  // N complex of the spectrum's type
  double scale;
};
template <typename R> cudaError_t launch_spectrum_phase(const SpecPhaseArgs &a, cudaStream_t s);
// every r-th value of a fine n_high^3 grid into a coarse (n_high / r)^3 grid
template <typename R>
cudaError_t launch_subsample(const void *fine, int64_t n_high, int r, void *coarse, cudaStream_t s);
// coordinate-based particle IDs (Sec. 2.2), int64 per cell of an N^3 grid
cudaError_t launch_particle_ids(int64_t n, int64_t n_finest, int64_t offset, int64_t *ids,
                                cudaStream_t s);

// Sec. 2.1 diagnostics (gg_stats.cu).
struct ShellArgs {
  const void *spec;  // N x N x N/2 complex (unnormalised forward transform)
  int n;
  int nbins;         // shells 0 .. nbins - 1 (nbins <= N / 2)
  double *sums;      // device, added to: geometry [2][nbins] weight, weight |m|;
                     // otherwise [nbins] weight |F|^2
};
template <typename R> cudaError_t launch_shell_sums(const ShellArgs &a, bool geometry, cudaStream_t s);
struct MomentArgs {
  const void *field;
  int64_t count;
  int second;        // 0: sum of values; 1: sum of squared deviations from mean
  double mean;
  double *slots;     // device [3 per CTA]: sum, min, max
};
template <typename R> int moment_blocks(int64_t count);
template <typename R> cudaError_t launch_moments(const MomentArgs &a, int blocks, cudaStream_t s);

struct NoiseArgs {
  void *out;              // N^3 reals
  uint64_t seed;
  int64_t cells;
};

template <typename R> cudaError_t launch_noise(const NoiseArgs &a, cudaStream_t s);
template <typename R> cudaError_t launch_zfwd(const ZFwdArgs &a, cudaStream_t s);
template <typename R> cudaError_t launch_axis(const AxisArgs &a, cudaStream_t s);
template <typename R> cudaError_t launch_zinv(const ZInvArgs &a, cudaStream_t s);
template <typename R> int max_block_threads_z(int kind, int e);  // kind 0: z forward, 2: z inverse
template <typename R> int max_block_threads_axis(int e);
// Size-specialised kernels (gg_ct_f32.cu / gg_ct_f64.cu) for the grid sizes of
// the named workloads; spec_has tells whether N has them.
template <typename R> bool spec_has(int n);
constexpr int kSpecAxisVariants = 3;  // tile variants the autotuner times per strided pass
constexpr int kSpecZVariants = 4;     // ... per z pass
template <typename R> cudaError_t spec_axis(const AxisArgs &a, cudaStream_t s);
// Tile width (complex columns) of the size-specialised strided pass at n in
// tile variant v (0 when n has no specialised kernels).
template <typename R> int spec_axis_cols(int n, int v);
template <typename R> cudaError_t spec_zinv(const ZInvArgs &a, cudaStream_t s);
template <typename R> cudaError_t spec_zfwd(const ZFwdArgs &a, cudaStream_t s);
// Persistent batched form (gg_persist.cu): every pass of every realization
// of a batch in one launch. Work items (pass, group, tile) are taken in that
// order from a device queue; a tile starts once its realization has
// completed every tile of the pass it reads (per-realization pass counters,
// bounded waits), then adds itself to its own pass's counter.
constexpr int kPersistMaxGroups = 4;
constexpr int kPersistPasses = 8;  // z fwd, y fwd, x fused, y inv (x), y inv (y/z), z inv x3
struct PersistGroupArgs {
  int n;                  // FP32, one of the sizes persist_has accepts
  int nb;                 // realizations of the group
  int first;              // index of its first realization in the pass counters
  int plain;              // z inverse: every realization wants pos and vel (no psi)
  int zi_on[3];           // which z inverse passes run
  ZFwdArgs zf;
  AxisArgs ax[4];         // y forward, x fused, y inverse (x branch), y inverse (y/z)
  ZInvArgs zi[3];
};
struct PersistPlan {
  int ngroups;
  int realizations;       // summed over the groups
  PersistGroupArgs g[kPersistMaxGroups];
  unsigned int *counters; // device, 64 + 8 * realizations words, zeroed before each launch
  int *err;               // device error word (2: a wait gave up)
  uint32_t wait_us;       // limit of every wait (0: two seconds)
  int chunk;              // most tiles per work item (a power of two; 0: 64)
  int test_stall;         // fault test: the first y forward item never counts itself done
};
bool persist_has(int n);
// Fills the tile shapes and tensor maps and launches on s (capturable).
cudaError_t launch_persist(PersistPlan p, cudaStream_t s, int *launched_blocks);

// Message returned by gg_last_error(NULL) on this host thread.
void set_thread_error(const char *msg);
cudaError_t launch_noise_bits(uint64_t seed, int64_t first, int64_t count, uint32_t *out,
                              cudaStream_t s);

// Shared-memory bytes of one CTA of each pass (the host sizes tiles with these).
size_t zpass_smem_bytes(int half_len, int lines, size_t complex_bytes);
size_t axis_smem_bytes(int len, int cols, size_t complex_bytes);
// Lines per CTA of the run-time z passes (forward and inverse) for lines of
// st_half.len complex points: about 256 threads, halved while the CTA would
// exceed the register cap of either kernel or the shared-memory limit.
template <typename R> int z_lines_per_cta(const FftStages &st_half);
// The FP64 cosmology of *p (growth, velocity factor, ...) and the Eq. 1
// filter S(m2) = D sqrt(P(k)/V) for m2 < count, from one evaluation of the
// model (its sigma_8 and growth integrals). Returns false with *msg set when
// *p is invalid.
bool info_and_filter(const gg_params *p, gg_info *info, double *s, int64_t count, const char **msg);

}  // namespace gg
