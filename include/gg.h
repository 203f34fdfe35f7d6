/*
 * gg.h -- C ABI of the GB300 (sm_103a) Zel'dovich initial-conditions path.
 *
 * The method is that of Ginnungagap (arXiv:2511.10353): Gaussian white noise
 * on a periodic N^3 grid (Sec. 2, step 1) is convolved with the square root
 * of the power spectrum in Fourier space (Sec. 2.1, Eq. 1), turned into the
 * three displacement/velocity-field components psi~_j = i k_j delta~ / k^2
 * (Eq. 2) and finally into Zel'dovich particle positions and velocities
 * (Sec. 2.2, Eq. 3).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid:  N points per axis (N even, N = 2^a 3^b, 4 <= N <= 4096), box side
 *        L [Mpc/h], cell Delta = L/N. Real fields are N^3 arrays in C order
 *        with z fastest: idx = (i_x N + i_y) N + i_z.
 * Type:  GG_F32 -> float, GG_F64 -> double for every real array of a plan.
 * Noise: W(idx) from Philox4x32-10 (Salmon et al., SC'11) with counter
 *        (g_lo, g_hi, 0, 0), g = idx >> 2, key (seed_lo, seed_hi); lane
 *        idx & 3 selects one output of the two Box-Muller pairs
 *        (u_a = (r_2p + 1) 2^-32, u_b = r_2p+1 2^-32, p = lane >> 1;
 *        W = sqrt(-2 ln u_a) cos(2 pi u_b) for even lanes, sin for odd).
 * Fourier: forward transform orthonormal, inverse unnormalised; the filter
 *        is D(z) sqrt(P(k)/V), V = L^3. Modes with k = 0 or any |m_j| = N/2
 *        are zeroed.
 * Output: psi_j = displacement [Mpc/h] (carries D(z)); pos_j = (q_j + psi_j)
 *        mod L with q_j = (i_j + 1/2) Delta (or i_j Delta with GG_Q_CORNER);
 *        vel_j = 100 a E(a) f(a) psi_j [km/s, peculiar].
 *
 * Memory ownership: the caller owns every input/output buffer; device
 * pointers must be CUDA device memory on the plan's device, aligned to 16
 * bytes. The plan owns its workspace and FP64-generated tables.
 *
 * Asynchrony: compute calls enqueue work on the plan's stream and return at
 * once. Argument errors return GG_EINVAL before anything is enqueued. Launch
 * errors return GG_ECUDA. The one error detected on the device, a tile-copy
 * wait that gave up (GG_ETIMEOUT, after two seconds), is latched in a device
 * word and returned by the next gg_sync(), which clears it.
 *
 * Thread safety: a plan may be used by one host thread at a time. Distinct
 * plans are independent.
 */
#ifndef GG_H
#define GG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GG_OK = 0,
  GG_EINVAL = -1,   /* invalid argument; nothing enqueued */
  GG_ENOMEM = -2,   /* device or host allocation failed */
  GG_ECUDA = -3,    /* a CUDA runtime call or a kernel launch failed */
  GG_ETIMEOUT = -4  /* a bounded device-side wait gave up */
} gg_status;

typedef enum { GG_F32 = 0, GG_F64 = 1 } gg_prec;

typedef enum {
  GG_TF_BBKS = 0,        /* Bardeen, Bond, Kaiser & Szalay (1986) eq. G3, q = k/(Om h) */
  GG_TF_EH_NOWIGGLE = 1, /* Eisenstein & Hu (1998) eqs. 26, 28-31 */
  GG_TF_TABLE = 2        /* caller's tabulated P(k, z=0), log-log interpolated */
} gg_tf;

/* Lagrangian lattice at cell corners (q = i Delta) instead of centres. */
#define GG_Q_CORNER 0x1u

/* Cosmological parameters and power spectrum (Sec. 2.1: "cosmological
 * parameters and the power spectrum in tabulated form"). */
typedef struct {
  double omega_m;  /* matter density today, > 0 */
  double omega_l;  /* Lambda today; < 0 means 1 - omega_m (flat) */
  double omega_b;  /* baryons (EH no-wiggle only) */
  double h;        /* H0 / (100 km/s/Mpc), > 0 */
  double n_s;      /* primordial spectral index */
  double sigma_8;  /* > 0: normalise sigma(8 Mpc/h, z=0); 0 with GG_TF_TABLE: keep the
                      table's amplitude */
  double t_cmb;    /* CMB temperature [K] (EH no-wiggle only) */
  int32_t tf;      /* gg_tf */
  int32_t reserved;
  const double *tab_k; /* GG_TF_TABLE: k [h/Mpc], strictly increasing, host memory */
  const double *tab_p; /* GG_TF_TABLE: P(k, z=0) [(Mpc/h)^3] > 0, host memory */
  int64_t tab_n;       /* GG_TF_TABLE: number of table rows, >= 2 */
} gg_cosmo;

/* One problem: grid, box, precision, cosmology, initial redshift. */
typedef struct {
  int64_t n;        /* grid points per axis */
  double box;       /* L [Mpc/h] > 0 */
  int32_t prec;     /* gg_prec */
  uint32_t flags;   /* GG_Q_CORNER */
  gg_cosmo cosmo;
  double z_init;    /* initial redshift >= 0 */
  double growth_override[2]; /* {D(z)/D(0), f(z)}; NaN entries are computed (FP64) */
} gg_params;

/* Scalars a plan derived from its parameters on the host in FP64. */
typedef struct {
  double a;          /* 1/(1+z_init) */
  double growth;     /* D(a)/D(1) */
  double growth_rate;/* f = dlnD/dlna */
  double hubble;     /* E(a) = H(a)/H0 */
  double vfac;       /* 100 a E f: km/s per Mpc/h of displacement */
  double amplitude;  /* A in P(k, 0) = A k^n_s T(k)^2 (or the table scale) */
  double sigma_8;    /* sigma(8 Mpc/h) of the normalised P at z = 0 */
  int64_t n;
  int64_t workspace_bytes;
} gg_info;

typedef struct gg_plan gg_plan_t;

/* Library version (major*10000 + minor*100 + patch). */
int gg_version(void);

/* Validate *p and compute the derived FP64 scalars on the host (no device use).
 * Returns GG_EINVAL for invalid parameters. */
gg_status gg_cosmo_eval(const gg_params *p, gg_info *out);

/* Normalised linear P(k) at z = 0 [(Mpc/h)^3] at `count` wavenumbers k [h/Mpc]
 * (host arrays). Host only: the same FP64 code that fills a plan's tables. */
gg_status gg_power(const gg_params *p, const double *k, double *pk, int64_t count);

/* The FP64 density filter S(m2) = D sqrt(P(2 pi sqrt(m2)/L) / V) for integer
 * m2 = 0 .. count-1 (S(0) = 0), before the N^-3/2 transform factor. Host only. */
gg_status gg_filter_table(const gg_params *p, double *s, int64_t count);

/* Device bytes a plan for *p allocates (workspace + tables). Host only. */
gg_status gg_workspace_size(const gg_params *p, size_t *bytes);

/* Create a plan on the current CUDA device: validates *p, computes the FP64
 * scalars and tables (Sec. 2.1 inputs), allocates the workspace.
 * `stream` is a cudaStream_t (NULL = the legacy default stream).
 * On failure *plan is NULL and the status says why. */
gg_status gg_plan(gg_plan_t **plan, const gg_params *p, void *stream);

/* Change the stream later calls enqueue on. */
gg_status gg_set_stream(gg_plan_t *plan, void *stream);

/* Derived scalars of a plan. */
gg_status gg_plan_info(const gg_plan_t *plan, gg_info *out);

/* Sec. 2, step 1: write W(idx) for all N^3 cells to noise_dev (N^3 reals of the
 * plan's type, caller-owned device memory). */
gg_status gg_white_noise(gg_plan_t *plan, uint64_t seed, void *noise_dev);

/* Raw Philox4x32-10 words for group counters first_group .. first_group+count-1
 * under `seed`: out_dev[4 i + w] = word w of counter first_group + i
 * (uint32, device memory, 4*count entries). `stream` as in gg_plan. The
 * integers behind W are bit-exact and independent of launch shape. */
gg_status gg_noise_bits(uint64_t seed, int64_t first_group, int64_t count, uint32_t *out_dev,
                        void *stream);

/* Sec. 2.1, Eq. 1: the density field delta(x) = sum_k delta~(k) e^{ik.x} with
 * delta~ = D sqrt(P/V) W~. noise_dev = NULL generates W from `seed` inside the
 * first transform pass; otherwise noise_dev (N^3 reals) is read and `seed`
 * ignored. delta_dev: N^3 reals, caller-owned. */
gg_status gg_gaussian_field(gg_plan_t *plan, uint64_t seed, const void *noise_dev,
                            void *delta_dev);

/* Secs. 2.1-2.2, Eqs. 1-3: noise -> delta~ -> psi_j (one component at a time)
 * -> Zel'dovich positions and velocities. Each of psi_dev[j], pos_dev[j],
 * vel_dev[j] (j = x, y, z) is NULL or an N^3-real device buffer; a component
 * with all three NULL is skipped. noise_dev as in gg_gaussian_field. The
 * arrays psi_dev, pos_dev, vel_dev themselves may be NULL (= all NULL). */
gg_status gg_zeldovich(gg_plan_t *plan, uint64_t seed, const void *noise_dev,
                       void *const psi_dev[3], void *const pos_dev[3], void *const vel_dev[3]);

/* gg_zeldovich with HOST buffers (pinned memory recommended): copies
 * noise_host (NULL = generate from seed) to the device and runs the path.
 * A component whose requested outputs are all pinned, mapped host memory is
 * written there directly by the last pass (on a coherent CPU-GPU node, over
 * the chip-to-chip link); otherwise each output goes through a device
 * staging buffer and a copy that overlaps the compute of the next
 * component. Synchronous: returns when the outputs are in host memory. */
gg_status gg_zeldovich_host(gg_plan_t *plan, uint64_t seed, const void *noise_host,
                            void *const psi_host[3], void *const pos_host[3],
                            void *const vel_host[3]);

/* Per-kernel timing: with `enable` != 0 every launch of the plan is bracketed
 * by CUDA events recorded on the plan's stream (the stream the kernel runs
 * on); gg_profile_read reports the accumulated device time per kernel kind. */
gg_status gg_set_profiling(gg_plan_t *plan, int enable);

/* Accumulated device time of each kernel kind since the last reset. On entry
 * *count is the capacity of the arrays; on return the number of kinds
 * written. names[i] are static strings; ms[i] the summed milliseconds;
 * launches[i] the launch count; bytes[i] the algorithmic HBM bytes of one
 * launch (compulsory reads + writes of that pass). Synchronises the plan's
 * stream. reset != 0 clears the accumulators afterwards. */
gg_status gg_profile_read(gg_plan_t *plan, int reset, int *count, const char **names, double *ms,
                          int64_t *launches, double *bytes);

/* Autotuner of the transform tiles (grid sizes with size-specialised kernels:
 * N = 64, 128, 192, 256, 384, 512, 1536 in FP32; 64, 512, 1536 in FP64).
 * Runs the whole path `reps` times per tile variant on the plan's own buffers
 * (allocating the component workspaces and one scratch grid for the call),
 * times each pass with CUDA events and keeps the fastest variant per pass for
 * later calls. Synchronous. Other sizes: returns GG_OK and changes nothing.
 * Results do not depend on the variant (same arithmetic, different tiling). */
gg_status gg_autotune(gg_plan_t *plan, int reps);

/* The tile variant in use per pass: out[0] z forward, [1] y forward,
 * [2] x fused, [3] y inverse (x branch), [4] y inverse (y/z branches),
 * [5] z inverse. */
gg_status gg_plan_variants(const gg_plan_t *plan, int32_t out[6]);

/* Sets the tile variant per pass explicitly (same layout as gg_plan_variants;
 * the z passes [0] and [5] take 0..3, the strided passes 0..2; other values
 * are rejected). */
gg_status gg_plan_set_variants(gg_plan_t *plan, const int32_t v[6]);

/* Layout of the spectrum between the y forward and the y inverse passes of
 * a three-component run (pos and/or vel of all components, no psi output,
 * no Sec. 2.4 cut): 0 plain [x][y][k_z]; 1 chunk-major [k_z chunk][x][y]
 * [tile width], in which a tile of the x pass spans a few hundred kilobytes
 * per chunk instead of one memory page per row. Results are bit-identical
 * (same arithmetic in the same order). The chunk-major layout needs the four
 * strided passes' variants to share a tile width; otherwise the plain one
 * runs. gg_autotune chooses between them; gg_plan_layout reports the layout
 * the next run takes (1 only where the chunk-major one applies). */
gg_status gg_plan_set_layout(gg_plan_t *plan, int32_t chunked);
gg_status gg_plan_layout(const gg_plan_t *plan, int32_t *out);

/* ---------------------------------------------------------------- batched form
 * Many independent realizations (each its own gg_params; seeds given per run)
 * in one set of launches. Realizations with identical parameters form a
 * group with one contiguous workspace; every pass of a group runs as one
 * persistent launch over all its realizations (tile -> realization, tile),
 * the groups run on forked streams, and the whole launch sequence is captured
 * into one CUDA graph on the first gg_batch_run and replayed afterwards (seeds
 * and output pointers are refreshed through captured copies from pinned host
 * staging). Noise of realization r is that of a solo gg_zeldovich with
 * seeds[r]: results equal the solo runs. */
typedef struct gg_batch gg_batch_t;

/* Plan `count` realizations (params[i], host array) on the current device;
 * `stream` as in gg_plan. Allocates each group's workspace (3 grids per
 * realization) and tables. */
gg_status gg_batch_plan(gg_batch_t **batch, const gg_params *params, int count, void *stream);

/* Autotune every group's tiles (as gg_autotune; synchronous). Call before
 * the first gg_batch_run (a captured graph keeps the tiles it was captured
 * with; autotuning afterwards drops the graph). */
gg_status gg_batch_autotune(gg_batch_t *batch, int reps);

/* Run all realizations: seeds[count] (host); psi/pos/vel are host arrays of
 * 3*count device pointers (entry 3*i + j: component j of realization i, N_i^3
 * reals; NULL skips that output; the arrays themselves may be NULL). The set
 * of non-NULL outputs must be the same on every call (else the graph is
 * captured again). Asynchronous on the batch's stream; gg_batch_sync waits. */
gg_status gg_batch_run(gg_batch_t *batch, const uint64_t *seeds, void *const *psi,
                       void *const *pos, void *const *vel);

/* Wait for the last gg_batch_run; return the first device error. */
gg_status gg_batch_sync(gg_batch_t *batch);

/* Schedule of later gg_batch_run calls: on = 0 (default) one launch per pass
 * and group as above; on = 1 the whole batch as ONE persistent launch
 * (captured in the graph after the staging copies and a clear of its
 * counters). Its CTAs take work items (pass, group, tile), numbered
 * pass-major, from a device counter; a tile starts once its realization has
 * completed every tile of the pass it reads (per-realization pass counters)
 * and then counts itself done. Every wait is bounded (two seconds, then
 * GG_ETIMEOUT from gg_batch_sync). Same butterflies as the per-pass launches
 * (bit-identical results: only the tile shape differs). A work item is a
 * run of consecutive tiles of one pass and realization (the bodies
 * double-buffer their copies across it): on = 1 takes runs of up to 64
 * tiles, on = 2, 4, ..., 256 runs of up to that many (single tiles cost
 * 1.7x, 64-tile runs match the per-pass launches on the 48-realization
 * workload). Requires FP32
 * realizations of N = 64, 128, 192, 256 or 384 in at most 4 parameter groups
 * (else GG_EINVAL); allocates the counters (64 + 8 * count words) on first
 * use. Waits for a previous run and drops the captured graph. */
gg_status gg_batch_set_persistent(gg_batch_t *batch, int on);

/* Fault test of the persistent launch's bounded waits (no paper
 * counterpart; off unless armed). kind GG_TEST_STALL_COUNT makes the next
 * gg_batch_run's first y forward work item of the first group skip counting
 * itself done: every wait on that pass of that realization gives up after
 * wait_us microseconds (1 <= wait_us <= 1000000), the launch stops early
 * (its outputs are meaningless) and gg_batch_sync returns GG_ETIMEOUT. The
 * graph is captured again for that run and again after it; later runs are
 * normal. Needs the persistent schedule (else GG_EINVAL). GG_TEST_NONE
 * disarms. No GPU fault, trap or unbounded wait is involved. */
#define GG_TEST_STALL_COUNT 2
gg_status gg_batch_test_arm_fault(gg_batch_t *batch, int kind, uint32_t wait_us);

/* Number of groups and total cells of the batch. */
gg_status gg_batch_info(const gg_batch_t *batch, int *groups, int64_t *cells);

/* Kernels one gg_batch_run launches: the kernel nodes of the captured CUDA
 * graph (0 before the first gg_batch_run). */
gg_status gg_batch_launches(const gg_batch_t *batch, int *kernels);

void gg_batch_free(gg_batch_t *batch);

/* Largest grid (points per axis) that gg_gaussian_field_static accepts. */
#define GG_STATIC_MAX_N 64

/* The density field of gg_gaussian_field, for grids of at most
 * GG_STATIC_MAX_N^3 cells, without any device allocation. (The paper has no
 * counterpart: this is a calling convention of this library.)
 *
 * For callers that cannot call cudaMalloc: e.g. an application whose device
 * memory is all owned by its own pool allocator, or code that must not incur
 * cudaMalloc's implicit synchronisation. Instead of a plan's workspace, the
 * call uses fixed arrays in the library's device image (about 2.2 MB per GPU
 * that loads the library, held until the process exits). The caller still
 * passes the input (noise_dev: N^3 reals of the precision in *p, or NULL to
 * generate Philox noise from `seed`) and the output (delta_dev: N^3 reals),
 * both 16-byte aligned device memory; `stream` is a cudaStream_t (NULL = the
 * legacy default stream). Synchronous: returns after the result is written.
 *
 * All calls on one device from any stream or host thread of the process
 * share those arrays: calls whose work overlaps on the GPU race and corrupt
 * each other's results, so serialise them. The first call on each device
 * looks the arrays' device addresses up (it may load the library's device
 * code) and keeps them for the life of the process: cudaDeviceReset between
 * calls is not supported. The call copies host-made tables with
 * cudaMemcpyAsync from host stack memory and synchronises its stream before
 * returning, so it cannot be called while its stream is being captured.
 * n > GG_STATIC_MAX_N returns GG_EINVAL with a message in gg_last_error(NULL);
 * invalid parameters as in gg_plan. */
gg_status gg_gaussian_field_static(const gg_params *p, uint64_t seed, const void *noise_dev,
                                   void *delta_dev, void *stream);

/* ---------------------------------------------------------------- adjoint form
 * Pieces of a differentiable chain noise -> displacement -> CIC density ->
 * smoothed density for gradient-based fitting of constrained realizations
 * (no paper counterpart; the map W -> psi is that of Eqs. 1-2). */

/* Transpose of the linear map W -> psi_j (Eqs. 1-2) applied to upstream
 * gradients: g_noise = sum_j J_j^T g_psi[j]. Each J_j multiplies the spectrum
 * by the purely imaginary, Hermitian i k_j D sqrt(P/V) / k^2, so J_j^T = -J_j:
 * g_noise = -sum_j J_j g_psi[j], one forward chain per non-NULL component;
 * no transform intermediates are stored. g_psi entries: N^3 reals or NULL;
 * g_noise_dev: N^3 reals (overwritten). */
gg_status gg_zeldovich_adjoint(gg_plan_t *plan, const void *const g_psi_dev[3], void *g_noise_dev);

/* Gaussian smoothing out = F^-1[exp(-k^2 R^2 / 2) F in] (R in Mpc/h, modes with
 * |m_j| = N/2 dropped); symmetric, hence its own adjoint. in may equal out. */
gg_status gg_smooth(gg_plan_t *plan, double radius, const void *in_dev, void *out_dev);

/* Cloud-in-cell density contrast of one particle per Lagrangian cell at
 * x = q + psi (periodic): delta(c) = sum_p w_c(x_p) - 1, nodes at the cell
 * centres, linear weights per axis. psi_dev: 3 x N^3 reals; delta_dev: N^3. */
gg_status gg_cic_density(gg_plan_t *plan, const void *const psi_dev[3], void *delta_dev);

/* Adjoint of gg_cic_density at psi: g_psi[j](p) = sum_c g_delta(c) dw_c(x_p)/dpsi_j
 * (one-sided where a particle sits exactly on a node plane). NULL entries of
 * g_psi_dev are skipped. */
gg_status gg_cic_density_adjoint(gg_plan_t *plan, const void *const psi_dev[3],
                                 const void *g_delta_dev, void *const g_psi_dev[3]);

/* ------------------------------------------------------------ particle options
 * Sec. 2.2 (particle generation) and Sec. 2.4 (degrading). */

/* Periodic shift (Mpc/h) added to every position the plan writes from now
 * on: x = (q + shift + psi) mod L (e.g. to put a zoom region at the box
 * centre). {0, 0, 0} turns it off. */
gg_status gg_set_shift(gg_plan_t *plan, const double shift[3]);

/* gg_zeldovich with gas partners: each dark-matter particle gets a gas
 * particle half a cell away along every axis, and both move so that the
 * pair's centre of mass stays at the particle: dark matter at
 * x - f d, gas at x + (1 - f) d, d = (L / 2N)(1, 1, 1), f = gas_fraction
 * (the gas mass fraction Omega_b / Omega_m, in [0, 1)); velocities (and psi)
 * are shared. pos_dm_dev[j] and pos_gas_dev[j] are given (or NULL) together.
 * Other arguments as gg_zeldovich. */
gg_status gg_zeldovich_gas(gg_plan_t *plan, uint64_t seed, const void *noise_dev, double gas_fraction,
                           void *const psi_dev[3], void *const pos_dm_dev[3],
                           void *const pos_gas_dev[3], void *const vel_dev[3]);

/* Coordinate-based particle IDs: ids_dev[(i N + j) N + k] (int64, N^3,
 * caller-owned device memory) = offset + (I n_finest + J) n_finest + K,
 * (I, J, K) = r (i, j, k) + floor(r / 2), r = n_finest / N: the cell of the
 * simulation's finest grid (n_finest points per axis, a multiple of N) that
 * holds the particle's Lagrangian position, so the ID gives that position
 * back at every zoom level. */
gg_status gg_particle_ids(gg_plan_t *plan, int64_t n_finest, int64_t offset, int64_t *ids_dev);

/* Sec. 2.4: degrade a field of n_high^3 points (n_high = r N) to the plan's
 * grid: coarse cell i takes the fine value at index r i (nearest grid
 * point), and the coarse field is moved in Fourier space by (r - 1) / (2 r)
 * cells along each axis so that the values sit at the coarse cell centres
 * (modes with any |m_j| = N/2 dropped). high_dev: n_high^3 reals, low_dev:
 * N^3 reals of the plan's type, 16-byte aligned. */
gg_status gg_degrade(gg_plan_t *plan, int64_t n_high, const void *high_dev, void *low_dev);

/* ---------------------------------------------------------------- diagnostics
 * Sec. 2.1: statistics of the white noise and the fields, and the power
 * spectrum measured from a field. Both calls are synchronous (they return
 * after the result is on the host) and use the plan's stream. */

/* P(b) = (V / N^6) <|F(k)|^2> over the modes of shell b = floor(|m| + 1/2),
 * b = 0 .. nbins - 1, F the unnormalised DFT of field_dev (N^3 reals of the
 * plan's type, 16-byte aligned); k_out[b] = mean |k| of the shell's modes
 * (h/Mpc), count_out[b] = modes of the full spectrum in the shell; modes
 * with any |m_j| = N/2 are left out. 1 <= nbins <= N/2; any output may be
 * NULL. Overwrites the plan's workspace. */
gg_status gg_power_spectrum(gg_plan_t *plan, const void *field_dev, int nbins, double *k_out,
                            double *p_out, int64_t *count_out);

/* out = {mean, variance (population), minimum, maximum} of field_dev (N^3
 * reals of the plan's type), accumulated in FP64. */
gg_status gg_field_moments(gg_plan_t *plan, const void *field_dev, double out[4]);

/* ------------------------------------------------------- large/small-scale merge
 * Sec. 2.4, Eqs. 4-5: the velocity field of a refined (high-resolution)
 * white noise takes its small scales from the fine grid and its large scales
 * from the coarse grid's field. k is the angular wavenumber 2 pi m / L; the
 * spherical top hat f(|k| r_s) = [|k| r_s < 1] splits them (the paper takes
 * r_s = 2 L / N_low). Grid values sit at cell centres. */

/* Eq. 5 with the cloud-in-cell deconvolution, on a real field of the plan's
 * grid: out = F^-1[ f(|k| r_s) F[in] / prod_j sinc^2(pi m_j / N) ] (modes with
 * any |m_j| = N/2 dropped). in_dev, out_dev: N^3 reals, 16-byte aligned,
 * caller-owned, may be the same buffer. Uses the plan's workspace. */
gg_status gg_large_scales(gg_plan_t *plan, double r_s, const void *in_dev, void *out_dev);

/* gg_zeldovich with Eq. 4 and the merge: the displacement of the plan's
 * grid keeps only modes with |k| r_s >= 1, then the cloud-in-cell
 * (trilinear, periodic, between cell centres) interpolation of the coarse
 * grid large_dev[j] (n_low^3 reals, e.g. gg_large_scales of a coarse plan's
 * psi_j) is added before the Eq. 3 epilogue; psi, pos and vel are those of
 * the merged displacement. NULL large_dev entries add nothing. Other
 * arguments as gg_zeldovich; 1 <= n_low <= n. */
gg_status gg_zeldovich_merge(gg_plan_t *plan, uint64_t seed, const void *noise_dev, double r_s,
                             int64_t n_low, const void *const large_dev[3], void *const psi_dev[3],
                             void *const pos_dev[3], void *const vel_dev[3]);

/* ---------------------------------------------------------------- refinement
 * Appendix A: a white-noise field of higher resolution whose large scales are
 * those of a given parent field. Each patch of N_L parent cells per axis is
 * expanded over an orthonormal parent basis F (Eq. A.1); the N_L^3
 * coefficients are kept, N_H^3 - N_L^3 new unit Gaussian coefficients are
 * added, and the patch's N_H^3 child values are W = sum a_ijk E_i E_j E_k
 * (Eqs. A.14, A.28). Kinds (cells per axis N_L -> N_H, bases): */
typedef enum {
  GG_REFINE_HR = 0,        /* 1 -> 2, Eqs. A.2-A.4 (Hoffman-Ribak) */
  GG_REFINE_3_2 = 1,       /* 2 -> 3, F: Eqs. A.5-A.6, E: Eqs. A.7-A.9 */
  GG_REFINE_2 = 2,         /* 2 -> 4, F: Eqs. A.5-A.6, E: Eqs. A.10-A.13 */
  GG_REFINE_2_LINEAR = 3,  /* 2 -> 4, E: Eqs. A.20-A.23 */
  GG_REFINE_2_SINE = 4,    /* 2 -> 4, E: Eqs. A.24-A.27 */
  GG_REFINE_4_3 = 5        /* 3 -> 4, F: the three-cell basis of Eqs. A.7-A.9,
                              E: Eqs. A.10-A.13 */
} gg_refine_kind;

typedef struct {
  int64_t n;               /* parent grid points per axis (periodic), a multiple of N_L */
  gg_prec prec;
  gg_refine_kind kind;
  int64_t origin[3];       /* first parent cell of the refined box, multiples of N_L, in [0, n) */
  int64_t extent[3];       /* parent cells per axis to refine, multiples of N_L, <= n;
                              0 => n (with origin 0: the whole box) */
} gg_refine_params;

/* Shape of the child grid gg_refine_noise writes: extent * N_H / N_L per axis. */
gg_status gg_refine_dims(const gg_refine_params *p, int64_t dims[3]);

/* Refine the parent white noise parent_dev (n^3 reals, [x][y][z], z fastest)
 * over the box of *p into child_dev (dims[0] x dims[1] x dims[2] reals of the
 * same type, [x][y][z]); both caller-owned, 16-byte aligned device memory.
 * The new coefficient (i, j, k) of the patch whose first child cell is
 * (X, Y, Z) is the white noise of seed_child (the Philox / Box-Muller mapping
 * of gg_white_noise) at child cell (X+i, Y+j, Z+k) of the whole refined grid
 * of n N_H / N_L cells per axis: the result is independent of the launch
 * shape, and a refined sub-box equals that part of the refined whole box.
 * Parent indices wrap periodically. Asynchronous on `stream` (a
 * cudaStream_t, NULL = legacy default stream). Invalid arguments return
 * GG_EINVAL before any device work, with a message in gg_last_error(NULL). */
gg_status gg_refine_noise(const gg_refine_params *p, const void *parent_dev, uint64_t seed_child,
                          void *child_dev, void *stream);

/* Wait for the plan's stream; return the first latched device error, if any
 * (GG_ETIMEOUT), and clear it. */
gg_status gg_sync(gg_plan_t *plan);

/* Fault test of the device-side waits (no paper counterpart; off unless
 * armed). kind GG_TEST_SKIP_COPY makes the next y forward pass of the plan
 * issue none of its tile copies: every CTA's first copy wait gives up after
 * wait_us microseconds (1 <= wait_us <= 1000000), the CTA returns, the rest
 * of the call runs on whatever the workspace holds (its outputs are
 * meaningless) and the next gg_sync() returns GG_ETIMEOUT. The fault applies
 * to that one launch only; later calls on the plan run normally. kind
 * GG_TEST_NONE disarms. No GPU fault, trap or unbounded wait is involved. */
#define GG_TEST_NONE 0
#define GG_TEST_SKIP_COPY 1
gg_status gg_test_arm_fault(gg_plan_t *plan, int kind, uint32_t wait_us);

/* Message of the last failed call on this plan (plan = NULL: of the last
 * failed call on this host thread that had no plan). Never NULL. */
const char *gg_last_error(const gg_plan_t *plan);

/* Release the plan's device memory. NULL is ignored. The caller must make sure
 * no enqueued work of the plan is still running (gg_sync first). */
void gg_free(gg_plan_t *plan);

#ifdef __cplusplus
}
#endif

#endif /* GG_H */
