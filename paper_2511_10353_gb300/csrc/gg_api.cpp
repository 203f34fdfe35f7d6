// C ABI of the Zel'dovich initial-conditions path (include/gg.h): parameter
// validation, FP64 tables, workspace ownership and the pass schedule.
//
// Pass schedule of gg_zeldovich (FP32 bytes per cell; FP64 doubles them):
//   z forward   noise made in registers -> half spectrum W~          write 4
//   y forward   W~ along y                                          r+w 8
//   x fused     forward x, then per output: filter, inverse x       read 4, write 4 per output
//                 A = X^-1[i m_x U W~]  (-> psi_x)
//                 B = X^-1[U W~]        (-> psi_y, psi_z)
//               with U = D sqrt(P/V) N^-3/2 (L / 2 pi) / m^2 (Eqs. 1-2)
//   y inverse   A -> Y^-1 A;  B -> Y^-1[i m_y B], Y^-1 B            read 4, write 4 per output
//   z inverse   c2r (i m_z applied on load for psi_z) + Eq. 3       read 4, write 4 per output
// i m_y and i m_z commute with the x (and y) transforms, so psi_y and psi_z
// share B: 80 B/cell for positions + velocities.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <limits>
#include <utility>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "gg.h"
#include "gg_cosmo.h"
#include "gg_internal.h"

namespace {

constexpr double kPi = 3.14159265358979323846;
thread_local std::string g_thread_error;

struct Tables {
  void *tw_n = nullptr;     // length N: exp(-2 pi i t / N)
  void *tw_half = nullptr;  // length N/2
  void *s_delta = nullptr;  // S(m2) N^-3/2, 3 (N/2)^2 + 1 entries (density filter, Eq. 1)
  void *u_phi = nullptr;    // S(m2) N^-3/2 (L / 2 pi) / m2 (potential; psi~_j = i m_j U W~)
  void *smooth = nullptr;   // exp(-k^2 R^2 / 2) / N^3 for the last gg_smooth radius
  double smooth_radius = -1.0;
  // FP32 shared-memory forms of the three filters (see AxisArgs::interp)
  void *interp_u = nullptr, *interp_s = nullptr, *interp_smooth = nullptr;
  int interp_cells = 0;
  void *cic_deconv = nullptr;  // N reals: 1 / sinc^2(pi m_i / N) per array index (Sec. 2.4)
};

}  // namespace

struct gg_plan {
  gg_params p{};
  gg_info info{};
  int device = 0;
  cudaStream_t stream = nullptr;
  size_t real_bytes = 0;  // sizeof(R)
  int64_t cells = 0;      // N^3
  void *work = nullptr;   // N^3 reals: half spectrum; the psi_x branch after the x pass
  void *work2 = nullptr;  // N^3 reals, allocated on first use: the psi_y branch
  void *work3 = nullptr;  // N^3 reals, allocated on first use: the psi_z branch
  Tables tab;
  int *err = nullptr;     // device error word
  gg::FftStages st_n{}, st_n_inv{}, st_half{};
  int z_lines = 1, col_b = 1;
  int col_e = 1, col_rows_box = 0;  // strided passes: elements per thread, TMA box height
  // tile variants of the size-specialised kernels, per pass (see gg_autotune):
  // 0 z forward, 1 y forward, 2 x fused, 3 y inverse (x branch),
  // 4 y inverse (y/z branches), 5 z inverse
  int variant[6] = {0, 0, 0, 0, 0, 0};
  int chunked = 0;  // 1: the three-component chain keeps the spectrum chunk-major
  // fault test (gg_test_arm_fault): the next y forward pass issues no copies
  int test_skip_copy = 0;
  uint32_t test_wait_us = 0;
  std::string last_error;
  // host-buffer entry point: device staging of two components, a copy stream
  void *stage[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
  void *noise_stage = nullptr;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_comp[2] = {nullptr, nullptr}, ev_copy[2] = {nullptr, nullptr};
  // per-kernel timing
  struct ProfRec { int kind; cudaEvent_t a, b; };
  bool prof_on = false;
  std::vector<ProfRec> prof;      // event pairs (reused)
  size_t prof_used = 0;
  double prof_ms[16] = {0};
  int64_t prof_launches[16] = {0};
  double prof_bytes[16] = {0};
  // Sec. 2.4 merge, set for the duration of gg_zeldovich_merge: top hat on the
  // x pass (modes with m2 < merge_qmin dropped) and the coarse grids whose
  // interpolation the z inverse passes add
  int merge_qmin = 0;
  const void *merge_large[3] = {nullptr, nullptr, nullptr};
  int merge_nlow = 0;
  // Sec. 2.2 particle options: periodic shift of every position (gg_set_shift)
  // and, for the duration of gg_zeldovich_gas, the gas partners' outputs
  double shift[3] = {0.0, 0.0, 0.0};
  double gas_fraction = 0.0;
  void *gas_pos[3] = {nullptr, nullptr, nullptr};
  void *phase = nullptr;  // degrading: N complex phases (gg_degrade)
  int64_t phase_r = 0;
  // power spectrum: the grid's shell weights and weighted |m| for shell_nb shells
  std::vector<double> shell_w, shell_m;
  int shell_nb = 0;
};

struct gg_batch {
  struct Group {
    gg_plan_t *plan = nullptr;          // tables, tiles and variants of the group
    std::vector<int> members;           // batch indices of its realizations
    void *work[3] = {nullptr, nullptr, nullptr};  // nb grids each: x, y, z branches
    uint64_t *d_seeds = nullptr;        // device [nb]
    void **d_lists = nullptr;           // device [3 outputs][3 components][nb]
    uint64_t *h_seeds = nullptr;        // pinned staging of the same
    void **h_lists = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
  };
  int count = 0;
  int64_t cells = 0;
  cudaStream_t stream = nullptr;
  std::vector<Group> groups;
  cudaEvent_t fork = nullptr, done = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint32_t signature = 0;  // which (output, component) pairs the graph writes
  bool ran = false;
  // one persistent launch for the whole batch (gg_batch_set_persistent)
  bool persistent = false;
  int persist_chunk = 0;             // most tiles per work item (0: the default)
  // fault test (gg_batch_test_arm_fault): the next persistent run stalls one
  // pass counter; the graph is captured again before and after that run
  int test_stall = 0, test_ran = 0;
  uint32_t test_wait_us = 0;
  unsigned int *counters = nullptr;  // device: work queue, abort flag, pass counters
  int persist_blocks = 0;
};

namespace {

gg_status fail(gg_plan_t *plan, gg_status st, const std::string &msg) {
  if (plan) plan->last_error = msg;
  else g_thread_error = msg;
  return st;
}

gg_status cuda_fail(gg_plan_t *plan, cudaError_t e, const char *what) {
  return fail(plan, GG_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bool smooth_23(int64_t n) {
  if (n <= 0) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  return n == 1;
}

std::string validate(const gg_params *p) {
  if (!p) return "params is NULL";
  if (p->n < 4 || p->n > 4096 || (p->n & 1) || !smooth_23(p->n))
    return "n must be even, 4 <= n <= 4096 and of the form 2^a 3^b";
  if (!(p->box > 0) || !std::isfinite(p->box)) return "box must be > 0";
  if (p->prec != GG_F32 && p->prec != GG_F64) return "prec must be GG_F32 or GG_F64";
  if (p->flags & ~GG_Q_CORNER) return "unknown flag bits";
  const gg_cosmo &c = p->cosmo;
  if (!(c.omega_m > 0) || !std::isfinite(c.omega_m)) return "omega_m must be > 0";
  if (!(c.h > 0) || !std::isfinite(c.h)) return "h must be > 0";
  if (!std::isfinite(c.n_s)) return "n_s must be finite";
  if (c.tf != GG_TF_BBKS && c.tf != GG_TF_EH_NOWIGGLE && c.tf != GG_TF_TABLE)
    return "unknown transfer function";
  if (!(c.sigma_8 > 0) && !(c.tf == GG_TF_TABLE && c.sigma_8 == 0.0))
    return "sigma_8 must be > 0 (or 0 with a table to keep its amplitude)";
  if (c.tf == GG_TF_EH_NOWIGGLE) {
    if (!(c.omega_b > 0) || !(c.omega_b < c.omega_m)) return "omega_b must be in (0, omega_m)";
    if (!(c.t_cmb > 0)) return "t_cmb must be > 0";
  }
  if (c.tf == GG_TF_TABLE) {
    if (!c.tab_k || !c.tab_p || c.tab_n < 2) return "table needs tab_k, tab_p and tab_n >= 2";
    for (int64_t i = 0; i < c.tab_n; ++i) {
      if (!(c.tab_k[i] > 0) || !(c.tab_p[i] > 0)) return "table entries must be > 0";
      if (i && !(c.tab_k[i] > c.tab_k[i - 1])) return "tab_k must be strictly increasing";
    }
  }
  if (!(p->z_init >= 0) || !std::isfinite(p->z_init)) return "z_init must be >= 0";
  const double ol = c.omega_l < 0 ? 1.0 - c.omega_m : c.omega_l;
  const double a = 1.0 / (1.0 + p->z_init);
  for (double x : {a, 1.0}) {
    const double e2 = c.omega_m / (x * x * x) + (1.0 - c.omega_m - ol) / (x * x) + ol;
    if (!(e2 > 0)) return "E(a)^2 <= 0 between z_init and today";
  }
  return "";
}

gg::cosmo::Model make_model(const gg_params *p) {
  gg::cosmo::Model m;
  const gg_cosmo &c = p->cosmo;
  m.om = c.omega_m;
  m.ol = c.omega_l < 0 ? 1.0 - c.omega_m : c.omega_l;
  m.ok = 1.0 - m.om - m.ol;
  m.ob = c.omega_b;
  m.h = c.h;
  m.ns = c.n_s;
  m.sigma8 = c.sigma_8;
  m.tcmb = c.t_cmb;
  m.tf = c.tf;
  if (c.tf == GG_TF_TABLE) {
    m.tab_k.assign(c.tab_k, c.tab_k + c.tab_n);
    m.tab_p.assign(c.tab_p, c.tab_p + c.tab_n);
  }
  m.normalise();
  return m;
}

void fill_info(const gg_params *p, const gg::cosmo::Model &m, gg_info *out) {
  const double a = 1.0 / (1.0 + p->z_init);
  out->a = a;
  out->growth = std::isnan(p->growth_override[0]) ? m.growth(a) : p->growth_override[0];
  out->growth_rate = std::isnan(p->growth_override[1]) ? m.growth_rate(a) : p->growth_override[1];
  out->hubble = m.E(a);
  out->vfac = 100.0 * a * out->hubble * out->growth_rate;
  out->amplitude = m.amp;
  out->sigma_8 = m.sigma(8.0);
  out->n = p->n;
}

size_t table_entries(int64_t n) { return (size_t)(3 * (n / 2) * (n / 2) + 1); }

size_t workspace_bytes(const gg_params *p) {
  const size_t rb = p->prec == GG_F64 ? 8 : 4;
  const size_t grid = (size_t)p->n * p->n * p->n * rb;
  return 3 * grid + (size_t)(p->n + p->n / 2) * 2 * rb + 2 * table_entries(p->n) * rb + 256;
}

template <typename R>
std::vector<R> twiddles(int len) {
  std::vector<R> t(2 * (size_t)len);
  for (int i = 0; i < len; ++i) {
    // exp(-2 pi i t / len) from FP64 cos/sin of the exactly reduced angle
    const double ang = -2.0 * kPi * (double)i / (double)len;
    t[2 * i] = (R)std::cos(ang);
    t[2 * i + 1] = (R)std::sin(ang);
  }
  return t;
}

template <typename R>
gg_status upload(gg_plan_t *plan, void **dst, const std::vector<R> &v) {
  cudaError_t e = cudaMalloc(dst, v.size() * sizeof(R));
  if (e != cudaSuccess) return fail(plan, GG_ENOMEM, "cudaMalloc (tables) failed");
  e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(R), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(plan, e, "cudaMemcpy (tables)");
  return GG_OK;
}

// S_delta(m2) = D sqrt(P(k)/V), k = 2 pi sqrt(m2) / L, S(0) = 0 (Eq. 1).
void filter_values(const gg_params *p, const gg::cosmo::Model &m, double growth, double *s,
                   int64_t count) {
  const double vol = p->box * p->box * p->box;
  for (int64_t i = 0; i < count; ++i) {
    if (i == 0) { s[0] = 0.0; continue; }
    const double k = 2.0 * kPi * std::sqrt((double)i) / p->box;
    s[i] = growth * std::sqrt(m.power(k) / vol);
  }
}

// Shared-memory form of a filter F(m2) (FP32 size-specialised kernels): the
// exact values for m2 < kInterpExact, then for each unit cell [j, j+1) of
// m = sqrt(m2) the FP64 values and derivatives (F_j, F'_j, F_j+1, F'_j+1) of
// F as a function of continuous m, rounded once; cubic Hermite interpolation
// inside a cell is accurate to < 1e-6 relative for m >= 32.
template <class F>
gg_status upload_interp(gg_plan_t *plan, void **dst, const F &fm) {
  const int64_t n = plan->p.n;
  // cells j = kInterpFirstCell ... (m2 >= kInterpExact reads no lower cell)
  const int last = (int)std::ceil(std::sqrt(3.0) * (double)(n / 2)) + 2;
  const int cells = std::max(0, last - gg::kInterpFirstCell);
  std::vector<float> buf(gg::kInterpExact + 4 * (size_t)cells);
  for (int q = 0; q < gg::kInterpExact; ++q) buf[q] = (float)fm(std::sqrt((double)q), q);
  auto d = [&](double x) {
    const double h = 1e-4 * std::max(1.0, x);
    return (fm(x + h, -1) - fm(x - h, -1)) / (2 * h);
  };
  // per cell the cubic Hermite interpolant through f and f' at both ends,
  // as its Taylor coefficients in t = m - j (FP64, rounded once), so that the
  // kernels evaluate it by Horner's rule: a0 + t (a1 + t (a2 + t a3))
  for (int i = 0; i < cells; ++i) {
    const int j = gg::kInterpFirstCell + i;
    const double x0 = (double)j, x1 = (double)j + 1.0;
    const double f0 = fm(x0, -1), d0 = d(x0), f1 = fm(x1, -1), d1 = d(x1);
    float *c = buf.data() + gg::kInterpExact + 4 * (size_t)i;
    c[0] = (float)f0;
    c[1] = (float)d0;
    c[2] = (float)(3.0 * (f1 - f0) - 2.0 * d0 - d1);
    c[3] = (float)(2.0 * (f0 - f1) + d0 + d1);
  }
  plan->tab.interp_cells = cells;
  return upload(plan, dst, buf);
}

template <typename R>
gg_status build_tables(gg_plan_t *plan, const gg::cosmo::Model &m) {
  const int64_t n = plan->p.n;
  gg_status st;
  if ((st = upload(plan, &plan->tab.tw_n, twiddles<R>((int)n))) != GG_OK) return st;
  if ((st = upload(plan, &plan->tab.tw_half, twiddles<R>((int)(n / 2)))) != GG_OK) return st;
  const size_t cnt = table_entries(n);
  std::vector<double> s(cnt);
  filter_values(&plan->p, m, plan->info.growth, s.data(), (int64_t)cnt);
  const double norm = 1.0 / std::pow((double)n, 1.5);  // orthonormal forward transform
  std::vector<R> sd(cnt), up(cnt);
  for (size_t i = 0; i < cnt; ++i) {
    sd[i] = (R)(s[i] * norm);
    up[i] = i ? (R)(s[i] * norm * plan->p.box / (2.0 * kPi * (double)i)) : (R)0;
  }
  if ((st = upload(plan, &plan->tab.s_delta, sd)) != GG_OK) return st;
  if ((st = upload(plan, &plan->tab.u_phi, up)) != GG_OK) return st;
  if (sizeof(R) == 4 && plan->p.cosmo.tf != GG_TF_TABLE) {
    // smooth analytic spectra: FP32 kernels interpolate instead of gathering
    const double box = plan->p.box, vol = box * box * box, growth = plan->info.growth;
    auto s_of = [&](double mm, int q) {  // S(m) N^-3/2 at continuous m (q: integer m2 or -1)
      if (q == 0 || mm <= 0) return 0.0;
      return growth * std::sqrt(m.power(2.0 * kPi * mm / box) / vol) * norm;
    };
    auto u_of = [&](double mm, int q) {
      if (q == 0 || mm <= 0) return 0.0;
      return s_of(mm, q) * box / (2.0 * kPi * mm * mm);
    };
    if ((st = upload_interp(plan, &plan->tab.interp_s, s_of)) != GG_OK) return st;
    if ((st = upload_interp(plan, &plan->tab.interp_u, u_of)) != GG_OK) return st;
  }
  return GG_OK;
}

template <typename R>
void choose_tiles(gg_plan_t *plan) {
  const int n = (int)plan->p.n, half = n / 2;
  const size_t cb = 2 * sizeof(R);
  plan->z_lines = gg::z_lines_per_cta<R>(plan->st_half);
  // strided passes: rows of up to 128 bytes, halved while two tiles would not
  // fit in shared memory or the CTA would exceed 512 threads (or what the
  // kernel's registers allow); TMA unless FP32 rows of N/2 complex values are
  // not a multiple of 16 bytes (odd N/2)
  int b = (int)(128 / cb);
  while (b > 1 && half % b != 0) b /= 2;
  while (b > 1 && gg::axis_smem_bytes(n, b, cb) > 200 * 1024) b /= 2;
  const int e = plan->st_n.e;
  int cap = gg::max_block_threads_axis<R>(e);
  if (cap <= 0) cap = 256;
  while (b > 1 && (n / e) * b > std::min(cap, 512)) b /= 2;
  int rows = 1;
  for (int d = 1; d <= 256 && d <= n; ++d)
    if (n % d == 0) rows = d;
  plan->col_b = b;
  plan->col_e = e;
  plan->col_rows_box = (sizeof(R) == 8 || half % 2 == 0) && (size_t)b * cb >= 16 ? rows : 0;
}

void release(gg_plan_t *plan) {
  if (!plan) return;
  void *bufs[] = {plan->work,        plan->work2,         plan->work3,
                  plan->tab.tw_n,    plan->tab.tw_half,   plan->tab.s_delta,
                  plan->tab.u_phi,   plan->err,           plan->noise_stage,
                  plan->tab.smooth,  plan->tab.interp_u,  plan->tab.interp_s,
                  plan->tab.interp_smooth, plan->tab.cic_deconv, plan->phase};
  for (void *b : bufs)
    if (b) cudaFree(b);
  for (auto &slot : plan->stage)
    for (void *b : slot)
      if (b) cudaFree(b);
  for (auto &r : plan->prof) {
    if (r.a) cudaEventDestroy(r.a);
    if (r.b) cudaEventDestroy(r.b);
  }
  for (int i = 0; i < 2; ++i) {
    if (plan->ev_comp[i]) cudaEventDestroy(plan->ev_comp[i]);
    if (plan->ev_copy[i]) cudaEventDestroy(plan->ev_copy[i]);
  }
  if (plan->copy_stream) cudaStreamDestroy(plan->copy_stream);
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// ------------------------------------------------------------ kernel timing
enum Kind { kZFwd = 0, kYFwd, kXFused, kYInvX, kYInvYZ, kZInv, kNoise, kNumKinds };
const char *const kKindNames[kNumKinds] = {"z_forward_noise", "y_forward",
                                           "x_fused_filter",  "y_inverse_x",
                                           "y_inverse_yz",    "z_inverse_epilogue",
                                           "noise"};

// An NVTX range named after the pass around every launch (visible to
// profilers and tracers; a no-op without one), and, when the plan's
// profiling is on, a start event before the launch and an end event after
// it; `bytes` is the launch's algorithmic HBM traffic.
struct ProfScope {
  gg_plan_t *plan;
  size_t slot = (size_t)-1;
  ProfScope(gg_plan_t *p, int kind, double bytes) : plan(p) {
    nvtxRangePushA(kKindNames[kind]);
    if (!plan->prof_on) return;
    if (plan->prof_used == plan->prof.size()) {
      gg_plan::ProfRec r{kind, nullptr, nullptr};
      if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) return;
      plan->prof.push_back(r);
    }
    slot = plan->prof_used++;
    plan->prof[slot].kind = kind;
    plan->prof_bytes[kind] = bytes;
    cudaEventRecord(plan->prof[slot].a, plan->stream);
  }
  ~ProfScope() {
    if (slot != (size_t)-1) cudaEventRecord(plan->prof[slot].b, plan->stream);
    nvtxRangePop();
  }
};

// ----------------------------------------------------------- pass launchers
template <typename R>
gg::AxisArgs axis_args(gg_plan_t *plan, int axis, const void *src) {
  const int n = (int)plan->p.n, half = n / 2;
  gg::AxisArgs c{};
  c.src = src;
  c.cols = plan->col_b;
  c.inner_chunks = half / plan->col_b;
  c.n = n;
  c.axis = axis;
  c.stride = axis == 1 ? half : (int64_t)n * half;
  c.outer_stride = axis == 1 ? (int64_t)n * half : half;
  c.st_fwd = plan->st_n;
  c.st_inv = plan->st_n_inv;
  c.tw = plan->tab.tw_n;
  c.e = plan->col_e;
  c.rows_box = plan->col_rows_box;
  c.err = plan->err;
  return c;
}

// One strided pass; the size-specialised kernel where N has one. Every
// output of a two-output pass comes from the one launch.
template <typename R>
gg_status launch_axis_timed(gg_plan_t *plan, const gg::AxisArgs &c, int kind, const char *what) {
  const double cb = (double)plan->cells * sizeof(R);
  const bool spec = gg::spec_has<R>(c.n);
  const double bytes = (c.fwd && !c.inv ? 2 : 1 + c.nout) * cb;
  cudaError_t e;
  {
    ProfScope ps(plan, kind, bytes);
    e = spec ? gg::spec_axis<R>(c, plan->stream) : gg::launch_axis<R>(c, plan->stream);
  }
  return e == cudaSuccess ? GG_OK : cuda_fail(plan, e, what);
}

// z forward (noise or caller noise) and y forward into plan->work.
template <typename R>
gg_status forward_zy(gg_plan_t *plan, uint64_t seed, const void *noise, void *chunked_dst = nullptr,
                     int chunk_b = 0) {
  const int n = (int)plan->p.n;
  gg::ZFwdArgs z{};
  z.noise = noise;
  z.out = plan->work;
  z.seed = seed;
  z.nlines = (int64_t)n * n;
  z.n = n;
  z.lines_per_cta = plan->z_lines;
  z.st = plan->st_half;
  z.tw_half = plan->tab.tw_half;
  z.tw_full = plan->tab.tw_n;
  z.variant = plan->variant[0];
  const double cb = (double)plan->cells * sizeof(R);
  cudaError_t e;
  {
    ProfScope ps(plan, kZFwd, noise ? 2 * cb : cb);
    e = gg::spec_has<R>(n) ? gg::spec_zfwd<R>(z, plan->stream) : gg::launch_zfwd<R>(z, plan->stream);
  }
  if (e != cudaSuccess) return cuda_fail(plan, e, "z forward pass");
  gg::AxisArgs c = axis_args<R>(plan, 1, plan->work);
  c.fwd = 1;
  c.inv = 0;
  c.nout = 1;
  c.dst[0] = chunked_dst ? chunked_dst : plan->work;
  c.mul[0] = gg::kMulNone;
  c.variant = plan->variant[1];
  if (chunked_dst) {
    c.cols = chunk_b;
    c.chunked_out = 1;
  }
  if (plan->test_skip_copy) {  // armed fault test: this launch only
    c.test_skip_copy = 1;
    c.wait_us = plan->test_wait_us;
    plan->test_skip_copy = 0;
  }
  return launch_axis_timed<R>(plan, c, kYFwd, "y forward pass");
}

template <typename R>
gg_status zinv_pass(gg_plan_t *plan, int comp, const void *src, void *psi, void *pos, void *vel,
                    bool mul_kz, bool accumulate = false, double alpha = 1.0) {
  const int n = (int)plan->p.n;
  gg::ZInvArgs z{};
  z.src = src;
  z.psi = psi;
  z.pos = pos;
  z.vel = vel;
  z.nlines = (int64_t)n * n;
  z.n = n;
  z.lines_per_cta = plan->z_lines;
  z.comp = comp;
  z.mul_kz = mul_kz ? 1 : 0;
  z.accumulate = accumulate ? 1 : 0;
  z.alpha = alpha;
  z.box = plan->p.box;
  z.cell = plan->p.box / (double)n;
  z.q_offset = (plan->p.flags & GG_Q_CORNER) ? 0.0 : 0.5;
  z.vfac = plan->info.vfac;
  z.st = plan->st_half;
  z.tw_half = plan->tab.tw_half;
  z.tw_full = plan->tab.tw_n;
  z.err = plan->err;
  z.variant = plan->variant[5];
  z.large = plan->merge_large[comp];
  z.n_low = plan->merge_nlow;
  {  // Sec. 2.2: shift, and the gas pairs' offsets of half a cell per axis
    const double half_cell = 0.5 * plan->p.box / (double)n;
    const bool gas = plan->gas_pos[comp] != nullptr;
    z.shift = plan->shift[comp] - (gas ? plan->gas_fraction * half_cell : 0.0);
    z.pos2 = plan->gas_pos[comp];
    z.shift2 = gas ? plan->shift[comp] + (1.0 - plan->gas_fraction) * half_cell : 0.0;
  }
  const double cb = (double)plan->cells * sizeof(R);
  const int outs = (psi ? 1 : 0) + (pos ? 1 : 0) + (vel ? 1 : 0);
  cudaError_t e;
  {
    ProfScope ps(plan, kZInv, (1 + outs) * cb);
    e = gg::spec_has<R>(n) ? gg::spec_zinv<R>(z, plan->stream) : gg::launch_zinv<R>(z, plan->stream);
  }
  return e == cudaSuccess ? GG_OK : cuda_fail(plan, e, "z inverse pass");
}

gg_status ensure_grid(gg_plan_t *plan, void **buf) {
  if (*buf) return GG_OK;
  if (cudaMalloc(buf, (size_t)plan->cells * plan->real_bytes) != cudaSuccess) {
    *buf = nullptr;
    return fail(plan, GG_ENOMEM, "cudaMalloc of a component workspace failed");
  }
  return GG_OK;
}

// The tile width shared by the four strided passes' variants (the width of
// a chunk-major spectrum's chunks), 0 if they differ or N has no
// size-specialised kernels.
template <typename R>
int chunk_cols(gg_plan_t *plan) {
  const int n = (int)plan->p.n;
  if (!gg::spec_has<R>(n) || plan->merge_qmin > 0) return 0;
  const int b = gg::spec_axis_cols<R>(n, plan->variant[1]);
  for (int i = 2; i <= 4; ++i)
    if (gg::spec_axis_cols<R>(n, plan->variant[i]) != b) return 0;
  return b;
}

// Positions and velocities of all three components with the spectrum
// chunk-major between the y forward and the y inverse passes ([k_z chunk][x]
// [y][cols]): a tile of the x pass, and the concurrent tiles around it, then
// span a few hundred kilobytes of each chunk instead of one memory page per
// row. Same arithmetic as the plain chain, in the same order; only the
// buffers differ:
//   y forward  work -> work3 (chunk-major)
//   x fused    work3 -> A: work3 (in place), B: work2 (both chunk-major)
//   y inverse  work3 -> work (plain); z inverse x from work
//   y inverse  work2 -> work (i m_y), work3; z inverses y, z
template <typename R>
gg_status run_zeldovich_chunked(gg_plan_t *plan, uint64_t seed, const void *noise,
                                void *const pos[3], void *const vel[3]) {
  const int b = chunk_cols<R>(plan);
  gg_status st = forward_zy<R>(plan, seed, noise, plan->work3, b);
  if (st != GG_OK) return st;
  gg::AxisArgs x = axis_args<R>(plan, 0, plan->work3);
  x.cols = b;
  x.fwd = 1;
  x.inv = 1;
  x.pre = 1;
  x.table = plan->tab.u_phi;
  x.interp = plan->tab.interp_u;
  x.interp_cells = plan->tab.interp_cells;
  x.nout = 2;
  x.dst[0] = plan->work3;
  x.mul[0] = gg::kMulIm;
  x.dst[1] = plan->work2;
  x.mul[1] = gg::kMulNone;
  x.chunked_in = 1;
  x.chunked_out = 1;
  x.variant = plan->variant[2];
  if ((st = launch_axis_timed<R>(plan, x, kXFused, "x fused pass")) != GG_OK) return st;
  gg::AxisArgs y = axis_args<R>(plan, 1, plan->work3);
  y.cols = b;
  y.inv = 1;
  y.nout = 1;
  y.dst[0] = plan->work;
  y.mul[0] = gg::kMulNone;
  y.chunked_in = 1;
  y.variant = plan->variant[3];
  if ((st = launch_axis_timed<R>(plan, y, kYInvX, "y inverse pass (x branch)")) != GG_OK) return st;
  auto out = [&](void *const *a, int j) { return a ? a[j] : nullptr; };
  if ((st = zinv_pass<R>(plan, 0, plan->work, nullptr, out(pos, 0), out(vel, 0), false)) != GG_OK)
    return st;
  gg::AxisArgs y2 = axis_args<R>(plan, 1, plan->work2);
  y2.cols = b;
  y2.inv = 1;
  y2.nout = 2;
  y2.dst[0] = plan->work;
  y2.mul[0] = gg::kMulIm;
  y2.dst[1] = plan->work3;
  y2.mul[1] = gg::kMulNone;
  y2.chunked_in = 1;
  y2.variant = plan->variant[4];
  if ((st = launch_axis_timed<R>(plan, y2, kYInvYZ, "y inverse pass (y/z branches)")) != GG_OK)
    return st;
  if ((st = zinv_pass<R>(plan, 1, plan->work, nullptr, out(pos, 1), out(vel, 1), false)) != GG_OK)
    return st;
  return zinv_pass<R>(plan, 2, plan->work3, nullptr, out(pos, 2), out(vel, 2), true);
}

// Everything up to the inverse z passes. On return src[j] holds, for each
// wanted component j, the half-spectrum lines whose c2r (times i m_z for
// j = 2) is psi_j. psi_dev[1] / psi_dev[2], when given, serve as the buffers
// of the y / z branches (the z pass then writes psi in place).
template <typename R>
gg_status spectral_passes(gg_plan_t *plan, uint64_t seed, const void *noise, const bool want[3],
                          void *const psi_dev[3], void *src[3]) {
  gg_status st = forward_zy<R>(plan, seed, noise);
  if (st != GG_OK) return st;
  void *buf_y = nullptr, *buf_z = nullptr;
  if (want[1]) {
    buf_y = (psi_dev && psi_dev[1]) ? psi_dev[1] : nullptr;
    if (!buf_y && (st = ensure_grid(plan, &plan->work2)) != GG_OK) return st;
    if (!buf_y) buf_y = plan->work2;
  }
  if (want[2]) {
    buf_z = (psi_dev && psi_dev[2]) ? psi_dev[2] : nullptr;
    if (!buf_z && (st = ensure_grid(plan, &plan->work3)) != GG_OK) return st;
    if (!buf_z) buf_z = plan->work3;
  }
  // x fused: A -> work (in place), B -> the y buffer (or the z buffer)
  void *buf_b = want[1] ? buf_y : buf_z;
  gg::AxisArgs x = axis_args<R>(plan, 0, plan->work);
  x.fwd = 1;
  x.inv = 1;
  x.pre = 1;
  x.table = plan->tab.u_phi;
  x.interp = plan->tab.interp_u;
  x.interp_cells = plan->tab.interp_cells;
  x.qmin = plan->merge_qmin;
  x.nout = 0;
  if (want[0]) {
    x.dst[x.nout] = plan->work;
    x.mul[x.nout++] = gg::kMulIm;
  }
  if (want[1] || want[2]) {
    x.dst[x.nout] = buf_b;
    x.mul[x.nout++] = gg::kMulNone;
  }
  x.variant = plan->variant[2];
  if ((st = launch_axis_timed<R>(plan, x, kXFused, "x fused pass")) != GG_OK) return st;
  if (want[0]) {
    gg::AxisArgs y = axis_args<R>(plan, 1, plan->work);
    y.inv = 1;
    y.nout = 1;
    y.dst[0] = plan->work;
    y.mul[0] = gg::kMulNone;
    y.variant = plan->variant[3];
    if ((st = launch_axis_timed<R>(plan, y, kYInvX, "y inverse pass (x branch)")) != GG_OK) return st;
  }
  if (want[1] || want[2]) {
    gg::AxisArgs y = axis_args<R>(plan, 1, buf_b);
    y.inv = 1;
    y.nout = 0;
    if (want[1]) {
      y.dst[y.nout] = buf_y;
      y.mul[y.nout++] = gg::kMulIm;
    }
    if (want[2]) {
      y.dst[y.nout] = buf_z;
      y.mul[y.nout++] = gg::kMulNone;
    }
    y.variant = plan->variant[4];
    if ((st = launch_axis_timed<R>(plan, y, kYInvYZ, "y inverse pass (y/z branches)")) != GG_OK)
      return st;
  }
  src[0] = want[0] ? plan->work : nullptr;
  src[1] = buf_y;
  src[2] = buf_z;
  return GG_OK;
}

template <typename R>
gg_status run_zeldovich(gg_plan_t *plan, uint64_t seed, const void *noise, void *const psi[3],
                        void *const pos[3], void *const vel[3]) {
  bool want[3];
  for (int j = 0; j < 3; ++j)
    want[j] = (psi && psi[j]) || (pos && pos[j]) || (vel && vel[j]);
  if (!want[0] && !want[1] && !want[2]) return GG_OK;
  const bool any_psi = psi && (psi[0] || psi[1] || psi[2]);
  if (plan->chunked && !any_psi && want[0] && want[1] && want[2] && chunk_cols<R>(plan) > 0) {
    gg_status st = GG_OK;
    if ((st = ensure_grid(plan, &plan->work2)) != GG_OK) return st;
    if ((st = ensure_grid(plan, &plan->work3)) != GG_OK) return st;
    return run_zeldovich_chunked<R>(plan, seed, noise, pos, vel);
  }
  void *src[3];
  gg_status st = spectral_passes<R>(plan, seed, noise, want, psi, src);
  if (st != GG_OK) return st;
  for (int j = 0; j < 3; ++j) {
    if (!want[j]) continue;
    st = zinv_pass<R>(plan, j, src[j], psi ? psi[j] : nullptr, pos ? pos[j] : nullptr,
                      vel ? vel[j] : nullptr, j == 2);
    if (st != GG_OK) return st;
  }
  return GG_OK;
}

template <typename R>
gg_status run_density(gg_plan_t *plan, uint64_t seed, const void *noise, void *delta,
                      const void *table = nullptr, const void *interp = nullptr) {
  gg_status st = forward_zy<R>(plan, seed, noise);
  if (st != GG_OK) return st;
  gg::AxisArgs x = axis_args<R>(plan, 0, plan->work);
  x.fwd = 1;
  x.inv = 1;
  x.pre = 1;
  x.table = table ? table : plan->tab.s_delta;
  x.interp = interp ? interp : (table ? nullptr : plan->tab.interp_s);
  x.interp_cells = plan->tab.interp_cells;
  x.nout = 1;
  x.dst[0] = plan->work;
  x.mul[0] = gg::kMulNone;
  x.variant = plan->variant[2];
  if ((st = launch_axis_timed<R>(plan, x, kXFused, "x fused pass")) != GG_OK) return st;
  gg::AxisArgs y = axis_args<R>(plan, 1, plan->work);
  y.inv = 1;
  y.nout = 1;
  y.dst[0] = plan->work;
  y.mul[0] = gg::kMulNone;
  y.variant = plan->variant[3];
  if ((st = launch_axis_timed<R>(plan, y, kYInvX, "y inverse pass")) != GG_OK) return st;
  return zinv_pass<R>(plan, 0, plan->work, delta, nullptr, nullptr, false);
}

template <typename R>
gg_status create(gg_plan_t *plan, const gg::cosmo::Model &m) {
  plan->real_bytes = sizeof(R);
  const int64_t n = plan->p.n;
  if (!gg::make_stages((int)n, &plan->st_n) || !gg::make_stages((int)(n / 2), &plan->st_half))
    return fail(plan, GG_EINVAL, "no FFT schedule for this n");
  plan->st_n_inv = gg::reversed_stages(plan->st_n);
  gg_status st = build_tables<R>(plan, m);
  if (st != GG_OK) return st;
  const size_t grid = (size_t)plan->cells * sizeof(R);
  if (cudaMalloc(&plan->work, grid) != cudaSuccess)
    return fail(plan, GG_ENOMEM, "cudaMalloc of the transform workspace failed");
  if (cudaMalloc(&plan->err, 256) != cudaSuccess)
    return fail(plan, GG_ENOMEM, "cudaMalloc of the error word failed");
  cudaError_t e = cudaMemset(plan->err, 0, 256);
  if (e != cudaSuccess) return cuda_fail(plan, e, "cudaMemset");
  choose_tiles<R>(plan);
  plan->info.workspace_bytes = (int64_t)workspace_bytes(&plan->p);
  return GG_OK;
}

// The device address of a host buffer the kernels can write directly
// (pinned and mapped; on a coherent CPU-GPU node the stores then cross the
// chip-to-chip link with no staging buffer and no copy engine); nullptr for
// any other buffer.
void *device_view(void *host) {
  if (!host) return nullptr;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, host) != cudaSuccess) {
    cudaGetLastError();  // an unregistered pointer is not an error here
    return nullptr;
  }
  if (at.type != cudaMemoryTypeHost || !at.devicePointer || !aligned16(at.devicePointer)) return nullptr;
  return at.devicePointer;
}

template <typename R>
gg_status run_host(gg_plan_t *plan, uint64_t seed, const void *noise_host, void *const psi[3],
                   void *const pos[3], void *const vel[3]) {
  const size_t grid = (size_t)plan->cells * sizeof(R);
  cudaError_t e;
  if (!plan->copy_stream) {
    if ((e = cudaStreamCreateWithFlags(&plan->copy_stream, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail(plan, e, "cudaStreamCreate");
    for (int i = 0; i < 2; ++i) {
      if ((e = cudaEventCreateWithFlags(&plan->ev_comp[i], cudaEventDisableTiming)) != cudaSuccess ||
          (e = cudaEventCreateWithFlags(&plan->ev_copy[i], cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(plan, e, "cudaEventCreate");
    }
  }
  bool want[3];
  for (int j = 0; j < 3; ++j)
    want[j] = (psi && psi[j]) || (pos && pos[j]) || (vel && vel[j]);
  if (!want[0] && !want[1] && !want[2]) return GG_OK;
  const void *noise_dev = nullptr;
  if (noise_host) {
    if (!plan->noise_stage && cudaMalloc(&plan->noise_stage, grid) != cudaSuccess)
      return fail(plan, GG_ENOMEM, "cudaMalloc of the noise staging buffer failed");
    if ((e = cudaMemcpyAsync(plan->noise_stage, noise_host, grid, cudaMemcpyHostToDevice,
                             plan->stream)) != cudaSuccess)
      return cuda_fail(plan, e, "noise upload");
    noise_dev = plan->noise_stage;
  }
  void *src[3];
  gg_status st = spectral_passes<R>(plan, seed, noise_dev, want, nullptr, src);
  if (st != GG_OK) return st;
  // inverse z per component into a staging slot; its download overlaps the
  // next component's z pass
  bool used[2] = {false, false};
  int slot = 0;
  for (int j = 0; j < 3; ++j) {
    if (!want[j]) continue;
    void *hs[3] = {psi ? psi[j] : nullptr, pos ? pos[j] : nullptr, vel ? vel[j] : nullptr};
    void *views[3] = {device_view(hs[0]), device_view(hs[1]), device_view(hs[2])};
    if ((!hs[0] || views[0]) && (!hs[1] || views[1]) && (!hs[2] || views[2])) {
      // every output of the component is device-addressable: the z inverse
      // pass writes it in place
      st = zinv_pass<R>(plan, j, src[j], views[0], views[1], views[2], j == 2);
      if (st != GG_OK) return st;
      continue;
    }
    for (int o = 0; o < 3; ++o)
      if (hs[o] && !plan->stage[slot][o] && cudaMalloc(&plan->stage[slot][o], grid) != cudaSuccess)
        return fail(plan, GG_ENOMEM, "cudaMalloc of an output staging buffer failed");
    if (used[slot] && (e = cudaStreamWaitEvent(plan->stream, plan->ev_copy[slot], 0)) != cudaSuccess)
      return cuda_fail(plan, e, "cudaStreamWaitEvent");
    void *dv[3] = {hs[0] ? plan->stage[slot][0] : nullptr, hs[1] ? plan->stage[slot][1] : nullptr,
                   hs[2] ? plan->stage[slot][2] : nullptr};
    st = zinv_pass<R>(plan, j, src[j], dv[0], dv[1], dv[2], j == 2);
    if (st != GG_OK) return st;
    if ((e = cudaEventRecord(plan->ev_comp[slot], plan->stream)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(plan->copy_stream, plan->ev_comp[slot], 0)) != cudaSuccess)
      return cuda_fail(plan, e, "event ordering");
    for (int o = 0; o < 3; ++o)
      if (hs[o] && (e = cudaMemcpyAsync(hs[o], dv[o], grid, cudaMemcpyDeviceToHost,
                                        plan->copy_stream)) != cudaSuccess)
        return cuda_fail(plan, e, "output download");
    if ((e = cudaEventRecord(plan->ev_copy[slot], plan->copy_stream)) != cudaSuccess)
      return cuda_fail(plan, e, "cudaEventRecord");
    used[slot] = true;
    slot ^= 1;
  }
  if ((e = cudaStreamSynchronize(plan->copy_stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(plan->stream)) != cudaSuccess)
    return cuda_fail(plan, e, "synchronize");
  return GG_OK;
}

// Times every tile variant of the size-specialised kernels on the plan's own
// buffers and keeps the fastest per pass. All passes are switched to variant v
// together and timed one by one through the per-kernel events; the pass ->
// kind map below picks each pass's time.
template <typename R>
gg_status autotune(gg_plan_t *plan, int reps) {
  if (!gg::spec_has<R>((int)plan->p.n)) return GG_OK;
  gg_status st;
  if ((st = ensure_grid(plan, &plan->work2)) != GG_OK) return st;
  if ((st = ensure_grid(plan, &plan->work3)) != GG_OK) return st;
  void *tmp = nullptr;
  if ((st = ensure_grid(plan, &tmp)) != GG_OK) return st;
  const size_t grid = (size_t)plan->cells * sizeof(R);
  cudaMemsetAsync(plan->work, 0, grid, plan->stream);
  const int kinds[6] = {kZFwd, kYFwd, kXFused, kYInvX, kYInvYZ, kZInv};
  const int nvar[6] = {gg::kSpecZVariants,    gg::kSpecAxisVariants, gg::kSpecAxisVariants,
                       gg::kSpecAxisVariants, gg::kSpecAxisVariants, gg::kSpecZVariants};
  double best[6];
  int best_v[6];
  for (int i = 0; i < 6; ++i) {
    best[i] = 1e300;
    best_v[i] = 0;
  }
  const bool prof_was = plan->prof_on;
  plan->chunked = 0;  // the variants are timed in the plain layout
  void *vel[3] = {tmp, tmp, tmp};
  const int vmax = std::max(gg::kSpecZVariants, gg::kSpecAxisVariants);
  for (int v = 0; v < vmax; ++v) {
    for (int i = 0; i < 6; ++i) plan->variant[i] = v < nvar[i] ? v : 0;
    plan->prof_on = false;
    if ((st = run_zeldovich<R>(plan, 1, nullptr, nullptr, nullptr, vel)) != GG_OK) break;  // warm
    plan->prof_on = true;
    for (int k = 0; k < kNumKinds; ++k) {
      plan->prof_ms[k] = 0;
      plan->prof_launches[k] = 0;
    }
    plan->prof_used = 0;
    for (int r = 0; r < reps && st == GG_OK; ++r)
      st = run_zeldovich<R>(plan, 1 + r, nullptr, nullptr, nullptr, vel);
    if (st != GG_OK) break;
    int cnt = kNumKinds;
    if ((st = gg_profile_read(plan, 0, &cnt, nullptr, nullptr, nullptr, nullptr)) != GG_OK) break;
    for (int i = 0; i < 6; ++i) {
      if (v >= nvar[i]) continue;
      const double ms = plan->prof_ms[kinds[i]];
      if (ms < best[i]) {
        best[i] = ms;
        best_v[i] = v;
      }
    }
  }
  plan->prof_on = prof_was;
  for (int k = 0; k < kNumKinds; ++k) {
    plan->prof_ms[k] = 0;
    plan->prof_launches[k] = 0;
  }
  for (int i = 0; i < 6; ++i) plan->variant[i] = best_v[i];
  // the layout between the y passes: chunk-major where the chosen strided
  // variants share a tile width and the whole three-component step is faster
  plan->chunked = 0;
  if (st == GG_OK && chunk_cols<R>(plan) > 0) {
    void *pos[3] = {tmp, tmp, tmp};  // same traffic for both layouts
    double t[2] = {0, 0};
    const bool prof_keep = plan->prof_on;
    plan->prof_on = false;
    cudaEvent_t ev[2];
    cudaEventCreate(&ev[0]);
    cudaEventCreate(&ev[1]);
    for (int layout = 0; layout < 2 && st == GG_OK; ++layout) {
      plan->chunked = layout;
      if ((st = run_zeldovich<R>(plan, 1, nullptr, nullptr, pos, vel)) != GG_OK) break;  // warm
      cudaEventRecord(ev[0], plan->stream);
      for (int r = 0; r < reps && st == GG_OK; ++r)
        st = run_zeldovich<R>(plan, 1 + r, nullptr, nullptr, pos, vel);
      cudaEventRecord(ev[1], plan->stream);
      float ms = 0;
      if (st == GG_OK && cudaEventSynchronize(ev[1]) == cudaSuccess &&
          cudaEventElapsedTime(&ms, ev[0], ev[1]) == cudaSuccess)
        t[layout] = ms;
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    plan->prof_on = prof_keep;
    plan->chunked = (st == GG_OK && t[1] > 0 && t[1] < t[0]) ? 1 : 0;
  }
  cudaStreamSynchronize(plan->stream);
  cudaFree(tmp);
  return st;
}

// ------------------------------------------------------------ adjoint form
// psi_j = J_j W with J_j = F^-1 diag(i m_j U) F (F the unnormalised DFT,
// U real and even in k). i m_j U is purely imaginary and Hermitian, so
// J_j^T = -J_j and dL/dW = sum_j J_j^T g_j = -sum_j J_j g_j: the forward
// chain run once per component on g_j, accumulated with weight -1. No
// transform intermediates are stored.
template <typename R>
gg_status run_adjoint(gg_plan_t *plan, const void *const g_psi[3], void *g_noise) {
  cudaError_t e = cudaMemsetAsync(g_noise, 0, (size_t)plan->cells * sizeof(R), plan->stream);
  if (e != cudaSuccess) return cuda_fail(plan, e, "cudaMemsetAsync");
  for (int j = 0; j < 3; ++j) {
    if (!g_psi || !g_psi[j]) continue;
    const bool want[3] = {j == 0, j == 1, j == 2};
    void *src[3];
    gg_status st = spectral_passes<R>(plan, 0, g_psi[j], want, nullptr, src);
    if (st != GG_OK) return st;
    st = zinv_pass<R>(plan, j, src[j], g_noise, nullptr, nullptr, j == 2, true, -1.0);
    if (st != GG_OK) return st;
  }
  return GG_OK;
}

template <typename R>
gg_status run_smooth(gg_plan_t *plan, double radius, const void *in, void *out) {
  const int64_t n = plan->p.n;
  if (radius != plan->tab.smooth_radius) {
    const size_t cnt = table_entries(n);
    std::vector<R> t(cnt);
    const double kf = 2.0 * kPi / plan->p.box;
    const double n3 = (double)n * n * n;
    for (size_t i = 0; i < cnt; ++i) t[i] = (R)(std::exp(-0.5 * kf * kf * (double)i * radius * radius) / n3);
    cudaError_t e;
    if (!plan->tab.smooth && (e = cudaMalloc(&plan->tab.smooth, cnt * sizeof(R))) != cudaSuccess)
      return fail(plan, GG_ENOMEM, "cudaMalloc of the smoothing table failed");
    if ((e = cudaMemcpy(plan->tab.smooth, t.data(), cnt * sizeof(R), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
      return cuda_fail(plan, e, "smoothing table upload");
    plan->tab.smooth_radius = radius;
    if (sizeof(R) == 4) {
      auto g_of = [&](double mm, int) { return std::exp(-0.5 * kf * kf * mm * mm * radius * radius) / n3; };
      if (plan->tab.interp_smooth) {
        cudaFree(plan->tab.interp_smooth);
        plan->tab.interp_smooth = nullptr;
      }
      gg_status st = upload_interp(plan, &plan->tab.interp_smooth, g_of);
      if (st != GG_OK) return st;
    }
  }
  return run_density<R>(plan, 0, in, out, plan->tab.smooth, plan->tab.interp_smooth);
}

// Sec. 2.4, Eq. 5 with the cloud-in-cell deconvolution: out = F^-1[f(|k| r_s)
// F[in] / W_CIC]. Forward z, y and x passes, the spectrum multiplied by the
// top hat and 1 / prod_j sinc^2(pi m_j / N) (and 1 / N^3), inverse x, y, z.
int64_t top_hat_qmax(double box, double r_s) {
  // |k| r_s < 1  <=>  m2 < X = (L / (2 pi r_s))^2  <=>  m2 < ceil(X) (integer m2)
  const double x = box / (2.0 * kPi * r_s);
  return (int64_t)std::ceil(x * x);
}

template <typename R>
gg_status run_large_scales(gg_plan_t *plan, double r_s, const void *in, void *out) {
  const int n = (int)plan->p.n;
  if (!plan->tab.cic_deconv) {
    std::vector<R> d(n);
    for (int i = 0; i < n; ++i) {
      const int m = i < n / 2 ? i : i - n;
      const double x = kPi * m / n;
      const double sinc = m == 0 ? 1.0 : std::sin(x) / x;
      d[i] = i == n / 2 ? (R)0 : (R)(1.0 / (sinc * sinc));
    }
    gg_status st = upload(plan, &plan->tab.cic_deconv, d);
    if (st != GG_OK) return st;
  }
  gg_status st = forward_zy<R>(plan, 0, in);
  if (st != GG_OK) return st;
  gg::AxisArgs x = axis_args<R>(plan, 0, plan->work);
  x.fwd = 1;
  x.inv = 0;
  x.nout = 1;
  x.dst[0] = plan->work;
  x.mul[0] = gg::kMulNone;
  x.variant = plan->variant[1];
  if ((st = launch_axis_timed<R>(plan, x, kXFused, "x forward pass")) != GG_OK) return st;
  gg::SpecScaleArgs sc{};
  sc.spec = plan->work;
  sc.n = n;
  sc.qmax = top_hat_qmax(plan->p.box, r_s);
  sc.axis_factor = plan->tab.cic_deconv;
  sc.scale = 1.0 / ((double)n * n * n);
  cudaError_t e = gg::launch_spectrum_scale<R>(sc, plan->stream);
  if (e != cudaSuccess) return cuda_fail(plan, e, "spectrum scale");
  x.fwd = 0;
  x.inv = 1;
  x.variant = plan->variant[3];
  if ((st = launch_axis_timed<R>(plan, x, kYInvX, "x inverse pass")) != GG_OK) return st;
  gg::AxisArgs y = axis_args<R>(plan, 1, plan->work);
  y.inv = 1;
  y.nout = 1;
  y.dst[0] = plan->work;
  y.mul[0] = gg::kMulNone;
  y.variant = plan->variant[3];
  if ((st = launch_axis_timed<R>(plan, y, kYInvX, "y inverse pass")) != GG_OK) return st;
  return zinv_pass<R>(plan, 0, plan->work, out, nullptr, nullptr, false);
}

template <typename R>
gg_status run_power_spectrum(gg_plan_t *plan, const void *field, int nbins, double *k_out,
                             double *p_out, int64_t *count_out) {
  const int n = (int)plan->p.n;
  gg_status st = forward_zy<R>(plan, 0, field);
  if (st != GG_OK) return st;
  gg::AxisArgs x = axis_args<R>(plan, 0, plan->work);
  x.fwd = 1;
  x.inv = 0;
  x.nout = 1;
  x.dst[0] = plan->work;
  x.mul[0] = gg::kMulNone;
  x.variant = plan->variant[1];
  if ((st = launch_axis_timed<R>(plan, x, kXFused, "x forward pass")) != GG_OK) return st;
  double *sums = nullptr;
  cudaError_t e = cudaMallocAsync((void **)&sums, sizeof(double) * 2 * nbins, plan->stream);
  if (e != cudaSuccess) return cuda_fail(plan, e, "cudaMallocAsync of the shell sums");
  gg::ShellArgs a{};
  a.spec = plan->work;
  a.n = n;
  a.nbins = nbins;
  a.sums = sums;
  auto pass = [&](bool geometry, std::vector<double> &h) {
    h.assign((geometry ? 2 : 1) * (size_t)nbins, 0.0);
    cudaError_t ee;
    if ((ee = cudaMemsetAsync(sums, 0, sizeof(double) * h.size(), plan->stream)) != cudaSuccess ||
        (ee = gg::launch_shell_sums<R>(a, geometry, plan->stream)) != cudaSuccess ||
        (ee = cudaMemcpyAsync(h.data(), sums, sizeof(double) * h.size(), cudaMemcpyDeviceToHost,
                              plan->stream)) != cudaSuccess)
      return ee;
    return cudaStreamSynchronize(plan->stream);
  };
  std::vector<double> geo, pw;
  if (plan->shell_nb != nbins) {  // the grid's own sums, once per shell count
    if ((e = pass(true, geo)) == cudaSuccess) {
      plan->shell_w.assign(geo.begin(), geo.begin() + nbins);
      plan->shell_m.assign(geo.begin() + nbins, geo.end());
      plan->shell_nb = nbins;
    }
  }
  if (e == cudaSuccess) e = pass(false, pw);
  const cudaError_t ef = cudaFreeAsync(sums, plan->stream);
  if (e != cudaSuccess) return cuda_fail(plan, e, "power spectrum shell sums");
  if (ef != cudaSuccess) return cuda_fail(plan, ef, "power spectrum shell sums");
  const double box = plan->p.box, vol = box * box * box, n6 = std::pow((double)n, 6.0);
  for (int b = 0; b < nbins; ++b) {
    const double c = plan->shell_w[b];
    if (count_out) count_out[b] = (int64_t)(c + 0.5);
    if (p_out) p_out[b] = c > 0 ? vol / n6 * pw[b] / c : 0.0;
    if (k_out) k_out[b] = c > 0 ? 2.0 * kPi / box * plan->shell_m[b] / c : 0.0;
  }
  return GG_OK;
}

template <typename R>
gg_status run_moments(gg_plan_t *plan, const void *field, double out[4]) {
  const int64_t count = plan->cells;
  const int blocks = gg::moment_blocks<R>(count);
  double *slots = nullptr;
  cudaError_t e = cudaMallocAsync((void **)&slots, sizeof(double) * 3 * blocks, plan->stream);
  if (e != cudaSuccess) return cuda_fail(plan, e, "cudaMallocAsync of the moment slots");
  std::vector<double> h(3 * (size_t)blocks);
  double mean = 0.0, var = 0.0, lo = 0.0, hi = 0.0;
  for (int pass = 0; pass < 2; ++pass) {
    gg::MomentArgs a{};
    a.field = field;
    a.count = count;
    a.second = pass;
    a.mean = mean;
    a.slots = slots;
    if ((e = gg::launch_moments<R>(a, blocks, plan->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(h.data(), slots, sizeof(double) * 3 * blocks, cudaMemcpyDeviceToHost,
                             plan->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(plan->stream)) != cudaSuccess)
      break;
    double s = 0.0;
    for (int b = 0; b < blocks; ++b) s += h[3 * b];
    if (pass == 0) {
      mean = s / (double)count;
      lo = h[1];
      hi = h[2];
      for (int b = 1; b < blocks; ++b) {
        lo = std::min(lo, h[3 * b + 1]);
        hi = std::max(hi, h[3 * b + 2]);
      }
    } else {
      var = s / (double)count;
    }
  }
  const cudaError_t ef = cudaFreeAsync(slots, plan->stream);
  if (e != cudaSuccess) return cuda_fail(plan, e, "field moments");
  if (ef != cudaSuccess) return cuda_fail(plan, ef, "field moments");
  out[0] = mean;
  out[1] = var;
  out[2] = lo;
  out[3] = hi;
  return GG_OK;
}

// Sec. 2.4 degrading: every r-th fine value (nearest grid point) into out,
// then moved by t = (r - 1) / (2 r) cells onto the coarse cell centres:
// forward passes, the spectrum times exp(2 pi i t m_j / N) per axis (and
// 1 / N^3), inverse passes.
template <typename R>
gg_status run_degrade(gg_plan_t *plan, int64_t n_high, const void *high, void *out) {
  const int n = (int)plan->p.n;
  const int r = (int)(n_high / n);
  if (plan->phase_r != r) {
    std::vector<R> ph(2 * (size_t)n);
    const double t = (double)(r - 1) / (2.0 * r);
    for (int i = 0; i < n; ++i) {
      const int m = i < n / 2 ? i : i - n;
      const double a = 2.0 * kPi * t * m / n;
      ph[2 * i] = i == n / 2 ? (R)0 : (R)std::cos(a);
      ph[2 * i + 1] = i == n / 2 ? (R)0 : (R)std::sin(a);
    }
    if (plan->phase) {
      cudaFree(plan->phase);
      plan->phase = nullptr;
    }
    gg_status st = upload(plan, &plan->phase, ph);
    if (st != GG_OK) return st;
    plan->phase_r = r;
  }
  cudaError_t e = gg::launch_subsample<R>(high, n_high, r, out, plan->stream);
  if (e != cudaSuccess) return cuda_fail(plan, e, "subsample");
  gg_status st = forward_zy<R>(plan, 0, out);
  if (st != GG_OK) return st;
  gg::AxisArgs x = axis_args<R>(plan, 0, plan->work);
  x.fwd = 1;
  x.inv = 0;
  x.nout = 1;
  x.dst[0] = plan->work;
  x.mul[0] = gg::kMulNone;
  x.variant = plan->variant[1];
  if ((st = launch_axis_timed<R>(plan, x, kXFused, "x forward pass")) != GG_OK) return st;
  gg::SpecPhaseArgs ph{};
  ph.spec = plan->work;
  ph.n = n;
  ph.phase = plan->phase;
  ph.scale = 1.0 / ((double)n * n * n);
  if ((e = gg::launch_spectrum_phase<R>(ph, plan->stream)) != cudaSuccess)
    return cuda_fail(plan, e, "spectrum phase");
  x.fwd = 0;
  x.inv = 1;
  x.variant = plan->variant[3];
  if ((st = launch_axis_timed<R>(plan, x, kYInvX, "x inverse pass")) != GG_OK) return st;
  gg::AxisArgs y = axis_args<R>(plan, 1, plan->work);
  y.inv = 1;
  y.nout = 1;
  y.dst[0] = plan->work;
  y.mul[0] = gg::kMulNone;
  y.variant = plan->variant[3];
  if ((st = launch_axis_timed<R>(plan, y, kYInvX, "y inverse pass")) != GG_OK) return st;
  return zinv_pass<R>(plan, 0, plan->work, out, nullptr, nullptr, false);
}

gg::CicArgs cic_args(const gg_plan_t *plan, const void *const psi[3]) {
  gg::CicArgs a{};
  for (int j = 0; j < 3; ++j) a.psi[j] = psi[j];
  a.n = (int)plan->p.n;
  a.cell = plan->p.box / (double)plan->p.n;
  a.q_offset = (plan->p.flags & GG_Q_CORNER) ? 0.0 : 0.5;
  return a;
}

// ------------------------------------------------------------ batched form
bool same_params(const gg_params &a, const gg_params &b) {
  auto eq = [](double x, double y) { return x == y || (std::isnan(x) && std::isnan(y)); };
  const gg_cosmo &c = a.cosmo, &d = b.cosmo;
  return a.n == b.n && eq(a.box, b.box) && a.prec == b.prec && a.flags == b.flags &&
         eq(a.z_init, b.z_init) && eq(a.growth_override[0], b.growth_override[0]) &&
         eq(a.growth_override[1], b.growth_override[1]) && eq(c.omega_m, d.omega_m) &&
         eq(c.omega_l, d.omega_l) && eq(c.omega_b, d.omega_b) && eq(c.h, d.h) && eq(c.n_s, d.n_s) &&
         eq(c.sigma_8, d.sigma_8) && eq(c.t_cmb, d.t_cmb) && c.tf == d.tf && c.tab_k == d.tab_k &&
         c.tab_p == d.tab_p && c.tab_n == d.tab_n;
}

// All passes of one group, on stream s, every launch covering all nb
// realizations (captured into the batch's graph).
// Arguments of the batched passes of one group (every realization of the
// group in each launch): z forward, y forward, x fused, the two y inverse
// passes, and the z inverse passes of the components some realization wants.
template <typename R>
void group_args(gg_batch::Group &g, uint32_t sig, gg::ZFwdArgs &z, gg::AxisArgs ax[4],
                gg::ZInvArgs zi[3], bool on[3]) {
  gg_plan_t *plan = g.plan;
  const int n = (int)plan->p.n, half = n / 2;
  const int nb = (int)g.members.size();
  const int64_t grid_c = (int64_t)n * n * half;  // complex values per realization
  z = gg::ZFwdArgs{};
  z.out = g.work[0];
  z.nlines = (int64_t)nb * n * n;
  z.lines_per_real = (int64_t)n * n;
  z.seeds = g.d_seeds;
  z.n = n;
  z.lines_per_cta = plan->z_lines;
  z.st = plan->st_half;
  z.tw_half = plan->tab.tw_half;
  z.tw_full = plan->tab.tw_n;
  z.variant = plan->variant[0];
  auto axb = [&](const void *src) {
    gg::AxisArgs c = axis_args<R>(plan, 1, src);
    c.nbatch = nb;
    c.batch_stride = grid_c;
    return c;
  };
  gg::AxisArgs &y = ax[0];
  y = axb(g.work[0]);
  y.fwd = 1;
  y.nout = 1;
  y.dst[0] = g.work[0];
  y.variant = plan->variant[1];
  gg::AxisArgs &x = ax[1];
  x = axb(g.work[0]);
  x.axis = 0;
  x.stride = (int64_t)n * half;
  x.outer_stride = half;
  x.fwd = 1;
  x.inv = 1;
  x.pre = 1;
  x.table = plan->tab.u_phi;
  x.interp = plan->tab.interp_u;
  x.interp_cells = plan->tab.interp_cells;
  x.nout = 2;
  x.dst[0] = g.work[0];
  x.mul[0] = gg::kMulIm;
  x.dst[1] = g.work[1];
  x.mul[1] = gg::kMulNone;
  x.variant = plan->variant[2];
  gg::AxisArgs &ya = ax[2];
  ya = axb(g.work[0]);
  ya.inv = 1;
  ya.nout = 1;
  ya.dst[0] = g.work[0];
  ya.variant = plan->variant[3];
  gg::AxisArgs &yb = ax[3];
  yb = axb(g.work[1]);
  yb.inv = 1;
  yb.nout = 2;
  yb.dst[0] = g.work[1];
  yb.mul[0] = gg::kMulIm;
  yb.dst[1] = g.work[2];
  yb.mul[1] = gg::kMulNone;
  yb.variant = plan->variant[4];
  for (int j = 0; j < 3; ++j) {
    on[j] = (sig >> j) & 0x49;  // psi_j, pos_j or vel_j wanted anywhere
    gg::ZInvArgs &zj = zi[j];
    zj = gg::ZInvArgs{};
    zj.src = g.work[j];
    zj.nlines = (int64_t)nb * n * n;
    zj.lines_per_real = (int64_t)n * n;
    zj.psi_list = ((sig >> (0 * 3 + j)) & 1) ? g.d_lists + (0 * 3 + j) * nb : nullptr;
    zj.pos_list = ((sig >> (1 * 3 + j)) & 1) ? g.d_lists + (1 * 3 + j) * nb : nullptr;
    zj.vel_list = ((sig >> (2 * 3 + j)) & 1) ? g.d_lists + (2 * 3 + j) * nb : nullptr;
    zj.lists_full = ((sig >> (9 + 1 * 3 + j)) & 1) && ((sig >> (9 + 2 * 3 + j)) & 1);
    zj.n = n;
    zj.lines_per_cta = plan->z_lines;
    zj.comp = j;
    zj.mul_kz = j == 2;
    zj.box = plan->p.box;
    zj.cell = plan->p.box / (double)n;
    zj.q_offset = (plan->p.flags & GG_Q_CORNER) ? 0.0 : 0.5;
    zj.vfac = plan->info.vfac;
    zj.st = plan->st_half;
    zj.tw_half = plan->tab.tw_half;
    zj.tw_full = plan->tab.tw_n;
    zj.err = plan->err;
    zj.variant = plan->variant[5];
  }
}

// The group's seeds and output lists, staged in pinned memory, to the device.
cudaError_t group_staging(gg_batch::Group &g, cudaStream_t s) {
  const int nb = (int)g.members.size();
  cudaError_t e = cudaMemcpyAsync(g.d_seeds, g.h_seeds, sizeof(uint64_t) * nb, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g.d_lists, g.h_lists, sizeof(void *) * 9 * nb, cudaMemcpyHostToDevice, s);
  return e;
}

template <typename R>
gg_status group_passes(gg_batch::Group &g, cudaStream_t s, uint32_t sig) {
  gg_plan_t *plan = g.plan;
  const cudaStream_t saved = plan->stream;
  plan->stream = s;
  const int n = (int)plan->p.n;
  gg_status st = GG_OK;
  cudaError_t e;
  if ((e = group_staging(g, s)) != cudaSuccess) {
    plan->stream = saved;
    return cuda_fail(nullptr, e, "batch staging copies");
  }
  gg::ZFwdArgs z;
  gg::AxisArgs ax[4];
  gg::ZInvArgs zi[3];
  bool on[3];
  group_args<R>(g, sig, z, ax, zi, on);
  const int kinds[4] = {kYFwd, kXFused, kYInvX, kYInvYZ};
  const char *const what[4] = {"batched y forward", "batched x fused", "batched y inverse (x)",
                               "batched y inverse (y/z)"};
  do {
    e = gg::spec_has<R>(n) ? gg::spec_zfwd<R>(z, s) : gg::launch_zfwd<R>(z, s);
    if (e != cudaSuccess) { st = cuda_fail(nullptr, e, "batched z forward"); break; }
    for (int k = 0; k < 4 && st == GG_OK; ++k) st = launch_axis_timed<R>(plan, ax[k], kinds[k], what[k]);
    for (int j = 0; j < 3 && st == GG_OK; ++j) {
      if (!on[j]) continue;
      e = gg::spec_has<R>(n) ? gg::spec_zinv<R>(zi[j], s) : gg::launch_zinv<R>(zi[j], s);
      if (e != cudaSuccess) st = cuda_fail(nullptr, e, "batched z inverse");
    }
  } while (false);
  plan->stream = saved;
  return st;
}

// The whole batch as one persistent launch (gg_persist.cu): staging copies
// of every group, the pass counters cleared, then the kernel.
gg_status persist_passes(gg_batch_t *b, cudaStream_t s, uint32_t sig) {
  gg::PersistPlan pp{};
  pp.ngroups = (int)b->groups.size();
  pp.realizations = b->count;
  pp.counters = b->counters;
  pp.err = b->groups[0].plan->err;
  pp.chunk = b->persist_chunk;
  pp.test_stall = b->test_stall;
  pp.wait_us = b->test_stall ? b->test_wait_us : 0;
  cudaError_t e;
  int first = 0;
  for (int gi = 0; gi < pp.ngroups; ++gi) {
    gg_batch::Group &g = b->groups[gi];
    if ((e = group_staging(g, s)) != cudaSuccess) return cuda_fail(nullptr, e, "batch staging copies");
    gg::PersistGroupArgs &pg = pp.g[gi];
    bool on[3];
    group_args<float>(g, sig, pg.zf, pg.ax, pg.zi, on);
    pg.n = (int)g.plan->p.n;
    pg.nb = (int)g.members.size();
    pg.first = first;
    first += pg.nb;
    for (int j = 0; j < 3; ++j) pg.zi_on[j] = on[j] ? 1 : 0;
    // the pos + vel instantiation when every realization wants both, no psi
    const bool lists_full = (((sig >> 9) >> 3) & 7) == 7 && (((sig >> 9) >> 6) & 7) == 7;
    pg.plain = lists_full && (sig & 7) == 0 ? 1 : 0;
    for (int j = 0; j < 3; ++j) pg.zi[j].err = pp.err;
    for (auto &a : pg.ax) a.err = pp.err;
  }
  const size_t words = 64 + (size_t)8 * b->count;
  if ((e = cudaMemsetAsync(b->counters, 0, words * sizeof(unsigned), s)) != cudaSuccess)
    return cuda_fail(nullptr, e, "clearing the pass counters");
  if ((e = gg::launch_persist(pp, s, &b->persist_blocks)) != cudaSuccess)
    return cuda_fail(nullptr, e, "persistent batched launch");
  return GG_OK;
}

void batch_release(gg_batch_t *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto &g : b->groups) {
    for (void *w : g.work)
      if (w) cudaFree(w);
    if (g.d_seeds) cudaFree(g.d_seeds);
    if (g.d_lists) cudaFree(g.d_lists);
    if (g.h_seeds) cudaFreeHost(g.h_seeds);
    if (g.h_lists) cudaFreeHost(g.h_lists);
    if (g.ev) cudaEventDestroy(g.ev);
    if (g.s) cudaStreamDestroy(g.s);
    if (g.plan) gg_free(g.plan);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->done) cudaEventDestroy(b->done);
  if (b->counters) cudaFree(b->counters);
}

}  // namespace

namespace gg {

template <typename R>
int z_lines_per_cta(const FftStages &st_half) {
  const int half = st_half.len, P = half / st_half.e;
  const size_t cb = 2 * sizeof(R), smem_cap = 110 * 1024;
  int cap = std::min(max_block_threads_z<R>(0, st_half.e), max_block_threads_z<R>(2, st_half.e));
  if (cap <= 0) cap = 256;
  int lines = std::max(1, 256 / P);
  while (lines > 1 && (P * lines > cap || zpass_smem_bytes(half, lines, cb) > smem_cap)) lines /= 2;
  return lines;
}
template int z_lines_per_cta<float>(const FftStages &);
template int z_lines_per_cta<double>(const FftStages &);

bool info_and_filter(const gg_params *p, gg_info *info, double *s, int64_t count, const char **msg) {
  thread_local std::string why;
  why = validate(p);
  if (!why.empty()) {
    if (msg) *msg = why.c_str();
    return false;
  }
  const cosmo::Model m = make_model(p);
  std::memset(info, 0, sizeof(*info));
  fill_info(p, m, info);
  info->workspace_bytes = (int64_t)workspace_bytes(p);
  filter_values(p, m, info->growth, s, count);
  return true;
}

bool make_stages(int len, FftStages *st) {
  std::memset(st, 0, sizeof(*st));
  if (len < 1) return false;
  int a = 0, b = 0, x = len;
  while (x % 2 == 0) { x /= 2; ++a; }
  while (x % 3 == 0) { x /= 3; ++b; }
  if (x != 1) return false;
  std::vector<int> rad;
  for (int i = 0; i < a / 3; ++i) rad.push_back(8);
  if (a % 3 == 2) rad.push_back(4);
  if (a % 3 == 1) rad.push_back(2);
  for (int i = 0; i < b; ++i) rad.push_back(3);
  if ((int)rad.size() > kMaxStages) return false;
  int pow2 = a >= 3 ? 8 : (a == 2 ? 4 : (a == 1 ? 2 : 1));
  st->e = pow2 * (b > 0 ? 3 : 1);
  if (len == 1) st->e = 1;
  st->len = len;
  st->nstages = (int)rad.size();
  int ns = 1;
  for (int s = 0; s < st->nstages; ++s) {
    st->radix[s] = rad[s];
    st->ns[s] = ns;
    st->ns_shift[s] = (ns & (ns - 1)) == 0 ? __builtin_ctz((unsigned)ns) : -1;
    st->tstep[s] = len / (ns * rad[s]);
    ns *= rad[s];
  }
  return true;
}

void set_thread_error(const char *msg) { g_thread_error = msg ? msg : ""; }

FftStages reversed_stages(const FftStages &f) {
  FftStages st;
  std::memset(&st, 0, sizeof(st));
  st.len = f.len;
  st.e = f.e;
  st.nstages = f.nstages;
  int ns = 1;
  for (int s = 0; s < f.nstages; ++s) {
    const int rad = f.radix[f.nstages - 1 - s];
    st.radix[s] = rad;
    st.ns[s] = ns;
    st.ns_shift[s] = (ns & (ns - 1)) == 0 ? __builtin_ctz((unsigned)ns) : -1;
    st.tstep[s] = f.len / (ns * rad);
    ns *= rad;
  }
  return st;
}

}  // namespace gg

// ---------------------------------------------------------------------- C ABI
extern "C" {

int gg_version(void) { return 100; }

gg_status gg_cosmo_eval(const gg_params *p, gg_info *out) {
  const std::string msg = validate(p);
  if (!msg.empty()) return fail(nullptr, GG_EINVAL, msg);
  if (!out) return fail(nullptr, GG_EINVAL, "out is NULL");
  std::memset(out, 0, sizeof(*out));
  const gg::cosmo::Model m = make_model(p);
  fill_info(p, m, out);
  out->workspace_bytes = (int64_t)workspace_bytes(p);
  return GG_OK;
}

gg_status gg_power(const gg_params *p, const double *k, double *pk, int64_t count) {
  const std::string msg = validate(p);
  if (!msg.empty()) return fail(nullptr, GG_EINVAL, msg);
  if (count < 0 || (count > 0 && (!k || !pk))) return fail(nullptr, GG_EINVAL, "bad arrays");
  const gg::cosmo::Model m = make_model(p);
  for (int64_t i = 0; i < count; ++i) pk[i] = m.power(k[i]);
  return GG_OK;
}

gg_status gg_filter_table(const gg_params *p, double *s, int64_t count) {
  const std::string msg = validate(p);
  if (!msg.empty()) return fail(nullptr, GG_EINVAL, msg);
  if (count < 0 || (count > 0 && !s)) return fail(nullptr, GG_EINVAL, "bad array");
  const gg::cosmo::Model m = make_model(p);
  gg_info info{};
  fill_info(p, m, &info);
  filter_values(p, m, info.growth, s, count);
  return GG_OK;
}

gg_status gg_workspace_size(const gg_params *p, size_t *bytes) {
  const std::string msg = validate(p);
  if (!msg.empty()) return fail(nullptr, GG_EINVAL, msg);
  if (!bytes) return fail(nullptr, GG_EINVAL, "bytes is NULL");
  *bytes = workspace_bytes(p);
  return GG_OK;
}

gg_status gg_plan(gg_plan_t **plan, const gg_params *p, void *stream) {
  if (!plan) return fail(nullptr, GG_EINVAL, "plan is NULL");
  *plan = nullptr;
  const std::string msg = validate(p);
  if (!msg.empty()) return fail(nullptr, GG_EINVAL, msg);
  gg_plan_t *pl = new (std::nothrow) gg_plan_t();
  if (!pl) return fail(nullptr, GG_ENOMEM, "host allocation failed");
  pl->p = *p;
  pl->p.cosmo.tab_k = pl->p.cosmo.tab_p = nullptr;  // not retained past the call
  pl->stream = (cudaStream_t)stream;
  pl->cells = p->n * p->n * p->n;
  cudaError_t e = cudaGetDevice(&pl->device);
  if (e != cudaSuccess) {
    delete pl;
    return cuda_fail(nullptr, e, "cudaGetDevice");
  }
  const gg::cosmo::Model m = make_model(p);
  fill_info(p, m, &pl->info);
  const gg_status st = p->prec == GG_F64 ? create<double>(pl, m) : create<float>(pl, m);
  if (st != GG_OK) {
    g_thread_error = pl->last_error;
    release(pl);
    delete pl;
    return st;
  }
  *plan = pl;
  return GG_OK;
}

gg_status gg_set_stream(gg_plan_t *plan, void *stream) {
  if (!plan) return fail(nullptr, GG_EINVAL, "plan is NULL");
  plan->stream = (cudaStream_t)stream;
  return GG_OK;
}

gg_status gg_plan_info(const gg_plan_t *plan, gg_info *out) {
  if (!plan || !out) return fail(nullptr, GG_EINVAL, "plan or out is NULL");
  *out = plan->info;
  return GG_OK;
}

gg_status gg_white_noise(gg_plan_t *plan, uint64_t seed, void *noise_dev) {
  if (!plan) return fail(nullptr, GG_EINVAL, "plan is NULL");
  if (!noise_dev || !aligned16(noise_dev)) return fail(plan, GG_EINVAL, "noise_dev NULL or unaligned");
  gg::NoiseArgs a{noise_dev, seed, plan->cells};
  cudaError_t e;
  {
    ProfScope ps(plan, kNoise, (double)plan->cells * plan->real_bytes);
    e = plan->real_bytes == 8 ? gg::launch_noise<double>(a, plan->stream)
                              : gg::launch_noise<float>(a, plan->stream);
  }
  return e == cudaSuccess ? GG_OK : cuda_fail(plan, e, "noise kernel");
}

gg_status gg_noise_bits(uint64_t seed, int64_t first_group, int64_t count, uint32_t *out_dev,
                        void *stream) {
  if (count < 0 || first_group < 0 || (count > 0 && (!out_dev || !aligned16(out_dev))))
    return fail(nullptr, GG_EINVAL, "bad arguments");
  const cudaError_t e = gg::launch_noise_bits(seed, first_group, count, out_dev, (cudaStream_t)stream);
  return e == cudaSuccess ? GG_OK : cuda_fail(nullptr, e, "noise bits kernel");
}

gg_status gg_gaussian_field(gg_plan_t *plan, uint64_t seed, const void *noise_dev, void *delta_dev) {
  if (!plan) return fail(nullptr, GG_EINVAL, "plan is NULL");
  if (!delta_dev || !aligned16(delta_dev) || (noise_dev && !aligned16(noise_dev)))
    return fail(plan, GG_EINVAL, "delta_dev NULL or a buffer unaligned");
  return plan->real_bytes == 8 ? run_density<double>(plan, seed, noise_dev, delta_dev)
                               : run_density<float>(plan, seed, noise_dev, delta_dev);
}

gg_status gg_zeldovich(gg_plan_t *plan, uint64_t seed, const void *noise_dev,
                       void *const psi_dev[3], void *const pos_dev[3], void *const vel_dev[3]) {
  if (!plan) return fail(nullptr, GG_EINVAL, "plan is NULL");
  if (noise_dev && !aligned16(noise_dev)) return fail(plan, GG_EINVAL, "noise_dev unaligned");
  for (int j = 0; j < 3; ++j) {
    const void *bufs[3] = {psi_dev ? psi_dev[j] : nullptr, pos_dev ? pos_dev[j] : nullptr,
                           vel_dev ? vel_dev[j] : nullptr};
    for (const void *b : bufs)
      if (b && !aligned16(b)) return fail(plan, GG_EINVAL, "output buffer unaligned");
  }
  return plan->real_bytes == 8 ? run_zeldovich<double>(plan, seed, noise_dev, psi_dev, pos_dev, vel_dev)
                               : run_zeldovich<float>(plan, seed, noise_dev, psi_dev, pos_dev, vel_dev);
}

gg_status gg_power_spectrum(gg_plan_t *plan, const void *field_dev, int nbins, double *k_out,
                            double *p_out, int64_t *count_out) {
  if (!plan) return fail(nullptr, GG_EINVAL, "plan is NULL");
  if (!field_dev || !aligned16(field_dev)) return fail(plan, GG_EINVAL, "field_dev NULL or unaligned");
  if (nbins < 1 || nbins > plan->p.n / 2) return fail(plan, GG_EINVAL, "nbins must be in [1, N/2]");
  return plan->real_bytes == 8 ? run_power_spectrum<double>(plan, field_dev, nbins, k_out, p_out, count_out)
                               : run_power_spectrum<float>(plan, field_dev, nbins, k_out, p_out, count_out);
}

gg_status gg_field_moments(gg_plan_t *plan, const void *field_dev, double out[4]) {
  if (!plan) return fail(nullptr, GG_EINVAL, "plan is NULL");
  if (!field_dev || !out) return fail(plan, GG_EINVAL, "field_dev and out are required");
  return plan->real_bytes == 8 ? run_moments<double>(plan, field_dev, out)
                               : run_moments<float>(plan, field_dev, out);
}

gg_status gg_set_shift(gg_plan_t *plan, const double shift[3]) {
  if (!plan || !shift) return fail(plan, GG_EINVAL, "plan and shift are required");
  for (int j = 0; j < 3; ++j)
    if (!std::isfinite(shift[j])) return fail(plan, GG_EINVAL, "shift must be finite");
  for (int j = 0; j < 3; ++j) {  // reduced into [0, L): positions are periodic
    double v = std::fmod(shift[j], plan->p.box);
    plan->shift[j] = v < 0 ? v + plan->p.box : v;
  }
  return GG_OK;
}

gg_status gg_zeldovich_gas(gg_plan_t *plan, uint64_t seed, const void *noise_dev, double gas_fraction,
                           void *const psi_dev[3], void *const pos_dm_dev[3],
                           void *const pos_gas_dev[3], void *const vel_dev[3]) {
  if (!plan) return fail(nullptr, GG_EINVAL, "plan is NULL");
  if (!(gas_fraction >= 0.0 && gas_fraction < 1.0))
    return fail(plan, GG_EINVAL, "gas_fraction must be in [0, 1)");
  if (!pos_dm_dev || !pos_gas_dev) return fail(plan, GG_EINVAL, "pos_dm_dev and pos_gas_dev are required");
  if (noise_dev && !aligned16(noise_dev)) return fail(plan, GG_EINVAL, "noise_dev unaligned");
  for (int j = 0; j < 3; ++j) {
    if (!pos_dm_dev[j] != !pos_gas_dev[j])
      return fail(plan, GG_EINVAL, "pos_dm_dev[j] and pos_gas_dev[j] must be given together");
    const void *bufs[4] = {psi_dev ? psi_dev[j] : nullptr, pos_dm_dev[j], pos_gas_dev[j],
                           vel_dev ? vel_dev[j] : nullptr};
    for (const void *b : bufs)
      if (b && !aligned16(b)) return fail(plan, GG_EINVAL, "buffer unaligned");
  }
  plan->gas_fraction = gas_fraction;
  for (int j = 0; j < 3; ++j) plan->gas_pos[j] = pos_gas_dev[j];
  const gg_status st =
      plan->real_bytes == 8 ? run_zeldovich<double>(plan, seed, noise_dev, psi_dev, pos_dm_dev, vel_dev)
                            : run_zeldovich<float>(plan, seed, noise_dev, psi_dev, pos_dm_dev, vel_dev);
  plan->gas_fraction = 0.0;
  for (int j = 0; j < 3; ++j) plan->gas_pos[j] = nullptr;
  return st;
}

gg_status gg_particle_ids(gg_plan_t *plan, int64_t n_finest, int64_t offset, int64_t *ids_dev) {
  if (!plan) return fail(nullptr, GG_EINVAL, "plan is NULL");
  const int64_t n = plan->p.n;
  if (n_finest < n || n_finest % n || n_finest > ((int64_t)1 << 20))
    return fail(plan, GG_EINVAL, "n_finest must be a multiple of N (<= 2^20)");
  if (offset < 0 || offset > INT64_MAX - n_finest * n_finest * n_finest)
    return fail(plan, GG_EINVAL, "offset out of range");
  if (!ids_dev || !aligned16(ids_dev)) return fail(plan, GG_EINVAL, "ids_dev NULL or unaligned");
  const cudaError_t e = gg::launch_particle_ids(n, n_finest, offset, ids_dev, plan->stream);
  return e == cudaSuccess ? GG_OK : cuda_fail(plan, e, "particle IDs");
}

gg_status gg_degrade(gg_plan_t *plan, int64_t n_high, const void *high_dev, void *low_dev) {
  if (!plan) return fail(nullptr, GG_EINVAL, "plan is NULL");
  if (n_high < plan->p.n || n_high % plan->p.n || n_high > 8192)
    return fail(plan, GG_EINVAL, "n_high must be a multiple of N (<= 8192)");
  if (!high_dev || !low_dev || !aligned16(high_dev) || !aligned16(low_dev))
    return fail(plan, GG_EINVAL, "high_dev / low_dev NULL or unaligned");
  return plan->real_bytes == 8 ? run_degrade<double>(plan, n_high, high_dev, low_dev)
                               : run_degrade<float>(plan, n_high, high_dev, low_dev);
}

gg_status gg_large_scales(gg_plan_t *plan, double r_s, const void *in_dev, void *out_dev) {
  if (!plan) return fail(nullptr, GG_EINVAL, "plan is NULL");
  if (!(r_s > 0) || !std::isfinite(r_s)) return fail(plan, GG_EINVAL, "r_s must be > 0");
  if (!in_dev || !out_dev || !aligned16(in_dev) || !aligned16(out_dev))
    return fail(plan, GG_EINVAL, "in/out NULL or unaligned");
  return plan->real_bytes == 8 ? run_large_scales<double>(plan, r_s, in_dev, out_dev)
                               : run_large_scales<float>(plan, r_s, in_dev, out_dev);
}

gg_status gg_zeldovich_merge(gg_plan_t *plan, uint64_t seed, const void *noise_dev, double r_s,
                             int64_t n_low, const void *const large_dev[3], void *const psi_dev[3],
                             void *const pos_dev[3], void *const vel_dev[3]) {
  if (!plan) return fail(nullptr, GG_EINVAL, "plan is NULL");
  if (!(r_s > 0) || !std::isfinite(r_s)) return fail(plan, GG_EINVAL, "r_s must be > 0");
  if (n_low < 1 || n_low > plan->p.n) return fail(plan, GG_EINVAL, "n_low must be in [1, n]");
  if (noise_dev && !aligned16(noise_dev)) return fail(plan, GG_EINVAL, "noise_dev unaligned");
  for (int j = 0; j < 3; ++j) {
    const void *bufs[4] = {large_dev ? large_dev[j] : nullptr, psi_dev ? psi_dev[j] : nullptr,
                           pos_dev ? pos_dev[j] : nullptr, vel_dev ? vel_dev[j] : nullptr};
    for (const void *b : bufs)
      if (b && !aligned16(b)) return fail(plan, GG_EINVAL, "buffer unaligned");
  }
  const int64_t qmax_all = 3 * (plan->p.n / 2) * (plan->p.n / 2) + 1;
  const int64_t q = top_hat_qmax(plan->p.box, r_s);
  plan->merge_qmin = (int)(q < qmax_all ? q : qmax_all);
  plan->merge_nlow = (int)n_low;
  for (int j = 0; j < 3; ++j) plan->merge_large[j] = large_dev ? large_dev[j] : nullptr;
  const gg_status st =
      plan->real_bytes == 8 ? run_zeldovich<double>(plan, seed, noise_dev, psi_dev, pos_dev, vel_dev)
                            : run_zeldovich<float>(plan, seed, noise_dev, psi_dev, pos_dev, vel_dev);
  plan->merge_qmin = 0;
  plan->merge_nlow = 0;
  for (int j = 0; j < 3; ++j) plan->merge_large[j] = nullptr;
  return st;
}

gg_status gg_zeldovich_adjoint(gg_plan_t *plan, const void *const g_psi_dev[3], void *g_noise_dev) {
  if (!plan) return fail(nullptr, GG_EINVAL, "plan is NULL");
  if (!g_noise_dev || !aligned16(g_noise_dev)) return fail(plan, GG_EINVAL, "g_noise_dev NULL or unaligned");
  for (int j = 0; j < 3; ++j)
    if (g_psi_dev && g_psi_dev[j] && !aligned16(g_psi_dev[j]))
      return fail(plan, GG_EINVAL, "g_psi buffer unaligned");
  return plan->real_bytes == 8 ? run_adjoint<double>(plan, g_psi_dev, g_noise_dev)
                               : run_adjoint<float>(plan, g_psi_dev, g_noise_dev);
}

gg_status gg_smooth(gg_plan_t *plan, double radius, const void *in_dev, void *out_dev) {
  if (!plan) return fail(nullptr, GG_EINVAL, "plan is NULL");
  if (!(radius >= 0) || !std::isfinite(radius)) return fail(plan, GG_EINVAL, "radius must be >= 0");
  if (!in_dev || !out_dev || !aligned16(in_dev) || !aligned16(out_dev))
    return fail(plan, GG_EINVAL, "in/out NULL or unaligned");
  return plan->real_bytes == 8 ? run_smooth<double>(plan, radius, in_dev, out_dev)
                               : run_smooth<float>(plan, radius, in_dev, out_dev);
}

gg_status gg_cic_density(gg_plan_t *plan, const void *const psi_dev[3], void *delta_dev) {
  if (!plan) return fail(nullptr, GG_EINVAL, "plan is NULL");
  if (!psi_dev || !psi_dev[0] || !psi_dev[1] || !psi_dev[2] || !delta_dev)
    return fail(plan, GG_EINVAL, "psi_dev[3] and delta_dev are required");
  gg::CicArgs a = cic_args(plan, psi_dev);
  a.delta = delta_dev;
  const cudaError_t e = plan->real_bytes == 8 ? gg::launch_cic_deposit<double>(a, plan->stream)
                                              : gg::launch_cic_deposit<float>(a, plan->stream);
  return e == cudaSuccess ? GG_OK : cuda_fail(plan, e, "CIC deposit");
}

gg_status gg_cic_density_adjoint(gg_plan_t *plan, const void *const psi_dev[3], const void *g_delta_dev,
                                 void *const g_psi_dev[3]) {
  if (!plan) return fail(nullptr, GG_EINVAL, "plan is NULL");
  if (!psi_dev || !psi_dev[0] || !psi_dev[1] || !psi_dev[2] || !g_delta_dev || !g_psi_dev)
    return fail(plan, GG_EINVAL, "psi_dev[3], g_delta_dev and g_psi_dev are required");
  gg::CicArgs a = cic_args(plan, psi_dev);
  a.g_delta = g_delta_dev;
  for (int j = 0; j < 3; ++j) a.g_psi[j] = g_psi_dev[j];
  const cudaError_t e = plan->real_bytes == 8 ? gg::launch_cic_adjoint<double>(a, plan->stream)
                                              : gg::launch_cic_adjoint<float>(a, plan->stream);
  return e == cudaSuccess ? GG_OK : cuda_fail(plan, e, "CIC adjoint");
}

gg_status gg_zeldovich_host(gg_plan_t *plan, uint64_t seed, const void *noise_host,
                            void *const psi_host[3], void *const pos_host[3],
                            void *const vel_host[3]) {
  if (!plan) return fail(nullptr, GG_EINVAL, "plan is NULL");
  return plan->real_bytes == 8 ? run_host<double>(plan, seed, noise_host, psi_host, pos_host, vel_host)
                               : run_host<float>(plan, seed, noise_host, psi_host, pos_host, vel_host);
}

gg_status gg_set_profiling(gg_plan_t *plan, int enable) {
  if (!plan) return fail(nullptr, GG_EINVAL, "plan is NULL");
  plan->prof_on = enable != 0;
  return GG_OK;
}

gg_status gg_profile_read(gg_plan_t *plan, int reset, int *count, const char **names, double *ms,
                          int64_t *launches, double *bytes) {
  if (!plan || !count || *count < 0) return fail(nullptr, GG_EINVAL, "bad arguments");
  cudaError_t e = cudaStreamSynchronize(plan->stream);
  if (e != cudaSuccess) return cuda_fail(plan, e, "cudaStreamSynchronize");
  for (size_t i = 0; i < plan->prof_used; ++i) {
    float t = 0.f;
    e = cudaEventElapsedTime(&t, plan->prof[i].a, plan->prof[i].b);
    if (e != cudaSuccess) return cuda_fail(plan, e, "cudaEventElapsedTime");
    plan->prof_ms[plan->prof[i].kind] += t;
    plan->prof_launches[plan->prof[i].kind] += 1;
  }
  plan->prof_used = 0;
  int w = 0;
  for (int k = 0; k < kNumKinds && w < *count; ++k) {
    if (!plan->prof_launches[k]) continue;
    if (names) names[w] = kKindNames[k];
    if (ms) ms[w] = plan->prof_ms[k];
    if (launches) launches[w] = plan->prof_launches[k];
    if (bytes) bytes[w] = plan->prof_bytes[k];
    ++w;
  }
  *count = w;
  if (reset) {
    for (int k = 0; k < kNumKinds; ++k) {
      plan->prof_ms[k] = 0;
      plan->prof_launches[k] = 0;
    }
  }
  return GG_OK;
}

gg_status gg_autotune(gg_plan_t *plan, int reps) {
  if (!plan || reps < 1) return fail(plan, GG_EINVAL, "plan NULL or reps < 1");
  return plan->real_bytes == 8 ? autotune<double>(plan, reps) : autotune<float>(plan, reps);
}

gg_status gg_plan_variants(const gg_plan_t *plan, int32_t out[6]) {
  if (!plan || !out) return fail(nullptr, GG_EINVAL, "plan or out is NULL");
  for (int i = 0; i < 6; ++i) out[i] = plan->variant[i];
  return GG_OK;
}

gg_status gg_plan_set_variants(gg_plan_t *plan, const int32_t v[6]) {
  if (!plan || !v) return fail(plan, GG_EINVAL, "plan or v is NULL");
  for (int i = 0; i < 6; ++i) {  // passes 0 and 5 are z passes
    const int nv = (i == 0 || i == 5) ? gg::kSpecZVariants : gg::kSpecAxisVariants;
    if (v[i] < 0 || v[i] >= nv) return fail(plan, GG_EINVAL, "variant out of range");
  }
  for (int i = 0; i < 6; ++i) plan->variant[i] = v[i];
  return GG_OK;
}

gg_status gg_plan_set_layout(gg_plan_t *plan, int32_t chunked) {
  if (!plan || (chunked != 0 && chunked != 1)) return fail(plan, GG_EINVAL, "plan NULL or layout not 0/1");
  plan->chunked = chunked;
  return GG_OK;
}

gg_status gg_plan_layout(const gg_plan_t *plan, int32_t *out) {
  if (!plan || !out) return fail(nullptr, GG_EINVAL, "plan or out is NULL");
  *out = plan->chunked && (plan->real_bytes == 8 ? chunk_cols<double>(const_cast<gg_plan_t *>(plan))
                                                 : chunk_cols<float>(const_cast<gg_plan_t *>(plan))) > 0;
  return GG_OK;
}

gg_status gg_sync(gg_plan_t *plan) {
  if (!plan) return fail(nullptr, GG_EINVAL, "plan is NULL");
  cudaError_t e = cudaStreamSynchronize(plan->stream);
  if (e != cudaSuccess) return cuda_fail(plan, e, "cudaStreamSynchronize");
  int word = 0;
  e = cudaMemcpy(&word, plan->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(plan, e, "reading the device error word");
  if (word == 0) return GG_OK;
  cudaMemset(plan->err, 0, sizeof(int));
  if (word == 2) return fail(plan, GG_ETIMEOUT, "a device-side tile-copy wait gave up");
  char msg[96];
  std::snprintf(msg, sizeof msg, "unexpected device error word %d", word);
  return fail(plan, GG_ECUDA, msg);
}

gg_status gg_test_arm_fault(gg_plan_t *plan, int kind, uint32_t wait_us) {
  if (!plan) return fail(nullptr, GG_EINVAL, "plan is NULL");
  if (kind == GG_TEST_NONE) {
    plan->test_skip_copy = 0;
    return GG_OK;
  }
  if (kind != GG_TEST_SKIP_COPY) return fail(plan, GG_EINVAL, "unknown fault kind");
  if (wait_us < 1 || wait_us > 1000000) return fail(plan, GG_EINVAL, "wait_us must be in [1, 1e6]");
  plan->test_skip_copy = 1;
  plan->test_wait_us = wait_us;
  return GG_OK;
}

const char *gg_last_error(const gg_plan_t *plan) {
  return plan ? plan->last_error.c_str() : g_thread_error.c_str();
}

void gg_free(gg_plan_t *plan) {
  if (!plan) return;
  release(plan);
  delete plan;
}

gg_status gg_batch_plan(gg_batch_t **batch, const gg_params *params, int count, void *stream) {
  if (!batch || !params || count < 1) return fail(nullptr, GG_EINVAL, "bad batch arguments");
  *batch = nullptr;
  int64_t lines = 0;  // the batched kernels index lines with 32-bit integers
  for (int i = 0; i < count; ++i) {
    const std::string msg = validate(&params[i]);
    if (!msg.empty()) return fail(nullptr, GG_EINVAL, "realization " + std::to_string(i) + ": " + msg);
    lines += params[i].n * params[i].n;
  }
  if (lines >= ((int64_t)1 << 31)) return fail(nullptr, GG_EINVAL, "batch too large (N^2 summed >= 2^31)");
  gg_batch_t *b = new (std::nothrow) gg_batch_t();
  if (!b) return fail(nullptr, GG_ENOMEM, "host allocation failed");
  b->count = count;
  b->stream = (cudaStream_t)stream;
  for (int i = 0; i < count; ++i) {
    b->cells += params[i].n * params[i].n * params[i].n;
    size_t gi = 0;
    for (; gi < b->groups.size(); ++gi)
      if (same_params(params[b->groups[gi].members[0]], params[i])) break;
    if (gi == b->groups.size()) b->groups.emplace_back();
    b->groups[gi].members.push_back(i);
  }
  gg_status st = GG_OK;
  cudaError_t e = cudaSuccess;
  for (auto &g : b->groups) {
    const gg_params &p = params[g.members[0]];
    if ((st = gg_plan(&g.plan, &p, stream)) != GG_OK) break;
    const size_t nb = g.members.size();
    const size_t bytes = (size_t)p.n * p.n * p.n * (p.prec == GG_F64 ? 8 : 4) * nb;
    for (void *&w : g.work)
      if (cudaMalloc(&w, bytes) != cudaSuccess) st = fail(nullptr, GG_ENOMEM, "cudaMalloc of a batch workspace failed");
    if (st != GG_OK) break;
    if ((e = cudaMalloc(&g.d_seeds, sizeof(uint64_t) * nb)) != cudaSuccess ||
        (e = cudaMalloc((void **)&g.d_lists, sizeof(void *) * 9 * nb)) != cudaSuccess ||
        (e = cudaMallocHost(&g.h_seeds, sizeof(uint64_t) * nb)) != cudaSuccess ||
        (e = cudaMallocHost((void **)&g.h_lists, sizeof(void *) * 9 * nb)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&g.s, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&g.ev, cudaEventDisableTiming)) != cudaSuccess) {
      st = cuda_fail(nullptr, e, "batch set-up");
      break;
    }
  }
  if (st == GG_OK && ((e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming)) != cudaSuccess ||
                      (e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming)) != cudaSuccess))
    st = cuda_fail(nullptr, e, "batch events");
  if (st != GG_OK) {
    batch_release(b);
    delete b;
    return st;
  }
  *batch = b;
  return GG_OK;
}

gg_status gg_batch_autotune(gg_batch_t *b, int reps) {
  if (!b || reps < 1) return fail(nullptr, GG_EINVAL, "bad arguments");
  for (auto &g : b->groups) {
    g.plan->stream = b->stream;
    const gg_status st = gg_autotune(g.plan, reps);
    if (st != GG_OK) return fail(nullptr, st, g.plan->last_error);
  }
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
  }
  return GG_OK;
}

gg_status gg_batch_run(gg_batch_t *b, const uint64_t *seeds, void *const *psi, void *const *pos,
                       void *const *vel) {
  if (!b || !seeds) return fail(nullptr, GG_EINVAL, "batch or seeds is NULL");
  cudaError_t e;
  if (b->ran && (e = cudaEventSynchronize(b->done)) != cudaSuccess)  // staging is re-read by the graph
    return cuda_fail(nullptr, e, "waiting for the previous batch run");
  void *const *outs[3] = {psi, pos, vel};
  // bits 0-8: (output o, component j) wanted by some realization; bits 9-17:
  // wanted by every realization (the graph's kernels may then skip the
  // per-realization null checks)
  uint32_t sig = 0, all = (1u << 9) - 1;
  for (int i = 0; i < b->count; ++i)
    for (int o = 0; o < 3; ++o)
      for (int j = 0; j < 3; ++j) {
        const void *ptr = outs[o] ? outs[o][3 * i + j] : nullptr;
        if (ptr && ((uintptr_t)ptr & 15u)) return fail(nullptr, GG_EINVAL, "output buffer unaligned");
        if (ptr) sig |= 1u << (o * 3 + j);
        else all &= ~(1u << (o * 3 + j));
      }
  sig |= all << 9;
  if ((b->test_stall || b->test_ran) && b->exec) {  // capture with (or again without) the fault
    cudaGraphExecDestroy(b->exec);
    cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
  }
  b->test_ran = b->test_stall;
  for (auto &g : b->groups) {
    const int nb = (int)g.members.size();
    for (int k = 0; k < nb; ++k) {
      const int i = g.members[k];
      g.h_seeds[k] = seeds[i];
      for (int o = 0; o < 3; ++o)
        for (int j = 0; j < 3; ++j) g.h_lists[(o * 3 + j) * nb + k] = outs[o] ? outs[o][3 * i + j] : nullptr;
    }
  }
  if (!b->exec || sig != b->signature) {
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      cudaGraphDestroy(b->graph);
      b->exec = nullptr;
      b->graph = nullptr;
    }
    if ((e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return cuda_fail(nullptr, e, "cudaStreamBeginCapture (a batch needs a non-default stream)");
    gg_status st = GG_OK;
    if (b->persistent) st = persist_passes(b, b->stream, sig);
    else if ((e = cudaEventRecord(b->fork, b->stream)) != cudaSuccess) st = cuda_fail(nullptr, e, "fork");
    for (auto &g : b->groups) {
      if (b->persistent) break;
      if (st != GG_OK) break;
      if ((e = cudaStreamWaitEvent(g.s, b->fork, 0)) != cudaSuccess) {
        st = cuda_fail(nullptr, e, "fork wait");
        break;
      }
      st = g.plan->real_bytes == 8 ? group_passes<double>(g, g.s, sig) : group_passes<float>(g, g.s, sig);
      if (st != GG_OK) break;
      if ((e = cudaEventRecord(g.ev, g.s)) != cudaSuccess ||
          (e = cudaStreamWaitEvent(b->stream, g.ev, 0)) != cudaSuccess)
        st = cuda_fail(nullptr, e, "join");
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(b->stream, &graph);
    if (st != GG_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (ec != cudaSuccess) return cuda_fail(nullptr, ec, "cudaStreamEndCapture");
    if ((e = cudaGraphInstantiate(&b->exec, graph, 0)) != cudaSuccess) {
      cudaGraphDestroy(graph);
      return cuda_fail(nullptr, e, "cudaGraphInstantiate");
    }
    b->graph = graph;
    b->signature = sig;
  }
  if ((e = cudaGraphLaunch(b->exec, b->stream)) != cudaSuccess ||
      (e = cudaEventRecord(b->done, b->stream)) != cudaSuccess)
    return cuda_fail(nullptr, e, "cudaGraphLaunch");
  b->ran = true;
  b->test_stall = 0;
  return GG_OK;
}

gg_status gg_batch_test_arm_fault(gg_batch_t *b, int kind, uint32_t wait_us) {
  if (!b) return fail(nullptr, GG_EINVAL, "batch is NULL");
  if (kind == GG_TEST_NONE) {
    b->test_stall = 0;
    return GG_OK;
  }
  if (kind != GG_TEST_STALL_COUNT) return fail(nullptr, GG_EINVAL, "unknown fault kind");
  if (!b->persistent) return fail(nullptr, GG_EINVAL, "the stall test needs the persistent schedule");
  if (wait_us < 1 || wait_us > 1000000) return fail(nullptr, GG_EINVAL, "wait_us must be in [1, 1e6]");
  b->test_stall = 1;
  b->test_wait_us = wait_us;
  return GG_OK;
}

gg_status gg_batch_sync(gg_batch_t *b) {
  if (!b) return fail(nullptr, GG_EINVAL, "batch is NULL");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaStreamSynchronize");
  for (auto &g : b->groups) {
    const gg_status st = gg_sync(g.plan);
    if (st != GG_OK) return fail(nullptr, st, g.plan->last_error);
  }
  return GG_OK;
}

gg_status gg_batch_info(const gg_batch_t *b, int *groups, int64_t *cells) {
  if (!b) return fail(nullptr, GG_EINVAL, "batch is NULL");
  if (groups) *groups = (int)b->groups.size();
  if (cells) *cells = b->cells;
  return GG_OK;
}

gg_status gg_batch_set_persistent(gg_batch_t *b, int on) {
  if (!b) return fail(nullptr, GG_EINVAL, "batch is NULL");
  if (on < 0 || on > 256 || (on > 1 && (on & (on - 1))))
    return fail(nullptr, GG_EINVAL, "on: 0, 1 or a power of two up to 256 (tiles per work item)");
  if (on) {
    if ((int)b->groups.size() > gg::kPersistMaxGroups)
      return fail(nullptr, GG_EINVAL, "persistent form: at most 4 parameter groups");
    for (auto &g : b->groups)
      if (g.plan->real_bytes != 4 || !gg::persist_has((int)g.plan->p.n))
        return fail(nullptr, GG_EINVAL, "persistent form: FP32 grids of N = 64, 128, 192, 256, 384 only");
    if (!b->counters) {
      const size_t words = 64 + (size_t)8 * b->count;
      if (cudaMalloc(&b->counters, words * sizeof(unsigned)) != cudaSuccess) {
        b->counters = nullptr;
        return fail(nullptr, GG_ENOMEM, "cudaMalloc of the pass counters failed");
      }
    }
  }
  cudaError_t e;
  if (b->ran && (e = cudaEventSynchronize(b->done)) != cudaSuccess)
    return cuda_fail(nullptr, e, "waiting for the previous batch run");
  if (b->exec) {  // the next gg_batch_run captures the other schedule
    cudaGraphExecDestroy(b->exec);
    cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
  }
  b->persistent = on != 0;
  b->persist_chunk = on > 1 ? on : 0;
  return GG_OK;
}

gg_status gg_batch_launches(const gg_batch_t *b, int *kernels) {
  if (!b || !kernels) return fail(nullptr, GG_EINVAL, "batch and kernels are required");
  *kernels = 0;
  if (!b->graph) return GG_OK;  // not captured yet: no gg_batch_run so far
  size_t count = 0;
  cudaError_t e = cudaGraphGetNodes(b->graph, nullptr, &count);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGraphGetNodes");
  std::vector<cudaGraphNode_t> nodes(count);
  if (count && (e = cudaGraphGetNodes(b->graph, nodes.data(), &count)) != cudaSuccess)
    return cuda_fail(nullptr, e, "cudaGraphGetNodes");
  int k = 0;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType t;
    if ((e = cudaGraphNodeGetType(nd, &t)) != cudaSuccess) return cuda_fail(nullptr, e, "cudaGraphNodeGetType");
    if (t == cudaGraphNodeTypeKernel) ++k;
  }
  *kernels = k;
  return GG_OK;
}

void gg_batch_free(gg_batch_t *b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  batch_release(b);
  delete b;
}

}  // extern "C"
