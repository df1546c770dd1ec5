// sft_api.cu -- host side of libsft: the C-ABI of include/sft.h.
//
// The handle keeps every realization's map resident in one device pool and
// three work arrays sized for one "wave" of realizations (the HBM-budget
// admission unit).  sft_step runs the Lie-split step of Sec. 3.5 for all
// realizations of a wave in lockstep: the advection stages then the RKL2
// stages, each ONE batched launch over a tile table whose prefix holds the
// realizations still active at that stage.  Each distinct step
// configuration (per-realization dt and stage count) owns its device
// parameter block and, by default, one captured CUDA graph that replays the
// whole step.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <numeric>
#include <string>
#include <type_traits>
#include <vector>

#include "sft.h"
#include "sft_device.cuh"
#include <nvtx3/nvToolsExt.h>

using namespace sft;

namespace {

// Sec. 3.3: R_sun = 6.96e8 m, time unit 1 hour.
constexpr double kRsunM = 6.96e8;
constexpr double kRsunCm = 6.96e10;
constexpr double kMsToRsHr = 3600.0 / kRsunM;
constexpr double kKm2sToRs2Hr = 3600.0 * 1.0e6 / (kRsunM * kRsunM);
constexpr double kPi = 3.14159265358979323846;

thread_local std::string g_create_error;

struct ShapeInfo {
  int nt = 0, np = 0, pitch = 0;
  int geo = 0;        // first row in the geometry tables
  int col = 0;        // first entry in the cos/sin(phi) tables
  int tile_rows = 0;  // 0 = autotune on first step
  int band_rows = 0;  // rows per band of the fused RKL2 work items; 0 = autotune on first step
  double dth = 0, dph = 0, cap = 0;
  std::vector<double> sin_t, sin_h, cos_t;  // sin th_j, sin th_{f+1/2}, cos th_j
};

struct RealInfo {
  int shape = 0;
  int64_t off = 0, woff = 0, cells = 0;  // cells = nt*pitch elements
  int wave = 0;
  int flow_row = 0;
  double t = 0.0;
  int64_t steps = 0;
  bool has_flows = false;
  sft_flow_params fp{};
  double nu = 0.0;        // R_sun^2/hr
  double dt_cfl = 0.0;    // hours (inf when advection is off)
  double dt_euler = 0.0;  // hours (inf when nu == 0)
  double cap_nu = 1.0;    // nu at the cap faces relative to nudt (grid-based nu: nu_g(theta_1/2))
  sft_rfe_params rfe{};   // random flux emergence (method 0: off)
  double rfe_t0 = 0.0;    // time of source map 0
  int64_t rfe_m0 = -1;    // map window whose balance factors are on the device (-1: none)
};

constexpr int kMaxChains = 6;   // concurrent launch chains of the fused RKL2 passes (at most)
constexpr int kStageRing = 8;   // pinned staging buffers of the configuration tables
constexpr int kMaxConfigs = 24; // cached step configurations (tile tables, graphs) per wave

struct Config {
  bool fused = false;            // built for the fused RKL2 path
  Tile* d_ftiles = nullptr;      // fused-pass tiles of every chain (pole blocks, then interior blocks)
  // The fused passes run as n_chains independent launch chains on their own
  // streams (realizations dealt alternately from the stage-sorted order), so
  // one chain's launches fill the SMs while the other's drain.
  int n_chains = 1;
  // A chain's tiles are its members' pole blocks (two per member, in member
  // order), then their interior blocks; a pass launches the pole blocks of
  // its active members (a prefix), then their interior blocks (a prefix).
  int fbase[kMaxChains] = {};                 // first tile of each chain in d_ftiles
  int fcaps[kMaxChains] = {};                 // pole tiles of each chain (the interior tiles start there)
  std::vector<int> fused_tiles[kMaxChains];   // [chain][j0] = interior tiles of the pass starting at stage j0
  std::vector<int> fused_caps[kMaxChains];    // [chain][j0] = pole tiles of that pass
  int64_t fused_launches = 0;           // non-empty fused-pass launches per step (pole + interior)
  std::vector<double> dt;        // per wave member (wave order)
  std::vector<int> s;            // per wave member
  std::vector<int> tr;           // tile rows per shape at build time
  std::vector<int> band;         // fused band rows per shape at build time
  int smax = 0, n_adv_tiles = 0;  // advection tiles (row groups of kAdvRun rows per thread)
  std::vector<int> stage_tiles;  // [j] = tiles launched at RKL2 stage j (1..smax)
  Tile* d_tiles = nullptr;       // single-stage RKL2 tiles
  Tile* d_atiles = nullptr;      // advection tiles
  StepParam* d_sp = nullptr;
  void* d_coef = nullptr;
  void* d_blob = nullptr;        // the one allocation holding the tables above
  cudaGraphExec_t exec = nullptr;
  uint64_t last_use = 0;
  int uses = 0;  // steps run with this configuration (graphs are captured from the second)
  double cells_adv = 0, cell_stages_diff = 0, cell_updates = 0, diff_words = 0;
  int64_t launches = 0;
  int realization_steps = 0;
};

struct Wave {
  std::vector<int> reals;
  std::vector<std::unique_ptr<Config>> configs;
};

template <typename T> struct Tables {
  RowGeo<T>* geo = nullptr;
  RowFlow<T>* flow = nullptr;
};

}  // namespace

struct sft_grid {
  int n_real = 0;
  sft_prec prec = SFT_FP32;
  size_t elem = 4;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  std::vector<ShapeInfo> shapes;
  std::vector<RealInfo> reals;
  std::vector<Wave> waves;
  int wave_size = 0;
  int64_t state_elems = 0, work_elems = 0;
  // device memory
  void* state = nullptr;
  void* work[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  int n_work = 3;              // 5 when the fused RKL2 path is possible
  bool fused_ok = false;       // FP32 and every shape has an interior band
  bool fused = false;          // use rkl2_fused_kernel (K stages per launch)
  void* polar = nullptr;       // ring-sum partials of the fused path (doubles)
  int64_t polar_elems = 0;
  RealDesc* d_desc = nullptr;
  std::vector<RealDesc> desc;  // host copy (geometry offsets change with grid-based nu)
  bool geo_custom = false;     // some realization has its own geometry block
  bool any_rfe = false;        // random flux emergence on for some realization
  RfeStep* d_rfe = nullptr;    // this step's maps and weights per realization
  double* d_rfe_fac = nullptr; // Eq. (fluxbal) factors of the step's maps (8 per realization)
  ShapeConst* d_shc = nullptr;
  void* d_geo = nullptr;       // RowGeo<T>
  RowGeoD* d_geod = nullptr;
  double* d_cosp = nullptr;
  double* d_sinp = nullptr;
  float4* d_csf = nullptr;     // cos / sin phi as (hi, lo) float pairs
  void* d_flow = nullptr;      // RowFlow<T>
  int* d_status = nullptr;
  RedTile* d_rtiles = nullptr;
  int* d_rstart = nullptr;
  int n_rtiles = 0;
  double* d_partials = nullptr;
  double* d_red = nullptr;     // per realization fold output
  double* h_red = nullptr;     // pinned mirror
  double* d_wpar = nullptr;
  std::vector<double> h_wpar_last;
  int64_t* d_obs_off = nullptr;
  std::vector<int64_t> h_obs_off_last;
  void* d_obs = nullptr;
  size_t obs_bytes = 0;
  int geo_rows = 0, flow_rows = 0, col_entries = 0;
  // step machinery
  bool flows_set = false;
  bool strang = false;         // Strang splitting (Sec. 3.5): A(dt/2) D(dt) A(dt/2)
  bool use_graphs = true;
  bool profiling = false;
  uint64_t use_counter = 0;
  cudaEvent_t ev[6] = {};      // advection, RKL2, second (Strang) advection phases
  cudaStream_t side[kMaxChains] = {};           // chains 1.. of the fused RKL2 passes
  int n_sm = 152;                               // streaming multiprocessors of the device
  cudaEvent_t fork = nullptr;                   // ordering events (no timing)
  cudaEvent_t join[kMaxChains] = {};
  // pinned staging of the step-configuration tables: a ring of buffers, each
  // reused once the upload that last read it has completed (its event)
  char* cfg_stage[kStageRing] = {};
  size_t cfg_stage_bytes[kStageRing] = {};
  cudaEvent_t cfg_stage_ev[kStageRing] = {};
  bool cfg_stage_pending[kStageRing] = {};
  int cfg_stage_next = 0;
  sft_stats stats{};
};

namespace {

// An NVTX range for the duration of a public call (a timeline marker for
// profilers; no cost without one attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

sft_status fail(sft_handle h, sft_status code, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return code;
}

// Host fault injection (sft_debug_fail_alloc): armed with n, the n-th device
// or pinned allocation made by an sft_* call from then on reports
// cudaErrorMemoryAllocation without allocating, then the injector disarms.
std::atomic<int> g_fail_alloc{0};

bool injected_alloc_failure() {
  int n = g_fail_alloc.load();
  while (n > 0)
    if (g_fail_alloc.compare_exchange_weak(n, n - 1)) return n == 1;
  return false;
}

template <typename P> cudaError_t dev_malloc(P** p, size_t bytes) {
  if (injected_alloc_failure()) return cudaErrorMemoryAllocation;
  return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}

template <typename P> cudaError_t dev_malloc_async(P** p, size_t bytes, cudaStream_t st) {
  if (injected_alloc_failure()) return cudaErrorMemoryAllocation;
  return cudaMallocAsync(reinterpret_cast<void**>(p), bytes, st);
}

template <typename P> cudaError_t host_malloc(P** p, size_t bytes) {
  if (injected_alloc_failure()) return cudaErrorMemoryAllocation;
  return cudaMallocHost(reinterpret_cast<void**>(p), bytes);
}

#define SFT_CUDA(h, call)                                                              \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(h, e_ == cudaErrorMemoryAllocation ? SFT_ERR_OOM : SFT_ERR_CUDA,     \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                 \
  } while (0)

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// ---- Sec. 3.2 geometry, per shape (FP64 on the host) ----------------------
void build_shape(ShapeInfo& s) {
  s.dth = kPi / (s.nt - 1);
  s.dph = 2.0 * kPi / s.np;
  s.cap = 2.0 * kPi * (1.0 - std::cos(0.5 * s.dth));
  s.sin_t.resize(s.nt);
  s.cos_t.resize(s.nt);
  s.sin_h.resize(s.nt - 1);
  for (int j = 0; j < s.nt; ++j) {
    const double th = j == s.nt - 1 ? kPi : j * s.dth;
    s.sin_t[j] = (j == 0 || j == s.nt - 1) ? 0.0 : std::sin(th);
    s.cos_t[j] = std::cos(th);
  }
  for (int f = 0; f < s.nt - 1; ++f) s.sin_h[f] = std::sin((f + 0.5) * s.dth);
}

template <typename T>
void geo_rows(const ShapeInfo& s, std::vector<RowGeo<T>>& g, std::vector<RowGeoD>& gd) {
  for (int j = 0; j < s.nt; ++j) {
    RowGeo<T> r{};
    RowGeoD d{};
    const bool pole = j == 0 || j == s.nt - 1;
    d.cos_t = s.cos_t[j];
    d.sin_t = s.sin_t[j];
    d.lat = 0.5 * kPi - (j == s.nt - 1 ? kPi : j * s.dth);
    if (pole) {
      d.area = s.cap / s.np;
    } else {
      const double st = s.sin_t[j];
      const double sdn = s.sin_h[j - 1], sup = s.sin_h[j];
      r.cN = T(sdn / (s.dth * s.dth * st));
      r.cS = T(sup / (s.dth * s.dth * st));
      r.cE = T(1.0 / (s.dph * s.dph * st * st));
      r.cC = -(r.cN + r.cS + T(2) * r.cE);
      r.inv_sdth = T(1.0 / (st * s.dth));
      r.inv_sdph = T(1.0 / (st * s.dph));
      r.sdn = T(sdn);
      r.sup = T(sup);
      d.area = st * s.dth * s.dph;
    }
    g.push_back(r);
    gd.push_back(d);
  }
}

// Eq. (diffgrid): nu_g at theta face f (f + 1/2), R_sun^2 / hour.
double grid_nu_face(const ShapeInfo& s, double alpha, int f) {
  const double a = s.dph * s.sin_h[f];
  return alpha * (s.dth * s.dth + a * a);
}

// A realization's own geometry block with the grid-based diffusivity folded
// into cN, cS, cE (computed in FP64 from the faces' nu, then rounded).
template <typename T>
void geo_rows_grid_nu(const ShapeInfo& s, double alpha, std::vector<RowGeo<T>>& g, std::vector<RowGeoD>& gd) {
  const size_t base = g.size();
  geo_rows<T>(s, g, gd);
  for (int j = 1; j < s.nt - 1; ++j) {
    const double st = s.sin_t[j], ndn = grid_nu_face(s, alpha, j - 1), nup = grid_nu_face(s, alpha, j);
    RowGeo<T>& r = g[base + j];
    r.cN = T(ndn * s.sin_h[j - 1] / (s.dth * s.dth * st));
    r.cS = T(nup * s.sin_h[j] / (s.dth * s.dth * st));
    r.cE = T(0.5 * (ndn + nup) / (s.dph * s.dph * st * st));
    r.cC = -(r.cN + r.cS + T(2) * r.cE);
  }
}

// ---- Sec. 2.1.1 flows and Sec. 3.6.2 / 3.7.2 limits -----------------------
struct FlowRows {
  std::vector<double> vt;  // faces f = 0..nt-2
  std::vector<double> vp;  // rows
};

FlowRows flow_profiles(const ShapeInfo& s, const sft_flow_params& p) {
  FlowRows f;
  f.vp.resize(s.nt);
  f.vt.resize(s.nt - 1);
  for (int j = 0; j < s.nt; ++j) {
    const double c = s.cos_t[j], c2 = c * c;
    f.vp[j] = (p.d0 + p.d2 * c2 + p.d4 * c2 * c2) * s.sin_t[j] * kMsToRsHr;
  }
  for (int i = 0; i < s.nt - 1; ++i) {
    const double c = std::cos((i + 0.5) * s.dth), c2 = c * c;
    f.vt[i] = -(p.m1 * c + p.m3 * c * c2 + p.m5 * c * c2 * c2) * s.sin_h[i] * kMsToRsHr;
  }
  return f;
}

// Eq. (ssprk43_dt) (or Eq. advection_timestep for FE / SSPRK(3,3)) with the
// flanking-maximum velocities, times the safety factor.
double cfl_limit(const ShapeInfo& s, const FlowRows& f, const sft_flow_params& p) {
  double rmax = 0.0;
  for (int j = 1; j < s.nt - 1; ++j) {
    const double vth = std::max(std::fabs(f.vt[j - 1]), std::fabs(f.vt[j]));
    const double r = vth / s.dth + std::fabs(f.vp[j]) / (s.sin_t[j] * s.dph);
    rmax = std::max(rmax, r);
  }
  if (rmax <= 0.0) return INFINITY;
  double lim = 1.0 / rmax;
  if (p.adv_time != SFT_TIME_SSPRK43) lim *= 0.5;
  return p.cfl_safety * lim;
}

// Explicit-Euler diffusion limit 1 / max_i |a_ii| (Gershgorin) of the
// Eq. (diffusion_matrix) operator with the App. A cap rows.
double euler_limit(const ShapeInfo& s, double nu) {
  if (nu <= 0.0) return INFINITY;
  double amax = 0.0;
  for (int j = 1; j < s.nt - 1; ++j) {
    const double st = s.sin_t[j];
    const double a = nu * ((s.sin_h[j - 1] + s.sin_h[j]) / (s.dth * s.dth * st) +
                           2.0 / (s.dph * s.dph * st * st));
    amax = std::max(amax, a);
  }
  const double pole = nu * std::sin(0.5 * s.dth) * s.dph * s.np / (s.dth * s.cap);
  amax = std::max(amax, pole);
  return 1.0 / amax;
}

// The same limit with the grid-based diffusivity of Eq. (diffgrid).
double euler_limit_grid(const ShapeInfo& s, double alpha) {
  double amax = 0.0;
  for (int j = 1; j < s.nt - 1; ++j) {
    const double st = s.sin_t[j], ndn = grid_nu_face(s, alpha, j - 1), nup = grid_nu_face(s, alpha, j);
    const double a = (ndn * s.sin_h[j - 1] + nup * s.sin_h[j]) / (s.dth * s.dth * st) +
                     (ndn + nup) / (s.dph * s.dph * st * st);
    amax = std::max(amax, a);
  }
  const double line = std::sin(0.5 * s.dth) * s.dph * s.np / (s.dth * s.cap);
  amax = std::max(amax, std::max(grid_nu_face(s, alpha, 0), grid_nu_face(s, alpha, s.nt - 2)) * line);
  return amax > 0.0 ? 1.0 / amax : INFINITY;
}

// Eq. (rfe_s) integrated over [a, b]: maps k (from t0, tau apart) and
// weights (hours) such that the integral is sum_k w_k S_k (each piece of the
// piecewise-linear source integrates exactly at its midpoint).  Returns the
// first map index; w[0..3] for maps m0..m0+3 (a step spans at most two
// segments because it is capped at tau).
int64_t rfe_weights(double t0, double tau, double a, double b, double (&w)[4]) {
  for (double& x : w) x = 0.0;
  if (!std::isfinite(tau) || tau <= 0.0) {
    w[0] = b - a;
    return 0;
  }
  const int64_t m0 = (int64_t)std::floor((a - t0) / tau + 1e-12);
  double t = a;
  while (t < b) {
    const int64_t k = (int64_t)std::floor((t - t0) / tau + 1e-12);
    const double end = std::min(b, t0 + (double)(k + 1) * tau);
    const double al = (0.5 * (t + end) - (t0 + (double)k * tau)) / tau;
    const int64_t i = k - m0;
    if (i >= 0 && i + 1 < 4) {
      w[i] += (end - t) * (1.0 - al);
      w[i + 1] += (end - t) * al;
    }
    t = end;
  }
  return m0;
}

// RKL2 stage count: smallest s >= 2 with dt <= dt_E (s^2 + s - 2) / 4.
int rkl2_stages(double dt, double dte) {
  if (!(dt > 0.0)) return 0;
  if (!std::isfinite(dte)) return 0;
  int s = (int)std::ceil(0.5 * (-1.0 + std::sqrt(9.0 + 16.0 * dt / dte)));
  if (s < 2) s = 2;
  while ((double)(s * (int64_t)s + s - 2) * dte < 4.0 * dt) ++s;
  while (s > 2 && (double)((s - 1) * (int64_t)(s - 1) + (s - 1) - 2) * dte >= 4.0 * dt) --s;
  return s;
}

// RKG2(3/2) stage count (Sec. 3.7.2): smallest s >= 2 with
// dt <= dt_E (s^2 + 3s - 4) / 6.
int rkg2_stages(double dt, double dte) {
  if (!(dt > 0.0)) return 0;
  if (!std::isfinite(dte)) return 0;
  int s = (int)std::ceil(0.5 * (-3.0 + std::sqrt(25.0 + 24.0 * dt / dte)));
  if (s < 2) s = 2;
  while ((double)(s * (int64_t)s + 3 * s - 4) * dte < 6.0 * dt) ++s;
  while (s > 2 && (double)((s - 1) * (int64_t)(s - 1) + 3 * (s - 1) - 4) * dte >= 6.0 * dt) --s;
  return s;
}

// Stage count of a realization's diffusion scheme for a step of dt hours.
int sts_stages(int scheme, double dt, double dte) {
  return scheme == SFT_DIFF_RKL2 ? rkl2_stages(dt, dte) : scheme == SFT_DIFF_RKG2 ? rkg2_stages(dt, dte) : 0;
}

// RKG2(3/2) coefficients for stages 0..s in the increment form of rkl2_coefs:
// the RKL2 construction on the Gegenbauer polynomials C_j^(3/2),
// R_j(z) = a_j + b_j C_j(1 + w1 z), w1 = 6 / ((s-1)(s+4)),
// b_j = 4(j-1)(j+4) / (3j(j+1)(j+2)(j+3)) (b_0 = b_1 = b_2), C_j(1) =
// (j+1)(j+2)/2, a_j = 1 - b_j C_j(1); the stages follow the recurrence
// j C_j(x) = (2j+1) x C_{j-1}(x) - (j+1) C_{j-2}(x).
template <typename T>
void rkg2_coefs(int s, std::vector<Coef<T>>& out) {
  const double w1 = 6.0 / ((s - 1.0) * (s + 4.0));
  auto b = [](int j) {
    const double jj = j < 2 ? 2.0 : (double)j;
    return 4.0 * (jj - 1.0) * (jj + 4.0) / (3.0 * jj * (jj + 1.0) * (jj + 2.0) * (jj + 3.0));
  };
  auto a = [&](int j) { return 1.0 - b(j) * (j + 1.0) * (j + 2.0) / 2.0; };
  out.push_back(Coef<T>{T(0), T(0), T(0), T(0)});  // stage 0 unused
  out.push_back(Coef<T>{T(0), T(0), T(3.0 * b(1) * w1), T(0)});
  for (int j = 2; j <= s; ++j) {
    const double mu = (2.0 * j + 1.0) / j * b(j) / b(j - 1);
    const double nu = -(j + 1.0) / j * b(j) / b(j - 2);
    const double mut = mu * w1;
    const double gt = -a(j - 1) * mut;
    out.push_back(Coef<T>{T(mu), T(nu), T(mut), T(mut + gt)});
  }
}

// RKL2 coefficients (Meyer, Balsara & Aslam 2014) for stages 0..s, stored in
// the increment form used by rkl2_stage_kernel: {mu_j, nu_j, mu~_j, mu~_j + gamma~_j}.
template <typename T>
void rkl2_coefs(int s, std::vector<Coef<T>>& out) {
  const double w1 = 4.0 / ((double)s * s + s - 2.0);
  auto b = [](int j) { return j <= 2 ? 1.0 / 3.0 : ((double)j * j + j - 2.0) / (2.0 * j * (j + 1.0)); };
  out.push_back(Coef<T>{T(0), T(0), T(0), T(0)});  // stage 0 unused
  out.push_back(Coef<T>{T(0), T(0), T(b(1) * w1), T(0)});
  for (int j = 2; j <= s; ++j) {
    const double mu = (2.0 * j - 1.0) / j * b(j) / b(j - 1);
    const double nu = -(j - 1.0) / j * b(j) / b(j - 2);
    const double mut = mu * w1;
    const double gt = -(1.0 - b(j - 1)) * mut;
    out.push_back(Coef<T>{T(mu), T(nu), T(mut), T(mut + gt)});
  }
}

template <typename T> T* ptr(void* p) { return static_cast<T*>(p); }

// Configuration buffers are stream-ordered allocations of the handle's
// stream: freeing an evicted configuration waits for no other work (a graph
// still in flight is released by the runtime when it completes).
void free_config(Config& c, cudaStream_t st) {
  if (c.exec) cudaGraphExecDestroy(c.exec);
  if (c.d_blob) cudaFreeAsync(c.d_blob, st);
  c.exec = nullptr;
  c.d_blob = nullptr;
  c.d_ftiles = nullptr;
  c.d_tiles = nullptr;
  c.d_atiles = nullptr;
  c.d_sp = nullptr;
  c.d_coef = nullptr;
}

void free_handle(sft_handle h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (auto& w : h->waves)
    for (auto& c : w.configs) free_config(*c, h->stream);
  if (h->stream) cudaStreamSynchronize(h->stream);
  cudaFree(h->state);
  for (auto& w : h->work) cudaFree(w);
  cudaFree(h->polar);
  cudaFree(h->d_desc);
  cudaFree(h->d_shc);
  cudaFree(h->d_geo);
  cudaFree(h->d_geod);
  cudaFree(h->d_cosp);
  cudaFree(h->d_sinp);
  cudaFree(h->d_csf);
  cudaFree(h->d_flow);
  cudaFree(h->d_status);
  cudaFree(h->d_rtiles);
  cudaFree(h->d_rstart);
  cudaFree(h->d_partials);
  cudaFree(h->d_rfe);
  cudaFree(h->d_rfe_fac);
  cudaFree(h->d_red);
  if (h->h_red) cudaFreeHost(h->h_red);
  cudaFree(h->d_wpar);
  cudaFree(h->d_obs_off);
  cudaFree(h->d_obs);
  for (auto& e : h->ev)
    if (e) cudaEventDestroy(e);
  if (h->fork) cudaEventDestroy(h->fork);
  for (auto& e : h->join)
    if (e) cudaEventDestroy(e);
  for (int i = 0; i < kStageRing; ++i) {
    if (h->cfg_stage_ev[i]) {
      if (h->cfg_stage_pending[i]) cudaEventSynchronize(h->cfg_stage_ev[i]);
      cudaEventDestroy(h->cfg_stage_ev[i]);
    }
    if (h->cfg_stage[i]) cudaFreeHost(h->cfg_stage[i]);
  }
  for (auto& q : h->side)
    if (q) cudaStreamDestroy(q);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

sft_status check_status_word(sft_handle h) {
  int st = 0;
  SFT_CUDA(h, cudaMemcpy(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st != 0) {
    SFT_CUDA(h, cudaMemset(h->d_status, 0, sizeof(int)));
    return fail(h, SFT_ERR_UNSTABLE, "non-finite values in the state (watchdog)");
  }
  return SFT_OK;
}

sft_status sync(sft_handle h) {
  SFT_CUDA(h, cudaStreamSynchronize(h->stream));
  return check_status_word(h);
}

// ---------------------------------------------------------------------------
// step configurations
// ---------------------------------------------------------------------------
int vec_width(const sft_grid* h) { return h->prec == SFT_FP32 ? 4 : 2; }

// Consistency of the host-built tables the kernels index by.  Every
// realization's rows lie inside the state pool, the work arrays, the cap
// scratch and the geometry, flow and longitude tables, and the state extents
// are disjoint; every tile names a realization and starts inside it.  Run
// whenever the tables are (re)built; a failure is an internal error reported
// as SFT_ERR_STATE before anything is launched.  Returns "" when consistent.
std::string check_desc(const sft_grid* h) {
  if ((int)h->desc.size() != h->n_real) return "descriptor count";
  std::vector<std::pair<int64_t, int64_t>> ext;
  for (int r = 0; r < h->n_real; ++r) {
    const RealDesc& d = h->desc[r];
    const auto at_ = [r]() { return " (realization " + std::to_string(r) + ")"; };  // formatted on failure only
    if (d.nt < 5 || d.np < 8 || d.pitch < (int)round_up(d.np, 4) || d.pitch % 4 != 0) return "shape" + at_();
    const int64_t cells = (int64_t)d.nt * d.pitch;
    if (d.off < 0 || d.off + cells > h->state_elems) return "state extent" + at_();
    if (d.woff < 0 || d.woff + cells > h->work_elems) return "work extent" + at_();
    if (h->fused_ok && (d.poff < 0 || d.poff + fused::part_elems(d.np) > h->polar_elems))
      return "ring-sum partials extent" + at_();
    if (h->fused_ok && (d.band <= fused::K || d.band > (1 << 16))) return "band rows" + at_();
    if (d.geo < 0 || d.geo + d.nt > h->geo_rows) return "geometry rows" + at_();
    if (d.flow < 0 || d.flow + d.nt > h->flow_rows) return "flow rows" + at_();
    if (d.col < 0 || d.col + d.np > h->col_entries) return "longitude table" + at_();
    if (d.shape < 0 || d.shape >= (int)h->shapes.size()) return "shape id" + at_();
    ext.emplace_back(d.off, d.off + cells);
  }
  std::sort(ext.begin(), ext.end());
  for (size_t i = 1; i < ext.size(); ++i)
    if (ext[i].first < ext[i - 1].second) return "overlapping state extents";
  return "";
}

std::string check_tiles(const sft_grid* h, const std::vector<Tile>& tiles, bool fused_tiles) {
  // (the message is formatted only for a failing tile: this runs over every
  // tile of every new step configuration)
  auto at = [](size_t i) { return " (tile " + std::to_string(i) + ")"; };
  for (size_t i = 0; i < tiles.size(); ++i) {
    const Tile& t = tiles[i];
    if (t.r < 0 || t.r >= h->n_real) return "realization index" + at(i);
    const RealDesc& d = h->desc[t.r];
    const int kind = t.kind & 3;
    if (kind == 3) return "tile kind" + at(i);
    if (kind != 0) continue;
    if (fused_tiles) {
      if (t.j0 < 0 || t.j0 >= fused::n_bands(d.nt, d.band) * fused::n_strips(d.np)) return "fused work item" + at(i);
    } else {
      const int lx = t.kind >> 8;
      if (lx < 0 || (1 << lx) > kThreads) return "tile width" + at(i);
      if (t.j0 < 1 || t.j0 > d.nt - 2 || t.k0 < 0 || t.k0 >= d.np) return "tile origin" + at(i);
    }
  }
  return "";
}

// Interior tiles of TR thread rows x (kThreads/TR) threads; each thread row
// covers `run` grid rows (1 for the RKL2 stages, kAdvRun for advection).
void append_tiles(const sft_grid* h, int r, int tr, int run, std::vector<Tile>& tiles) {
  const RealInfo& ri = h->reals[r];
  const ShapeInfo& s = h->shapes[ri.shape];
  const int tx = kThreads / tr;
  int lx = 0;
  while ((1 << lx) < tx) ++lx;
  const int tc = tx * vec_width(h);
  for (int j0 = 1; j0 <= s.nt - 2; j0 += tr * run)
    for (int k0 = 0; k0 < s.np; k0 += tc) tiles.push_back(Tile{r, j0, k0, lx << 8});
  tiles.push_back(Tile{r, 0, 0, 1});
  tiles.push_back(Tile{r, 0, 0, 2});
}

// The two pole-triangle blocks of realization r (north, south).
void append_fused_poles(int r, std::vector<Tile>& tiles) {
  tiles.push_back(Tile{r, 0, 0, 1});
  tiles.push_back(Tile{r, 0, 0, 2});
}

void append_fused_interior(const sft_grid* h, int r, std::vector<Tile>& tiles) {
  const ShapeInfo& s = h->shapes[h->reals[r].shape];
  // rows 1 .. nt-2: (band, strip) work items, one per warp, WARPS per block
  const int items = fused::n_bands(s.nt, h->desc[r].band) * fused::n_strips(s.np);
  for (int i0 = 0; i0 < items; i0 += fused::WARPS) tiles.push_back(Tile{r, i0, 0, 0});
}

template <typename T>
sft_status build_config(sft_handle h, Wave& w, const std::vector<double>& dt,
                        const std::vector<int>& s, Config** out) {
  auto c = std::make_unique<Config>();
  // a failed allocation or copy below releases what was allocated before it
  struct Release {
    cudaStream_t st;
    Config* c;
    ~Release() {
      if (c) free_config(*c, st);
    }
  } release{h->stream, c.get()};
  c->dt = dt;
  c->s = s;
  for (auto& sh : h->shapes) c->tr.push_back(sh.tile_rows);
  for (auto& sh : h->shapes) c->band.push_back(sh.band_rows);
  const int nw = (int)w.reals.size();
  // active members (dt > 0) sorted by stage count, descending
  std::vector<int> order;
  for (int i = 0; i < nw; ++i)
    if (dt[i] > 0.0) order.push_back(i);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return s[a] > s[b]; });
  std::vector<Tile> tiles, atiles;
  std::vector<int> tile_end;
  std::vector<StepParam> sp(h->n_real);
  std::memset(sp.data(), 0, sp.size() * sizeof(StepParam));
  std::vector<Coef<T>> coefs;
  for (int i : order) {
    const int r = w.reals[i];
    const RealInfo& ri = h->reals[r];
    const ShapeInfo& sh = h->shapes[ri.shape];
    append_tiles(h, r, std::max(1, sh.tile_rows), 1, tiles);
    append_tiles(h, r, std::max(1, sh.tile_rows), kAdvRun, atiles);
    tile_end.push_back((int)tiles.size());
    StepParam& p = sp[r];
    p.dt = dt[i];
    p.dt_adv = h->strang ? 0.5 * dt[i] : dt[i];
    p.nudt = ri.nu * dt[i];
    p.eps_t = ri.fp.eps_w > 0.0 ? ri.fp.eps_w : sh.dth;
    p.eps_p = ri.fp.eps_w > 0.0 ? ri.fp.eps_w : sh.dph;
    p.alpha_uw = ri.fp.alpha_uw;
    p.s = s[i];
    p.weno = ri.fp.adv_space == SFT_ADV_WENO3_CSH ? 1 : 0;
    p.adv = ri.fp.advection ? 1 : 0;
    p.inv_b0 = ri.fp.atten_b0 > 0.0 ? 1.0 / ri.fp.atten_b0 : 0.0;
    p.cap_nu = ri.cap_nu;
    p.coef = (int)coefs.size();
    if (s[i] > 0 && ri.fp.diffusion == SFT_DIFF_RKG2) rkg2_coefs<T>(s[i], coefs);
    else if (s[i] > 0) rkl2_coefs<T>(s[i], coefs);
    else coefs.push_back(Coef<T>{});
    const double cells = (double)sh.nt * sh.np;
    if (ri.fp.advection) c->cells_adv += cells;
    c->cell_stages_diff += cells * s[i];
    if (s[i] > 0) c->diff_words += cells * (4.0 * s[i] - 1.0);
    c->cell_updates += cells;
    c->smax = std::max(c->smax, s[i]);
  }
  c->realization_steps = (int)order.size();
  c->fused = h->fused;
  std::vector<Tile> ft;  // fused-pass tiles
  if (c->fused) {
    // fused passes start at stages 2, 2+K, 2+2K, ...; stage 1 uses the
    // single-stage kernel (it forms G = dt L(Y_0)).
    // more chains pay off only when a pass fills the GPU several times over
    // (their launches overlap the other chains' shrinking tails as the
    // members with fewer stages finish); small batches keep one chain.  Six
    // chains for large grids, two for small ones: measured on GB300, 64 x
    // 1024x2048 (2 M cells a realization) runs 57.9 / 56.3 / 56.2 ms per
    // step with 2 / 4 / 6 chains, 512 x 256x512 (131 K) 9250 / 9020 / 8880
    // member-days/s.
    size_t pass_tiles = 0;
    double pass_cells = 0.0;
    {
      std::vector<Tile> tmp;
      for (int i : order) {
        append_fused_interior(h, w.reals[i], tmp);
        const ShapeInfo& sh = h->shapes[h->reals[w.reals[i]].shape];
        pass_cells += (double)sh.nt * sh.np;
      }
      pass_tiles = tmp.size();
    }
    const int want = pass_cells >= (double)(1 << 20) * (double)order.size() ? kMaxChains : 2;
    c->n_chains = pass_tiles >= (size_t)4 * h->n_sm ? std::min<int>(want, (int)order.size()) : 1;
    for (int ch = 0; ch < c->n_chains; ++ch) {
      c->fbase[ch] = (int)ft.size();
      std::vector<int> mem, fend;  // chain members (descending s) and their interior tile ends
      for (size_t q = ch; q < order.size(); q += c->n_chains) mem.push_back(order[q]);
      for (int i : mem) append_fused_poles(w.reals[i], ft);
      c->fcaps[ch] = (int)ft.size() - c->fbase[ch];
      for (int i : mem) {
        append_fused_interior(h, w.reals[i], ft);
        fend.push_back((int)ft.size() - c->fbase[ch] - c->fcaps[ch]);
      }
      c->fused_tiles[ch].assign(c->smax + 1, 0);
      c->fused_caps[ch].assign(c->smax + 1, 0);
      for (int j0 = 2; j0 <= c->smax; j0 += fused::K) {
        int n = 0;
        while (n < (int)mem.size() && s[mem[n]] >= j0) ++n;
        c->fused_caps[ch][j0] = 2 * n;
        c->fused_tiles[ch][j0] = n == 0 ? 0 : fend[n - 1];
        if (n > 0) c->fused_launches += 1;
      }
    }
    c->diff_words = 0.0;
    for (int i : order) {
      const ShapeInfo& sh = h->shapes[h->reals[w.reals[i]].shape];
      if (s[i] > 0) c->diff_words += (double)sh.nt * sh.np * (3.0 + 5.0 * ((s[i] - 1 + fused::K - 1) / fused::K));
    }
    const std::string bad = check_tiles(h, ft, true);
    if (!bad.empty()) return fail(h, SFT_ERR_STATE, "internal table check: " + bad);
  }
  c->n_adv_tiles = (int)atiles.size();
  c->stage_tiles.assign(c->smax + 1, 0);
  for (int j = 1; j <= c->smax; ++j) {
    int n = 0;
    while (n < (int)order.size() && s[order[n]] >= j) ++n;
    c->stage_tiles[j] = n == 0 ? 0 : tile_end[n - 1];
  }
  {
    std::string bad = check_tiles(h, tiles, false);
    if (bad.empty()) bad = check_tiles(h, atiles, false);
    if (!bad.empty()) return fail(h, SFT_ERR_STATE, "internal table check: " + bad);
  }
  if (coefs.empty()) coefs.push_back(Coef<T>{});
  {
    // all tables in one device allocation, uploaded by one copy from a pinned
    // staging buffer (a handful of allocations and pageable copies per new
    // configuration cost more host time than the step's launches)
    size_t total = 0;
    auto place = [&total](size_t bytes) {
      const size_t o = total;
      total += (bytes + 255) & ~(size_t)255;
      return o;
    };
    const size_t o_ft = place(ft.size() * sizeof(Tile)), o_at = place(atiles.size() * sizeof(Tile));
    const size_t o_ti = place(tiles.size() * sizeof(Tile)), o_sp = place(sp.size() * sizeof(StepParam));
    const size_t o_cf = place(coefs.size() * sizeof(Coef<T>));
    const int slot = h->cfg_stage_next;
    h->cfg_stage_next = (slot + 1) % kStageRing;
    if (h->cfg_stage_pending[slot]) {  // the upload that last read this buffer
      SFT_CUDA(h, cudaEventSynchronize(h->cfg_stage_ev[slot]));
      h->cfg_stage_pending[slot] = false;
    }
    if (h->cfg_stage_bytes[slot] < total) {
      const size_t want = std::max<size_t>(total, 2 * h->cfg_stage_bytes[slot]);
      if (h->cfg_stage[slot]) cudaFreeHost(h->cfg_stage[slot]);
      h->cfg_stage[slot] = nullptr;
      h->cfg_stage_bytes[slot] = 0;
      SFT_CUDA(h, host_malloc(&h->cfg_stage[slot], want));
      h->cfg_stage_bytes[slot] = want;
    }
    char* st = h->cfg_stage[slot];
    if (!ft.empty()) std::memcpy(st + o_ft, ft.data(), ft.size() * sizeof(Tile));
    if (!atiles.empty()) std::memcpy(st + o_at, atiles.data(), atiles.size() * sizeof(Tile));
    if (!tiles.empty()) std::memcpy(st + o_ti, tiles.data(), tiles.size() * sizeof(Tile));
    std::memcpy(st + o_sp, sp.data(), sp.size() * sizeof(StepParam));
    std::memcpy(st + o_cf, coefs.data(), coefs.size() * sizeof(Coef<T>));
    SFT_CUDA(h, dev_malloc_async(&c->d_blob, total, h->stream));
    char* b = static_cast<char*>(c->d_blob);
    SFT_CUDA(h, cudaMemcpyAsync(b, st, total, cudaMemcpyHostToDevice, h->stream));
    SFT_CUDA(h, cudaEventRecord(h->cfg_stage_ev[slot], h->stream));
    h->cfg_stage_pending[slot] = true;
    c->d_ftiles = ft.empty() ? nullptr : reinterpret_cast<Tile*>(b + o_ft);
    c->d_atiles = atiles.empty() ? nullptr : reinterpret_cast<Tile*>(b + o_at);
    c->d_tiles = tiles.empty() ? nullptr : reinterpret_cast<Tile*>(b + o_ti);
    c->d_sp = reinterpret_cast<StepParam*>(b + o_sp);
    c->d_coef = b + o_cf;
  }
  // keep at most kMaxConfigs configurations per wave
  if ((int)w.configs.size() >= kMaxConfigs) {
    auto it = std::min_element(w.configs.begin(), w.configs.end(),
                               [](const std::unique_ptr<Config>& a, const std::unique_ptr<Config>& b) {
                                 return a->last_use < b->last_use;
                               });
    free_config(**it, h->stream);
    w.configs.erase(it);
  }
  release.c = nullptr;
  *out = c.get();
  w.configs.push_back(std::move(c));
  return SFT_OK;
}

// The launches of one step (advection stages, then RKL2 stages).
// Record a profiling event; under stream capture it must be an external
// event node (a plain record would only mark a capture dependency).
cudaError_t record(cudaEvent_t e, cudaStream_t st, bool capturing) {
  return capturing ? cudaEventRecordWithFlags(e, st, cudaEventRecordExternal) : cudaEventRecord(e, st);
}

// One advection advance (the SSPRK / FE stages) of every realization, by
// StepParam::dt_adv.
template <typename T>
sft_status enqueue_adv(sft_handle h, Config& c, cudaStream_t st) {
  if (c.n_adv_tiles <= 0) return SFT_OK;
  T* B = ptr<T>(h->state);
  T* W0 = ptr<T>(h->work[0]);
  T* W1 = ptr<T>(h->work[1]);
  const auto* geo = ptr<const RowGeo<T>>(h->d_geo);
  const auto* flow = ptr<const RowFlow<T>>(h->d_flow);
  const int adv_time = h->reals.empty() ? SFT_TIME_SSPRK43 : h->reals[0].fp.adv_time;
  std::vector<AdvStage<T>> stages;
  auto S = [&](const T* fin, int finw, const T* fn, int fnw, T* out, int outw, double a, double b, double cc) {
    stages.push_back(AdvStage<T>{fin, fn, out, finw, fnw, outw, T(a), T(b), T(cc)});
  };
  if (adv_time == SFT_TIME_SSPRK43) {
    S(B, 0, nullptr, 0, W0, 1, 0.0, 1.0, 0.5);
    S(W0, 1, nullptr, 0, W1, 1, 0.0, 1.0, 0.5);
    S(W1, 1, B, 0, W0, 1, 2.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0);
    S(W0, 1, nullptr, 0, B, 0, 0.0, 1.0, 0.5);
  } else if (adv_time == SFT_TIME_SSPRK33) {
    S(B, 0, nullptr, 0, W0, 1, 0.0, 1.0, 1.0);
    S(W0, 1, B, 0, W1, 1, 0.75, 0.25, 0.25);
    S(W1, 1, B, 0, B, 0, 1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0);
  } else {
    S(B, 0, nullptr, 0, W0, 1, 0.0, 1.0, 1.0);
    S(W0, 1, nullptr, 0, B, 0, 0.0, 1.0, 0.0);  // copy back
  }
  for (auto& s : stages) {
    SFT_CUDA(h, launch_adv_stage<T>(c.n_adv_tiles, st, c.d_atiles, h->d_desc, c.d_sp, geo, flow, h->d_shc, B, W0,
                                    W1, s));
  }
  return SFT_OK;
}

// The launches of one step: advection, then the RKL2 stages (Lie); with
// Strang splitting a second advection advance follows (each by dt/2).
template <typename T>
sft_status enqueue_step(sft_handle h, Config& c, bool record_events, bool capturing) {
  const cudaStream_t st = h->stream;
  T* B = ptr<T>(h->state);
  T* W0 = ptr<T>(h->work[0]);
  T* W1 = ptr<T>(h->work[1]);
  T* W2 = ptr<T>(h->work[2]);
  const auto* geo = ptr<const RowGeo<T>>(h->d_geo);
  if (h->any_rfe) {  // the step's source maps: Eq. (fluxbal) factors, then the first application
    SFT_CUDA(h, launch_rfe_sums<T>(h->n_rtiles, st, h->d_rtiles, h->d_desc, h->d_geod, h->d_rfe, h->d_partials));
    SFT_CUDA(h, launch_rfe_fold(h->n_real, st, h->d_rstart, h->d_rfe, h->d_partials, h->d_rfe_fac));
    if (h->strang)
      SFT_CUDA(h, launch_rfe_apply<T>(h->n_rtiles, st, h->d_rtiles, h->d_desc, h->d_geod, h->d_rfe, h->d_rfe_fac, 0,
                                      B));
  }
  if (record_events) SFT_CUDA(h, record(h->ev[0], st, capturing));
  {
    sft_status sa = enqueue_adv<T>(h, c, st);
    if (sa != SFT_OK) return sa;
  }
  if (record_events) {
    SFT_CUDA(h, record(h->ev[1], st, capturing));
    SFT_CUDA(h, record(h->ev[2], st, capturing));
  }
  if (c.fused && c.smax >= 1) {
    // stage 1 (forms G and delta_1 = W2), then passes of K stages that
    // alternate between the increment pairs (W1, W2) and (W3, W4)
    SFT_CUDA(h, launch_rkl2_stage<T>(c.stage_tiles[1], st, c.d_tiles, h->d_desc, c.d_sp, geo,
                                     h->d_shc, ptr<const Coef<T>>(c.d_coef), B, W0, W1, W2, 1, 1,
                                     h->d_status));
    float* P[4] = {ptr<float>(h->work[1]), ptr<float>(h->work[2]), ptr<float>(h->work[3]),
                   ptr<float>(h->work[4])};
    // ring sums next to the poles of delta_1 and G for the first fused launch
    for (int ch = 0; ch < c.n_chains; ++ch)
      SFT_CUDA(h, launch_ring_sums(c.fused_caps[ch].size() > 2 ? c.fused_caps[ch][2] : 0, st,
                                   c.d_ftiles + c.fbase[ch], h->d_desc, P[1], ptr<const float>(h->work[0]),
                                   ptr<double>(h->polar)));
    if (c.n_chains > 1) {  // fork: the side chains start after stage 1
      SFT_CUDA(h, cudaEventRecord(h->fork, st));
      for (int ch = 1; ch < c.n_chains; ++ch) SFT_CUDA(h, cudaStreamWaitEvent(h->side[ch], h->fork, 0));
    }
    for (int ch = 0; ch < c.n_chains; ++ch) {
      const cudaStream_t cs = ch == 0 ? st : h->side[ch];
      int in = 0;  // input pair (P[in], P[in+1]) = (delta_{j0-2}, delta_{j0-1})
      for (int j0 = 2; j0 <= c.smax; j0 += fused::K) {
        const int out = 2 - in;
        SFT_CUDA(h, launch_rkl2_fused(c.fused_tiles[ch][j0], cs, c.d_ftiles + c.fbase[ch] + c.fcaps[ch],
                                      h->d_desc, c.d_sp, ptr<const RowGeo<float>>(h->d_geo), h->d_shc,
                                      ptr<const Coef<float>>(c.d_coef), ptr<float>(h->state),
                                      ptr<const float>(h->work[0]), P[in], P[in + 1], P[out], P[out + 1],
                                      ptr<double>(h->polar), in / 2, j0, h->d_status));
        in = out;
      }
    }
    for (int ch = 1; ch < c.n_chains; ++ch) {  // join
      SFT_CUDA(h, cudaEventRecord(h->join[ch], h->side[ch]));
      SFT_CUDA(h, cudaStreamWaitEvent(st, h->join[ch], 0));
    }
  } else {
    for (int j = 1; j <= c.smax; ++j) {
      SFT_CUDA(h, launch_rkl2_stage<T>(c.stage_tiles[j], st, c.d_tiles, h->d_desc, c.d_sp, geo,
                                       h->d_shc, ptr<const Coef<T>>(c.d_coef), B, W0, W1, W2, j, 1,
                                       h->d_status));
    }
  }
  if (record_events) SFT_CUDA(h, record(h->ev[3], st, capturing));
  if (h->strang) {
    if (record_events) SFT_CUDA(h, record(h->ev[4], st, capturing));
    sft_status sa = enqueue_adv<T>(h, c, st);
    if (sa != SFT_OK) return sa;
    if (record_events) SFT_CUDA(h, record(h->ev[5], st, capturing));
  }
  if (h->any_rfe)  // Lie: the source after D; Strang: its second half
    SFT_CUDA(h, launch_rfe_apply<T>(h->n_rtiles, st, h->d_rtiles, h->d_desc, h->d_geod, h->d_rfe, h->d_rfe_fac,
                                    h->strang ? 1 : 0, B));
  return SFT_OK;
}

int adv_stage_count(sft_handle h) {
  if (h->reals.empty()) return 0;
  switch (h->reals[0].fp.adv_time) {
    case SFT_TIME_SSPRK43: return 4;
    case SFT_TIME_SSPRK33: return 3;
    default: return 2;
  }
}

template <typename T>
sft_status autotune(sft_handle h, Wave& w, const std::vector<int>& active);

template <typename T>
sft_status run_step(sft_handle h, Wave& w, double t_target, bool* any) {
  const int nw = (int)w.reals.size();
  std::vector<double> dt(nw, 0.0);
  std::vector<int> s(nw, 0);
  *any = false;
  for (int i = 0; i < nw; ++i) {
    const RealInfo& ri = h->reals[w.reals[i]];
    const double rem = t_target - ri.t;
    if (!(rem > 0.0)) continue;
    // Sec. 3.4: the remaining time, cut to the flow limit
    double lim = h->strang ? 2.0 * ri.dt_cfl : ri.dt_cfl;  // Strang: two dt/2 advances
    if (ri.rfe.method != 0 && ri.rfe.rate_mx_per_hour > 0.0 && std::isfinite(ri.rfe.lifetime_hours) &&
        ri.rfe.lifetime_hours > 0.0)
      lim = std::min(lim, ri.rfe.lifetime_hours);  // a step spans at most two source segments
    dt[i] = rem <= lim ? rem : lim;
    s[i] = sts_stages(ri.fp.diffusion, dt[i], ri.dt_euler);
    *any = true;
  }
  if (!*any) return SFT_OK;
  for (int r : w.reals) {
    const ShapeInfo& sh = h->shapes[h->reals[r].shape];
    if (sh.tile_rows == 0 || (h->fused && sh.band_rows == 0)) {
      std::vector<int> active;  // realizations this step advances: the batch the choice serves
      for (int i = 0; i < nw; ++i)
        if (dt[i] > 0.0) active.push_back(w.reals[i]);
      sft_status st = autotune<T>(h, w, active);
      if (st != SFT_OK) return st;
      break;
    }
  }
  Config* c = nullptr;
  for (auto& cfg : w.configs) {
    bool same = cfg->dt == dt && cfg->s == s && cfg->fused == h->fused;
    for (size_t i = 0; same && i < h->shapes.size(); ++i)
      same = cfg->tr[i] == h->shapes[i].tile_rows && cfg->band[i] == h->shapes[i].band_rows;
    if (same) {
      c = cfg.get();
      break;
    }
  }
  if (!c) {
    sft_status st = build_config<T>(h, w, dt, s, &c);
    if (st != SFT_OK) return st;
  }
  c->last_use = ++h->use_counter;
  // map windows whose balance factors this step computes (recorded once the
  // step's launches are enqueued: a step that fails leaves them unclaimed)
  std::vector<std::pair<int, int64_t>> rfe_fresh;
  if (h->any_rfe) {  // this step's source maps and weights (read by the step's kernels)
    std::vector<RfeStep> rs(h->n_real);
    std::memset(rs.data(), 0, rs.size() * sizeof(RfeStep));
    for (int i = 0; i < nw; ++i) {
      const int r = w.reals[i];
      const RealInfo& ri = h->reals[r];
      if (!(dt[i] > 0.0) || ri.rfe.method == 0 || !(ri.rfe.rate_mx_per_hour > 0.0)) continue;
      RfeStep& q = rs[r];
      const ShapeInfo& sh = h->shapes[ri.shape];
      const double ncell = (double)(sh.nt - 2) * sh.np + 2.0, r2 = kRsunCm * kRsunCm;
      q.method = ri.rfe.method;
      q.seed = ri.rfe.seed;
      q.c = ri.rfe.rate_mx_per_hour * std::sqrt(0.5 * kPi) / (ri.rfe.method == 1 ? r2 * ncell : 4.0 * kPi * r2);
      const double tau = ri.rfe.lifetime_hours, t = ri.t;
      double wa[4], wb[4];
      if (h->strang) {
        const int64_t ma = rfe_weights(ri.rfe_t0, tau, t, t + 0.5 * dt[i], wa);
        const int64_t mb = rfe_weights(ri.rfe_t0, tau, t + 0.5 * dt[i], t + dt[i], wb);
        q.m0 = std::min(ma, mb);
        for (int k = 0; k < 4; ++k) {
          if (k + ma - q.m0 < 4) q.wa[k + ma - q.m0] = wa[k];
          if (k + mb - q.m0 < 4) q.wb[k + mb - q.m0] = wb[k];
        }
      } else {
        q.m0 = rfe_weights(ri.rfe_t0, tau, t, t + dt[i], wa);
        for (int k = 0; k < 4; ++k) q.wa[k] = wa[k];
      }
      q.fresh = ri.rfe_m0 != q.m0 ? 1 : 0;  // the factors of a kept window stay valid
      rfe_fresh.emplace_back(r, q.m0);
    }
    SFT_CUDA(h, cudaMemcpyAsync(h->d_rfe, rs.data(), rs.size() * sizeof(RfeStep), cudaMemcpyHostToDevice,
                                h->stream));
  }
  c->uses += 1;
  const bool ev = h->profiling;
  // A configuration used once (a shortened last step, a one-off member
  // subset) launches eagerly; capture and instantiation pay off from its
  // second use on.
  if (h->use_graphs && c->uses >= 2) {
    if (!c->exec) {
      cudaGraph_t g = nullptr;
      SFT_CUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
      sft_status st = enqueue_step<T>(h, *c, true, true);
      cudaError_t e = cudaStreamEndCapture(h->stream, &g);
      if (st != SFT_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      if (e != cudaSuccess) return fail(h, SFT_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
      e = cudaGraphInstantiate(&c->exec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return fail(h, SFT_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    SFT_CUDA(h, cudaGraphLaunch(c->exec, h->stream));
    h->stats.graph_launches += 1;
  } else {
    sft_status st = enqueue_step<T>(h, *c, ev, false);
    if (st != SFT_OK) return st;
  }
  for (auto& f : rfe_fresh) h->reals[f.first].rfe_m0 = f.second;
  const int n_adv = (c->n_adv_tiles > 0 ? adv_stage_count(h) : 0) * (h->strang ? 2 : 1);
  // RKL2 passes (one fused pass = K stages, over both chains) and launches
  const int n_diff = c->fused ? (c->smax >= 1 ? 1 + (c->smax - 1 + fused::K - 1) / fused::K : 0) : c->smax;
  const int64_t n_diff_launches =
      c->fused ? (c->smax >= 1 ? 1 + (c->smax >= 2 ? c->n_chains : 0) + c->fused_launches : 0) : c->smax;
  h->stats.kernel_launches += n_adv + n_diff_launches;
  h->stats.realization_steps += c->realization_steps;
  h->stats.cell_updates += c->cell_updates;
  h->stats.adv_cell_stages +=
      c->cells_adv * (adv_stage_count(h) == 2 ? 1 : adv_stage_count(h)) * (h->strang ? 2 : 1);
  (void)0;
  h->stats.diff_cell_stages += c->cell_stages_diff;
  if (ev) {
    SFT_CUDA(h, cudaEventSynchronize(h->ev[h->strang ? 5 : 3]));
    float a = 0.f, d = 0.f;
    SFT_CUDA(h, cudaEventElapsedTime(&a, h->ev[0], h->ev[1]));
    SFT_CUDA(h, cudaEventElapsedTime(&d, h->ev[2], h->ev[3]));
    if (h->strang) {
      float a2 = 0.f;
      SFT_CUDA(h, cudaEventElapsedTime(&a2, h->ev[4], h->ev[5]));
      a += a2;
    }
    h->stats.adv_ms += a;
    h->stats.diff_ms += d;
    h->stats.adv_launches += n_adv;
    h->stats.diff_launches += n_diff;
    const double eb = (double)h->elem;
    // Algorithmic bytes.  RKL2: stage 1 reads B, writes G and delta_1 (3
    // words); stage 2 reads delta_1, G, writes delta_2 (3); middle stages
    // read delta_{j-1}, delta_{j-2}, G and write delta_j (4); the last reads
    // delta_{s-1}, delta_{s-2}, G, B and writes B (5): 4s - 1 words per cell.
    // SSPRK(4,3): 2 + 2 + 3 + 2 = 9 words; SSPRK(3,3): 2 + 3 + 3 = 8; FE + copy: 4.
    h->stats.diff_bytes += eb * c->diff_words;
    const int na = adv_stage_count(h);
    h->stats.adv_bytes += (na == 4 ? 9.0 : (na == 3 ? 8.0 : 4.0)) * eb * c->cells_adv * (h->strang ? 2 : 1);
  }
  for (int i = 0; i < nw; ++i) {
    if (!(dt[i] > 0.0)) continue;
    RealInfo& ri = h->reals[w.reals[i]];
    const double rem = t_target - ri.t;
    ri.t = dt[i] == rem ? t_target : ri.t + dt[i];
    ri.steps += 1;
  }
  return SFT_OK;
}

// Pick the tile height of the stage kernels per shape by timing RKL2 stage 2
// (a non-final stage: it writes only work arrays) for each candidate.
// Band rows of shape si for the fused RKL2 kernel, and the descriptors of
// its realizations (uploaded when no step is in flight).
sft_status set_band(sft_handle h, int si, int band) {
  h->shapes[si].band_rows = band;
  for (int r = 0; r < h->n_real; ++r)
    if (h->reals[r].shape == si) h->desc[r].band = band;
  SFT_CUDA(h, cudaStreamSynchronize(h->stream));
  SFT_CUDA(h, cudaMemcpy(h->d_desc, h->desc.data(), h->desc.size() * sizeof(RealDesc), cudaMemcpyHostToDevice));
  return SFT_OK;
}

// The fused kernel's band rows for shape si: one launch of eight stages
// (stages 10..17 of a 30-stage super step, so that no launch is final and
// only work arrays are written) over the realizations of that shape that the
// step being planned advances (up to 1024: the batch the choice serves),
// timed for each candidate (64, 128, 256, 512 rows; those above 128 no
// wider than twice the interior), two rounds keeping each candidate's
// faster time.  Short bands pay more halo rows but give a small batch more,
// shorter work items (the march of one band is serial).
// Results do not depend on the choice (every band computes the same stages
// point for point); the work arrays and ring-sum partials it overwrites are
// rebuilt by every step before they are read.
sft_status tune_band(sft_handle h, const std::vector<int>& active, int si) {
  ShapeInfo& sh = h->shapes[si];
  std::vector<int> members;  // the shape's realizations in the step being planned (at most 1024)
  for (int r : active)
    if (h->reals[r].shape == si && members.size() < 1024) members.push_back(r);
  if (members.empty()) return SFT_OK;
  const int S = 30, J0 = 10;
  std::vector<StepParam> sp(h->n_real);
  std::memset(sp.data(), 0, sp.size() * sizeof(StepParam));
  for (int r : members) {
    sp[r].dt = 1.0;
    sp[r].nudt = 1e-6;
    sp[r].s = S;
    sp[r].coef = 0;
    sp[r].cap_nu = 1.0;
  }
  std::vector<Coef<float>> coefs;
  rkl2_coefs<float>(S, coefs);
  StepParam* d_sp = nullptr;
  Coef<float>* d_coef = nullptr;
  Tile* d_tiles = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int best = fused::default_band_rows(sh.nt);
  float best_ms = 1e30f;
  cudaError_t err = dev_malloc(&d_sp, sp.size() * sizeof(StepParam));
  if (err == cudaSuccess) err = dev_malloc(&d_coef, coefs.size() * sizeof(Coef<float>));
  if (err == cudaSuccess) err = cudaMemcpy(d_sp, sp.data(), sp.size() * sizeof(StepParam), cudaMemcpyHostToDevice);
  if (err == cudaSuccess)
    err = cudaMemcpy(d_coef, coefs.data(), coefs.size() * sizeof(Coef<float>), cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  constexpr int kCand = 4;
  const int cand[kCand] = {64, 128, 256, 512};
  float* P[4] = {ptr<float>(h->work[1]), ptr<float>(h->work[2]), ptr<float>(h->work[3]), ptr<float>(h->work[4])};
  for (int ci = 0; ci < 2 * kCand && err == cudaSuccess; ++ci) {
    const int band = cand[ci % kCand];
    if (band > 128 && band >= 2 * (sh.nt - 2)) continue;
    sft_status st = set_band(h, si, band);
    if (st != SFT_OK) {
      err = cudaErrorUnknown;
      break;
    }
    std::vector<Tile> tiles;
    for (int r : members) append_fused_interior(h, r, tiles);
    cudaFree(d_tiles);
    d_tiles = nullptr;
    if (!check_tiles(h, tiles, true).empty()) {
      err = cudaErrorInvalidValue;
      break;
    }
    err = dev_malloc(&d_tiles, tiles.size() * sizeof(Tile));
    if (err == cudaSuccess) err = cudaMemcpy(d_tiles, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice);
    const int nt = (int)tiles.size();
    auto launch = [&]() {
      return launch_rkl2_fused(nt, h->stream, d_tiles, h->d_desc, d_sp, ptr<const RowGeo<float>>(h->d_geo),
                               h->d_shc, d_coef, ptr<float>(h->state), ptr<const float>(h->work[0]), P[0], P[1],
                               P[2], P[3], ptr<double>(h->polar), 0, J0, h->d_status);
    };
    if (err == cudaSuccess) err = launch();
    if (err == cudaSuccess) err = cudaEventRecord(e0, h->stream);
    for (int it = 0; it < 3 && err == cudaSuccess; ++it) err = launch();
    if (err == cudaSuccess) err = cudaEventRecord(e1, h->stream);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess && ms < best_ms) {
      best_ms = ms;
      best = band;
    }
  }
  cudaFree(d_tiles);
  cudaFree(d_sp);
  cudaFree(d_coef);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (err != cudaSuccess)
    return fail(h, err == cudaErrorMemoryAllocation ? SFT_ERR_OOM : SFT_ERR_CUDA,
                std::string("band autotune: ") + cudaGetErrorString(err));
  return set_band(h, si, best);
}

template <typename T>
sft_status autotune(sft_handle h, Wave& w, const std::vector<int>& active) {
  for (size_t si = 0; si < h->shapes.size(); ++si) {
    ShapeInfo& sh = h->shapes[si];
    if constexpr (std::is_same<T, float>::value) {
      if (h->fused && sh.band_rows == 0) {
        sft_status st = tune_band(h, active, (int)si);
        if (st != SFT_OK) return st;
      }
    }
    if (sh.tile_rows != 0) continue;
    std::vector<int> members;
    for (int r : w.reals)
      if (h->reals[r].shape == (int)si && members.size() < 8) members.push_back(r);
    if (members.empty()) continue;
    std::vector<StepParam> sp(h->n_real);
    std::memset(sp.data(), 0, sp.size() * sizeof(StepParam));
    for (int r : members) {
      sp[r].dt = 1.0;
      sp[r].nudt = 1e-6;
      sp[r].s = 3;
      sp[r].coef = 0;
    }
    std::vector<Coef<T>> coefs;
    rkl2_coefs<T>(3, coefs);
    StepParam* d_sp = nullptr;
    Coef<T>* d_coef = nullptr;
    Tile* d_tiles = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int best = 8;
    float best_ms = 1e30f;
    cudaError_t err = cudaSuccess;
    err = dev_malloc(&d_sp, sp.size() * sizeof(StepParam));
    if (err == cudaSuccess) err = dev_malloc(&d_coef, coefs.size() * sizeof(Coef<T>));
    if (err == cudaSuccess) err = cudaMemcpy(d_sp, sp.data(), sp.size() * sizeof(StepParam), cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(d_coef, coefs.data(), coefs.size() * sizeof(Coef<T>), cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    // candidates whose tile rows would leave half the threads past the row
    // end are skipped (8 rows per tile always runs); two rounds over the
    // candidates, each keeping its faster time, damp timing noise
    const int cand[4] = {1, 2, 4, 8};
    for (int ci = 0; ci < 8 && err == cudaSuccess; ++ci) {
      const int tr = cand[ci % 4];
      if (tr != 8 && (kThreads / tr) * vec_width(h) >= 2 * sh.np) continue;
      std::vector<Tile> tiles;
      for (int r : members) append_tiles(h, r, tr, 1, tiles);
      cudaFree(d_tiles);
      d_tiles = nullptr;
      if (!check_tiles(h, tiles, false).empty()) {
        err = cudaErrorInvalidValue;
        break;
      }
      err = dev_malloc(&d_tiles, tiles.size() * sizeof(Tile));
      if (err != cudaSuccess) break;
      err = cudaMemcpy(d_tiles, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice);
      if (err != cudaSuccess) break;
      const int nt = (int)tiles.size();
      const auto* geo = ptr<const RowGeo<T>>(h->d_geo);
      T* B = ptr<T>(h->state);
      T* W0 = ptr<T>(h->work[0]);
      T* W1 = ptr<T>(h->work[1]);
      T* W2 = ptr<T>(h->work[2]);
      err = launch_rkl2_stage<T>(nt, h->stream, d_tiles, h->d_desc, d_sp, geo, h->d_shc, d_coef, B,
                                 W0, W1, W2, 1, 0, h->d_status);
      for (int it = 0; it < 2 && err == cudaSuccess; ++it)
        err = launch_rkl2_stage<T>(nt, h->stream, d_tiles, h->d_desc, d_sp, geo, h->d_shc, d_coef,
                                   B, W0, W1, W2, 2, 0, h->d_status);
      if (err == cudaSuccess) err = cudaEventRecord(e0, h->stream);
      const int reps = 6;
      for (int it = 0; it < reps && err == cudaSuccess; ++it)
        err = launch_rkl2_stage<T>(nt, h->stream, d_tiles, h->d_desc, d_sp, geo, h->d_shc, d_coef,
                                   B, W0, W1, W2, 2, 0, h->d_status);
      if (err == cudaSuccess) err = cudaEventRecord(e1, h->stream);
      if (err == cudaSuccess) err = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
      if (err == cudaSuccess && ms < best_ms) {
        best_ms = ms;
        best = tr;
      }
    }
    cudaFree(d_tiles);
    cudaFree(d_sp);
    cudaFree(d_coef);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (err != cudaSuccess)
      return fail(h, err == cudaErrorMemoryAllocation ? SFT_ERR_OOM : SFT_ERR_CUDA,
                  std::string("autotune: ") + cudaGetErrorString(err));
    sh.tile_rows = best;
  }
  return SFT_OK;
}

template <typename T>
sft_status upload_tables(sft_handle h) {
  std::vector<RowGeo<T>> g;
  std::vector<RowGeoD> gd;
  std::vector<ShapeConst> sc;
  std::vector<double> cp, sp;
  for (auto& s : h->shapes) {
    s.geo = (int)g.size();
    geo_rows<T>(s, g, gd);
    s.col = (int)cp.size();
    for (int k = 0; k < s.np; ++k) {
      cp.push_back(std::cos(k * s.dph));
      sp.push_back(std::sin(k * s.dph));
    }
    const double line = std::sin(0.5 * s.dth) * s.dph;
    sc.push_back(ShapeConst{line / (s.dth * s.cap), line / s.cap, s.dth, s.dph});
  }
  h->geo_rows = (int)g.size();
  h->col_entries = (int)cp.size();
  SFT_CUDA(h, dev_malloc(&h->d_geo, g.size() * sizeof(RowGeo<T>)));
  SFT_CUDA(h, cudaMemcpy(h->d_geo, g.data(), g.size() * sizeof(RowGeo<T>), cudaMemcpyHostToDevice));
  SFT_CUDA(h, dev_malloc(&h->d_geod, gd.size() * sizeof(RowGeoD)));
  SFT_CUDA(h, cudaMemcpy(h->d_geod, gd.data(), gd.size() * sizeof(RowGeoD), cudaMemcpyHostToDevice));
  SFT_CUDA(h, dev_malloc(&h->d_cosp, cp.size() * sizeof(double)));
  SFT_CUDA(h, cudaMemcpy(h->d_cosp, cp.data(), cp.size() * sizeof(double), cudaMemcpyHostToDevice));
  SFT_CUDA(h, dev_malloc(&h->d_sinp, sp.size() * sizeof(double)));
  SFT_CUDA(h, cudaMemcpy(h->d_sinp, sp.data(), sp.size() * sizeof(double), cudaMemcpyHostToDevice));
  {
    std::vector<float4> cf(cp.size());
    for (size_t i = 0; i < cp.size(); ++i) {
      const float ch = (float)cp[i], sh = (float)sp[i];
      cf[i] = make_float4(ch, (float)(cp[i] - (double)ch), sh, (float)(sp[i] - (double)sh));
    }
    SFT_CUDA(h, dev_malloc(&h->d_csf, cf.size() * sizeof(float4)));
    SFT_CUDA(h, cudaMemcpy(h->d_csf, cf.data(), cf.size() * sizeof(float4), cudaMemcpyHostToDevice));
  }
  SFT_CUDA(h, dev_malloc(&h->d_shc, sc.size() * sizeof(ShapeConst)));
  SFT_CUDA(h, cudaMemcpy(h->d_shc, sc.data(), sc.size() * sizeof(ShapeConst), cudaMemcpyHostToDevice));
  // flow tables: one block of nt rows per realization (filled by sft_set_flows)
  int rows = 0;
  for (auto& r : h->reals) {
    r.flow_row = rows;
    rows += h->shapes[r.shape].nt;
  }
  h->flow_rows = rows;
  SFT_CUDA(h, dev_malloc(&h->d_flow, (size_t)rows * sizeof(RowFlow<T>)));
  SFT_CUDA(h, cudaMemset(h->d_flow, 0, (size_t)rows * sizeof(RowFlow<T>)));
  return SFT_OK;
}

template <typename T>
sft_status set_flows_t(sft_handle h, const sft_flow_params* params) {
  std::vector<RowFlow<T>> rows(h->flow_rows);
  for (int r = 0; r < h->n_real; ++r) {
    RealInfo& ri = h->reals[r];
    const ShapeInfo& s = h->shapes[ri.shape];
    const sft_flow_params& p = params[r];
    const FlowRows f = flow_profiles(s, p);
    for (int j = 0; j < s.nt; ++j) {
      RowFlow<T> rf{};
      if (j >= 1 && j <= s.nt - 2) {
        rf.vdn = T(f.vt[j - 1]);
        rf.vup = T(f.vt[j]);
        double a = 0.0;
        for (int fi = std::max(j - 3, 0); fi <= std::min(j + 2, s.nt - 2); ++fi)
          a = std::max(a, std::fabs(f.vt[fi]));
        rf.alpha = T(a);
      }
      rf.vp = T(f.vp[j]);
      rows[ri.flow_row + j] = rf;
    }
    ri.fp = p;
    const bool grid_nu = p.nu_grid_alpha > 0.0;
    ri.nu = grid_nu ? 1.0 : p.nu * kKm2sToRs2Hr;  // grid-based nu lives in the geometry block
    ri.cap_nu = grid_nu ? grid_nu_face(s, p.nu_grid_alpha, 0) : 1.0;
    ri.dt_cfl = p.advection ? cfl_limit(s, f, p) : INFINITY;
    ri.dt_euler = p.diffusion == SFT_DIFF_OFF ? INFINITY
                  : (grid_nu ? euler_limit_grid(s, p.nu_grid_alpha) : euler_limit(s, ri.nu));
    ri.has_flows = true;
  }
  SFT_CUDA(h, cudaMemcpyAsync(h->d_flow, rows.data(), rows.size() * sizeof(RowFlow<T>),
                              cudaMemcpyHostToDevice, h->stream));
  // geometry: the shapes' blocks, then one block per grid-based-nu realization
  bool any_grid = false;
  for (int r = 0; r < h->n_real; ++r) any_grid = any_grid || params[r].nu_grid_alpha > 0.0;
  if (any_grid || h->geo_custom) {
    std::vector<RowGeo<T>> g;
    std::vector<RowGeoD> gd;
    for (auto& sh : h->shapes) {
      sh.geo = (int)g.size();
      geo_rows<T>(sh, g, gd);
    }
    std::vector<RealDesc> nd = h->desc;
    for (int r = 0; r < h->n_real; ++r) {
      const ShapeInfo& sh = h->shapes[h->reals[r].shape];
      if (params[r].nu_grid_alpha > 0.0) {
        nd[r].geo = (int)g.size();
        geo_rows_grid_nu<T>(sh, params[r].nu_grid_alpha, g, gd);
      } else {
        nd[r].geo = sh.geo;
      }
    }
    SFT_CUDA(h, cudaStreamSynchronize(h->stream));
    if ((int)g.size() != h->geo_rows) {
      // new tables first: a failed allocation leaves the old ones (and the
      // descriptors that index them) in place
      void* ng = nullptr;
      RowGeoD* ngd = nullptr;
      cudaError_t e = dev_malloc(&ng, g.size() * sizeof(RowGeo<T>));
      if (e == cudaSuccess) e = dev_malloc(&ngd, gd.size() * sizeof(RowGeoD));
      if (e != cudaSuccess) {
        cudaFree(ng);
        return fail(h, e == cudaErrorMemoryAllocation ? SFT_ERR_OOM : SFT_ERR_CUDA,
                    std::string("geometry tables: ") + cudaGetErrorString(e));
      }
      cudaFree(h->d_geo);
      cudaFree(h->d_geod);
      h->d_geo = ng;
      h->d_geod = ngd;
      h->geo_rows = (int)g.size();
    }
    h->desc = nd;
    {
      const std::string bad = check_desc(h);
      if (!bad.empty()) return fail(h, SFT_ERR_STATE, "internal table check: " + bad);
    }
    SFT_CUDA(h, cudaMemcpy(h->d_geo, g.data(), g.size() * sizeof(RowGeo<T>), cudaMemcpyHostToDevice));
    SFT_CUDA(h, cudaMemcpy(h->d_geod, gd.data(), gd.size() * sizeof(RowGeoD), cudaMemcpyHostToDevice));
    SFT_CUDA(h, cudaMemcpy(h->d_desc, h->desc.data(), h->desc.size() * sizeof(RealDesc), cudaMemcpyHostToDevice));
    h->geo_custom = any_grid;
  }
  SFT_CUDA(h, cudaStreamSynchronize(h->stream));
  return SFT_OK;
}

// reduction machinery
template <typename T>
sft_status reduce_fold(sft_handle h, int mode, double lat_cut, AssimArgs aa) {
  SFT_CUDA(h, launch_reduce<T>(mode, h->n_rtiles, h->stream, h->d_rtiles, h->d_desc, h->d_geod,
                               h->d_cosp, h->d_sinp, h->d_csf, ptr<const T>(h->state), lat_cut, aa,
                               h->d_partials));
  SFT_CUDA(h, launch_fold(mode, h->n_real, h->stream, h->d_rstart, h->d_partials, aa.wpar, h->d_red));
  return SFT_OK;
}

}  // namespace

namespace sft {
// Error text of calls without a handle (read by sft_last_error(NULL)).
void set_global_error(const std::string& msg) { g_create_error = msg; }
}  // namespace sft

// ===========================================================================
// C-ABI
// ===========================================================================
extern "C" {

int32_t sft_abi_version(void) { return SFT_ABI_VERSION; }

const char* sft_last_error(sft_handle h) { return h ? h->err.c_str() : g_create_error.c_str(); }

sft_status sft_create_grid(const sft_shape* shapes, int32_t n_real, sft_prec prec,
                           size_t hbm_budget_bytes, void* cuda_stream, sft_handle* out) {
  if (!out) return fail(nullptr, SFT_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!shapes || n_real <= 0) return fail(nullptr, SFT_ERR_ARG, "need n_real > 0 shapes");
  if (prec != SFT_FP32 && prec != SFT_FP64) return fail(nullptr, SFT_ERR_ARG, "bad precision");
  for (int r = 0; r < n_real; ++r)
    if (shapes[r].ntheta < 5 || shapes[r].nphi < 8 || shapes[r].ntheta > (1 << 20) ||
        shapes[r].nphi > (1 << 20))
      return fail(nullptr, SFT_ERR_ARG, "shape out of range (ntheta >= 5, nphi >= 8)");
  sft_handle h = new sft_grid();
  h->n_real = n_real;
  h->prec = prec;
  h->elem = prec == SFT_FP32 ? 4 : 8;
  auto bail = [&](sft_status st) {
    g_create_error = h->err;
    free_handle(h);
    return st;
  };
#define CREATE_CUDA(call)                                                                \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      h->err = std::string(#call) + ": " + cudaGetErrorString(e_);                       \
      return bail(e_ == cudaErrorMemoryAllocation ? SFT_ERR_OOM : SFT_ERR_CUDA);         \
    }                                                                                    \
  } while (0)
  CREATE_CUDA(cudaGetDevice(&h->device));
  if (cuda_stream) {
    h->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    CREATE_CUDA(cudaStreamCreate(&h->stream));  // blocking: ordered with the legacy stream
    h->own_stream = true;
  }
  // shapes in order of first appearance
  std::map<std::pair<int, int>, int> shape_id;
  h->reals.resize(n_real);
  for (int r = 0; r < n_real; ++r) {
    auto key = std::make_pair(shapes[r].ntheta, shapes[r].nphi);
    auto it = shape_id.find(key);
    if (it == shape_id.end()) {
      ShapeInfo s;
      s.nt = key.first;
      s.np = key.second;
      s.pitch = (int)round_up(s.np, 32);
      build_shape(s);
      it = shape_id.emplace(key, (int)h->shapes.size()).first;
      h->shapes.push_back(std::move(s));
    }
    RealInfo& ri = h->reals[r];
    ri.shape = it->second;
    const ShapeInfo& s = h->shapes[ri.shape];
    ri.cells = (int64_t)s.nt * s.pitch;
    ri.off = h->state_elems;
    h->state_elems += ri.cells;
  }
  // The fused RKL2 path (FP32, every shape with an interior band) needs two
  // more increment arrays and a small cap-block scratch.
  h->fused_ok = prec == SFT_FP32;
  for (auto& s : h->shapes) h->fused_ok = h->fused_ok && fused::shape_ok(s.nt, s.np);
  h->fused = h->fused_ok;
  h->n_work = h->fused_ok ? 5 : 3;
  // HBM admission: the state stays resident; work arrays hold one wave.
  const int64_t state_bytes = h->state_elems * (int64_t)h->elem;
  int64_t avail = INT64_MAX;
  if (hbm_budget_bytes > 0) {
    const int64_t reserve = 64ll << 20;  // tables, tiles, reductions
    avail = (int64_t)hbm_budget_bytes - state_bytes - reserve;
  }
  {
    Wave cur;
    int64_t used = 0;  // bytes per work array in the current wave
    for (int r = 0; r < n_real; ++r) {
      const int64_t per_array = h->reals[r].cells * (int64_t)h->elem;
      const int64_t nw = h->n_work;
      if (nw * per_array > avail) {
        h->err = "HBM budget too small for one realization's work buffers";
        return bail(SFT_ERR_OOM);
      }
      if (nw * (used + per_array) > avail && !cur.reals.empty()) {
        h->waves.push_back(std::move(cur));
        cur = Wave();
        used = 0;
      }
      h->reals[r].woff = used / (int64_t)h->elem;
      h->reals[r].wave = (int)h->waves.size();
      cur.reals.push_back(r);
      used += per_array;
      h->work_elems = std::max<int64_t>(h->work_elems, used / (int64_t)h->elem);
    }
    if (!cur.reals.empty()) h->waves.push_back(std::move(cur));
    h->wave_size = 0;
    for (auto& w : h->waves) h->wave_size = std::max<int>(h->wave_size, (int)w.reals.size());
  }
  CREATE_CUDA(dev_malloc(&h->state, state_bytes));
  CREATE_CUDA(cudaMemsetAsync(h->state, 0, state_bytes, h->stream));
  for (int i = 0; i < h->n_work; ++i) {
    CREATE_CUDA(dev_malloc(&h->work[i], std::max<int64_t>(h->work_elems, 32) * (int64_t)h->elem));
    CREATE_CUDA(cudaMemsetAsync(h->work[i], 0, std::max<int64_t>(h->work_elems, 32) * (int64_t)h->elem,
                                h->stream));
  }
  std::vector<int32_t> poff(n_real, 0);
  if (h->fused_ok) {
    // ring-sum partials of the rows next to the poles, per realization, per wave
    for (auto& w : h->waves) {
      int64_t used = 0;
      for (int r : w.reals) {
        poff[r] = (int32_t)used;
        used += fused::part_elems(h->shapes[h->reals[r].shape].np);
      }
      h->polar_elems = std::max(h->polar_elems, used);
    }
    CREATE_CUDA(dev_malloc(&h->polar, std::max<int64_t>(h->polar_elems, 32) * sizeof(double)));
    CREATE_CUDA(cudaMemsetAsync(h->polar, 0, std::max<int64_t>(h->polar_elems, 32) * sizeof(double), h->stream));
    CREATE_CUDA(prepare_rkl2_fused());
  }
  sft_status st = prec == SFT_FP32 ? upload_tables<float>(h) : upload_tables<double>(h);
  if (st != SFT_OK) return bail(st);
  std::vector<RealDesc> desc(n_real);
  for (int r = 0; r < n_real; ++r) {
    const RealInfo& ri = h->reals[r];
    const ShapeInfo& s = h->shapes[ri.shape];
    desc[r] = RealDesc{ri.off,  ri.woff,       s.nt,  s.np,    s.pitch,
                       ri.shape, s.geo, ri.flow_row, s.col, poff[r], fused::default_band_rows(s.nt)};
  }
  CREATE_CUDA(dev_malloc(&h->d_desc, desc.size() * sizeof(RealDesc)));
  CREATE_CUDA(cudaMemcpy(h->d_desc, desc.data(), desc.size() * sizeof(RealDesc), cudaMemcpyHostToDevice));
  h->desc = desc;
  {
    const std::string bad = check_desc(h);
    if (!bad.empty()) {
      h->err = "internal table check: " + bad;
      return bail(SFT_ERR_STATE);
    }
  }
  CREATE_CUDA(dev_malloc(&h->d_status, sizeof(int)));
  CREATE_CUDA(cudaMemset(h->d_status, 0, sizeof(int)));
  // reduction tiles: bands of about 32k cells
  std::vector<RedTile> rt;
  std::vector<int> rstart;
  for (int r = 0; r < n_real; ++r) {
    const ShapeInfo& s = h->shapes[h->reals[r].shape];
    rstart.push_back((int)rt.size());
    const int band = std::max(1, 32768 / s.np);
    for (int j0 = 0; j0 < s.nt; j0 += band) rt.push_back(RedTile{r, j0, std::min(s.nt, j0 + band), 0});
  }
  rstart.push_back((int)rt.size());
  h->n_rtiles = (int)rt.size();
  CREATE_CUDA(dev_malloc(&h->d_rtiles, rt.size() * sizeof(RedTile)));
  CREATE_CUDA(cudaMemcpy(h->d_rtiles, rt.data(), rt.size() * sizeof(RedTile), cudaMemcpyHostToDevice));
  CREATE_CUDA(dev_malloc(&h->d_rstart, rstart.size() * sizeof(int)));
  CREATE_CUDA(cudaMemcpy(h->d_rstart, rstart.data(), rstart.size() * sizeof(int), cudaMemcpyHostToDevice));
  CREATE_CUDA(dev_malloc(&h->d_partials, (size_t)h->n_rtiles * kDiagFields * sizeof(double)));
  CREATE_CUDA(dev_malloc(&h->d_red, (size_t)n_real * kDiagFields * sizeof(double)));
  CREATE_CUDA(host_malloc(&h->h_red, (size_t)n_real * kDiagFields * sizeof(double)));
  CREATE_CUDA(dev_malloc(&h->d_wpar, (size_t)n_real * 4 * sizeof(double)));
  CREATE_CUDA(dev_malloc(&h->d_obs_off, (size_t)n_real * sizeof(int64_t)));
  for (auto& e : h->ev) CREATE_CUDA(cudaEventCreate(&e));
  CREATE_CUDA(cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, h->device));
  CREATE_CUDA(cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming));
  for (auto& e : h->cfg_stage_ev) CREATE_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  for (int ch = 1; ch < kMaxChains; ++ch) {
    CREATE_CUDA(cudaStreamCreateWithFlags(&h->side[ch], cudaStreamNonBlocking));
    CREATE_CUDA(cudaEventCreateWithFlags(&h->join[ch], cudaEventDisableTiming));
  }
  CREATE_CUDA(cudaStreamSynchronize(h->stream));
#undef CREATE_CUDA
  *out = h;
  return SFT_OK;
}

sft_status sft_destroy(sft_handle h) {
  free_handle(h);
  return SFT_OK;
}

static sft_status check_r(sft_handle h, int32_t r) {
  if (!h) return fail(nullptr, SFT_ERR_ARG, "NULL handle");
  if (r < 0 || r >= h->n_real) return fail(h, SFT_ERR_ARG, "realization index out of range");
  SFT_CUDA(h, cudaSetDevice(h->device));
  return SFT_OK;
}

sft_status sft_set_state(sft_handle h, int32_t r, const void* br, int32_t on_device) {
  sft_status st = check_r(h, r);
  if (st != SFT_OK) return st;
  if (!br) return fail(h, SFT_ERR_ARG, "br is NULL");
  const RealInfo& ri = h->reals[r];
  const ShapeInfo& s = h->shapes[ri.shape];
  char* dst = static_cast<char*>(h->state) + ri.off * h->elem;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (s.pitch == s.np)  // unpadded rows: one linear copy
    SFT_CUDA(h, cudaMemcpyAsync(dst, br, (size_t)s.nt * s.np * h->elem, kind, h->stream));
  else
    SFT_CUDA(h, cudaMemcpy2DAsync(dst, s.pitch * h->elem, br, s.np * h->elem, s.np * h->elem, s.nt, kind,
                                  h->stream));
  if (h->prec == SFT_FP32) {
    SFT_CUDA(h, launch_fix_poles<float>(h->n_real, h->stream, h->d_desc, ptr<float>(h->state), r));
  } else {
    SFT_CUDA(h, launch_fix_poles<double>(h->n_real, h->stream, h->d_desc, ptr<double>(h->state), r));
  }
  return SFT_OK;
}

sft_status sft_get_state(sft_handle h, int32_t r, void* br, int32_t on_device) {
  sft_status st = check_r(h, r);
  if (st != SFT_OK) return st;
  if (!br) return fail(h, SFT_ERR_ARG, "br is NULL");
  const RealInfo& ri = h->reals[r];
  const ShapeInfo& s = h->shapes[ri.shape];
  const char* src = static_cast<const char*>(h->state) + ri.off * h->elem;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (s.pitch == s.np)  // unpadded rows: one linear copy
    SFT_CUDA(h, cudaMemcpyAsync(br, src, (size_t)s.nt * s.np * h->elem, kind, h->stream));
  else
    SFT_CUDA(h, cudaMemcpy2DAsync(br, s.np * h->elem, src, s.pitch * h->elem, s.np * h->elem, s.nt, kind,
                                  h->stream));
  if (!on_device) return sync(h);
  return SFT_OK;
}

// Checks a member subset for the batched state calls: indices in range,
// one grid shape (returned in *shape), distinct when `distinct`.
static sft_status check_subset(sft_handle h, int32_t n, const int32_t* idx, bool distinct, int* shape) {
  if (!h) return fail(nullptr, SFT_ERR_ARG, "NULL handle");
  if (n < 0 || (n > 0 && !idx)) return fail(h, SFT_ERR_ARG, "bad member subset");
  *shape = -1;
  std::vector<char> seen(distinct ? h->n_real : 0, 0);
  for (int q = 0; q < n; ++q) {
    const int r = idx[q];
    if (r < 0 || r >= h->n_real) return fail(h, SFT_ERR_ARG, "realization index out of range");
    const int sh = h->reals[r].shape;
    if (*shape >= 0 && sh != *shape) return fail(h, SFT_ERR_ARG, "member subset mixes grid shapes");
    *shape = sh;
    if (distinct) {
      if (seen[r]) return fail(h, SFT_ERR_ARG, "repeated realization in the subset");
      seen[r] = 1;
    }
  }
  return SFT_OK;
}

sft_status sft_set_states(sft_handle h, int32_t n, const int32_t* idx, const void* maps, int32_t on_device) {
  int shape = -1;
  sft_status st = check_subset(h, n, idx, true, &shape);
  if (st != SFT_OK) return st;
  if (n == 0) return SFT_OK;
  if (!maps) return fail(h, SFT_ERR_ARG, "maps is NULL");
  const ShapeInfo& s = h->shapes[shape];
  const size_t map_bytes = (size_t)s.nt * s.np * h->elem;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  for (int q = 0; q < n; ++q) {
    char* dst = static_cast<char*>(h->state) + h->reals[idx[q]].off * h->elem;
    const char* src = static_cast<const char*>(maps) + q * map_bytes;
    if (s.pitch == s.np)
      SFT_CUDA(h, cudaMemcpyAsync(dst, src, map_bytes, kind, h->stream));
    else
      SFT_CUDA(h, cudaMemcpy2DAsync(dst, s.pitch * h->elem, src, s.np * h->elem, s.np * h->elem, s.nt, kind,
                                    h->stream));
  }
  // pole rows from their k = 0 entries, every realization in one launch (idempotent elsewhere)
  if (h->prec == SFT_FP32)
    SFT_CUDA(h, launch_fix_poles<float>(h->n_real, h->stream, h->d_desc, ptr<float>(h->state), -1));
  else
    SFT_CUDA(h, launch_fix_poles<double>(h->n_real, h->stream, h->d_desc, ptr<double>(h->state), -1));
  return SFT_OK;
}

sft_status sft_get_states(sft_handle h, int32_t n, const int32_t* idx, void* maps, int32_t on_device) {
  int shape = -1;
  sft_status st = check_subset(h, n, idx, false, &shape);
  if (st != SFT_OK) return st;
  if (n == 0) return SFT_OK;
  if (!maps) return fail(h, SFT_ERR_ARG, "maps is NULL");
  const ShapeInfo& s = h->shapes[shape];
  const size_t map_bytes = (size_t)s.nt * s.np * h->elem;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  for (int q = 0; q < n; ++q) {
    const char* src = static_cast<const char*>(h->state) + h->reals[idx[q]].off * h->elem;
    char* dst = static_cast<char*>(maps) + q * map_bytes;
    if (s.pitch == s.np)
      SFT_CUDA(h, cudaMemcpyAsync(dst, src, map_bytes, kind, h->stream));
    else
      SFT_CUDA(h, cudaMemcpy2DAsync(dst, s.np * h->elem, src, s.pitch * h->elem, s.np * h->elem, s.nt, kind,
                                    h->stream));
  }
  if (!on_device) return sync(h);
  return SFT_OK;
}

sft_status sft_set_times(sft_handle h, int32_t n, const int32_t* idx, const double* t_hours) {
  if (!h) return fail(nullptr, SFT_ERR_ARG, "NULL handle");
  if (n < 0 || (n > 0 && (!idx || !t_hours))) return fail(h, SFT_ERR_ARG, "NULL argument");
  for (int q = 0; q < n; ++q) {
    if (idx[q] < 0 || idx[q] >= h->n_real) return fail(h, SFT_ERR_ARG, "realization index out of range");
    if (!std::isfinite(t_hours[q])) return fail(h, SFT_ERR_ARG, "time must be finite");
  }
  for (int q = 0; q < n; ++q) h->reals[idx[q]].t = t_hours[q];
  return SFT_OK;
}

sft_status sft_set_time(sft_handle h, int32_t r, double t_hours) {
  if (!h) return fail(nullptr, SFT_ERR_ARG, "NULL handle");
  if (r < -1 || r >= h->n_real) return fail(h, SFT_ERR_ARG, "realization index out of range");
  if (!std::isfinite(t_hours)) return fail(h, SFT_ERR_ARG, "time must be finite");
  for (int i = 0; i < h->n_real; ++i)
    if (r < 0 || i == r) h->reals[i].t = t_hours;
  return SFT_OK;
}

sft_status sft_get_time(sft_handle h, double* t_hours) {
  if (!h || !t_hours) return fail(h, SFT_ERR_ARG, "NULL argument");
  for (int r = 0; r < h->n_real; ++r) t_hours[r] = h->reals[r].t;
  return SFT_OK;
}

sft_status sft_set_flows(sft_handle h, const sft_flow_params* params) {
  if (!h || !params) return fail(h, SFT_ERR_ARG, "NULL argument");
  SFT_CUDA(h, cudaSetDevice(h->device));
  for (int r = 0; r < h->n_real; ++r) {
    const sft_flow_params& p = params[r];
    if (p.adv_time != params[0].adv_time || p.diffusion != params[0].diffusion ||
        p.splitting != params[0].splitting)
      return fail(h, SFT_ERR_ARG, "adv_time, diffusion and splitting must be the same for all realizations");
    if (p.splitting != SFT_SPLIT_LIE && p.splitting != SFT_SPLIT_STRANG)
      return fail(h, SFT_ERR_ARG, "bad splitting");
    if (p.adv_space != SFT_ADV_WENO3_CSH && p.adv_space != SFT_ADV_UPWIND)
      return fail(h, SFT_ERR_ARG, "bad adv_space");
    if (p.adv_time < SFT_TIME_SSPRK43 || p.adv_time > SFT_TIME_FE)
      return fail(h, SFT_ERR_ARG, "bad adv_time");
    if (p.diffusion != SFT_DIFF_RKL2 && p.diffusion != SFT_DIFF_RKG2 && p.diffusion != SFT_DIFF_OFF)
      return fail(h, SFT_ERR_ARG, "bad diffusion");
    if (!(p.nu >= 0.0) || !(p.cfl_safety > 0.0) || !std::isfinite(p.d0 + p.d2 + p.d4 + p.m1 + p.m3 + p.m5))
      return fail(h, SFT_ERR_ARG, "bad flow parameters (nu >= 0, cfl_safety > 0, finite)");
    if (!(p.atten_b0 >= 0.0) || !std::isfinite(p.atten_b0))
      return fail(h, SFT_ERR_ARG, "atten_b0 must be 0 (off) or a finite positive field");
    if (!(p.nu_grid_alpha >= 0.0) || !std::isfinite(p.nu_grid_alpha))
      return fail(h, SFT_ERR_ARG, "nu_grid_alpha must be 0 (constant nu) or finite positive");
  }
  // stale configurations refer to the old parameters
  SFT_CUDA(h, cudaStreamSynchronize(h->stream));
  for (auto& w : h->waves) {
    for (auto& c : w.configs) free_config(*c, h->stream);
    w.configs.clear();
  }
  // tables are rewritten in place: until they are complete no step may run
  h->flows_set = false;
  sft_status st = h->prec == SFT_FP32 ? set_flows_t<float>(h, params) : set_flows_t<double>(h, params);
  if (st == SFT_OK) {
    h->flows_set = true;
    h->strang = params[0].splitting == SFT_SPLIT_STRANG;
  }
  return st;
}

sft_status sft_step(sft_handle h, double t_target_hours, int32_t max_steps, int32_t* steps_taken) {
  NvtxRange nvtx("sft_step");
  if (!h) return fail(nullptr, SFT_ERR_ARG, "NULL handle");
  if (steps_taken) *steps_taken = 0;
  if (!h->flows_set) return fail(h, SFT_ERR_STATE, "sft_set_flows must come before sft_step");
  if (!std::isfinite(t_target_hours)) return fail(h, SFT_ERR_ARG, "t_target must be finite");
  SFT_CUDA(h, cudaSetDevice(h->device));
  int n = 0;
  while (max_steps <= 0 || n < max_steps) {
    bool any_wave = false;
    for (auto& w : h->waves) {
      bool any = false;
      sft_status st = h->prec == SFT_FP32 ? run_step<float>(h, w, t_target_hours, &any)
                                          : run_step<double>(h, w, t_target_hours, &any);
      if (st != SFT_OK) return st;
      any_wave |= any;
    }
    if (!any_wave) break;
    ++n;
    h->stats.global_steps += 1;
    if (h->profiling) {
      sft_status st = check_status_word(h);
      if (st != SFT_OK) return st;
    }
  }
  if (steps_taken) *steps_taken = n;
  return SFT_OK;
}

sft_status sft_assimilate(sft_handle h, const void* br_obs, const void* mu, int32_t obs_per_realization,
                          int32_t on_device, const sft_assim_params* params) {
  NvtxRange nvtx("sft_assimilate");
  if (!h || !br_obs || !mu || !params) return fail(h, SFT_ERR_ARG, "NULL argument");
  SFT_CUDA(h, cudaSetDevice(h->device));
  std::vector<int64_t> off(h->n_real, 0);
  int64_t total = 0;
  if (obs_per_realization == 1) {  // one map per realization, in realization order
    for (int r = 0; r < h->n_real; ++r) {
      const ShapeInfo& s = h->shapes[h->reals[r].shape];
      off[r] = total;
      total += (int64_t)s.nt * s.np;
    }
  } else if (obs_per_realization == 2) {  // one map per grid shape, in shape order
    std::vector<int64_t> soff(h->shapes.size());
    for (size_t si = 0; si < h->shapes.size(); ++si) {
      soff[si] = total;
      total += (int64_t)h->shapes[si].nt * h->shapes[si].np;
    }
    for (int r = 0; r < h->n_real; ++r) off[r] = soff[h->reals[r].shape];
  } else if (obs_per_realization == 0) {
    for (int r = 1; r < h->n_real; ++r)
      if (h->reals[r].shape != h->reals[0].shape)
        return fail(h, SFT_ERR_ARG, "shared observations need one grid shape for all realizations");
    const ShapeInfo& s = h->shapes[h->reals[0].shape];
    total = (int64_t)s.nt * s.np;
  } else {
    return fail(h, SFT_ERR_ARG, "obs_per_realization must be 0, 1 or 2");
  }
  std::vector<double> w(4 * h->n_real);
  for (int r = 0; r < h->n_real; ++r) {
    const sft_assim_params& p = params[r];
    if (!(p.mu_lim >= -1.0) || !std::isfinite(p.alpha_mu)) return fail(h, SFT_ERR_ARG, "bad assim params");
    w[4 * r + 0] = p.alpha_mu;
    w[4 * r + 1] = p.mu_lim;
    w[4 * r + 2] = p.lat_lim_deg * kPi / 180.0;
    w[4 * r + 3] = p.flux_balance ? 1.0 : 0.0;
  }
  if (w != h->h_wpar_last) {
    SFT_CUDA(h, cudaMemcpyAsync(h->d_wpar, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice,
                                h->stream));
    SFT_CUDA(h, cudaStreamSynchronize(h->stream));
    h->h_wpar_last = w;
  }
  if (off != h->h_obs_off_last) {
    SFT_CUDA(h, cudaMemcpyAsync(h->d_obs_off, off.data(), off.size() * sizeof(int64_t),
                                cudaMemcpyHostToDevice, h->stream));
    SFT_CUDA(h, cudaStreamSynchronize(h->stream));
    h->h_obs_off_last = off;
  }
  const void* dobs = br_obs;
  const void* dmu = mu;
  if (!on_device) {
    const size_t bytes = (size_t)total * h->elem;
    if (2 * bytes > h->obs_bytes) {
      SFT_CUDA(h, cudaStreamSynchronize(h->stream));
      cudaFree(h->d_obs);
      h->d_obs = nullptr;
      h->obs_bytes = 0;
      SFT_CUDA(h, dev_malloc(&h->d_obs, 2 * bytes));
      h->obs_bytes = 2 * bytes;
    }
    char* base = static_cast<char*>(h->d_obs);
    SFT_CUDA(h, cudaMemcpyAsync(base, br_obs, bytes, cudaMemcpyHostToDevice, h->stream));
    SFT_CUDA(h, cudaMemcpyAsync(base + bytes, mu, bytes, cudaMemcpyHostToDevice, h->stream));
    dobs = base;
    dmu = base + bytes;
  }
  AssimArgs aa{dobs, dmu, h->d_obs_off, h->d_wpar};
  sft_status st;
  if (h->prec == SFT_FP32) {
    st = reduce_fold<float>(h, RED_ASSIM, 0.0, aa);
    if (st != SFT_OK) return st;
    SFT_CUDA(h, launch_apply<float>(RED_ASSIM, h->n_rtiles, h->stream, h->d_rtiles, h->d_desc, h->d_geod,
                                    ptr<float>(h->state), aa, h->d_red));
  } else {
    st = reduce_fold<double>(h, RED_ASSIM, 0.0, aa);
    if (st != SFT_OK) return st;
    SFT_CUDA(h, launch_apply<double>(RED_ASSIM, h->n_rtiles, h->stream, h->d_rtiles, h->d_desc, h->d_geod,
                                     ptr<double>(h->state), aa, h->d_red));
  }
  if (!on_device) SFT_CUDA(h, cudaStreamSynchronize(h->stream));  // staging reused next call
  return SFT_OK;
}

sft_status sft_set_rfe(sft_handle h, const sft_rfe_params* params) {
  if (!h) return fail(nullptr, SFT_ERR_ARG, "NULL handle");
  SFT_CUDA(h, cudaSetDevice(h->device));
  if (params) {
    for (int r = 0; r < h->n_real; ++r) {
      const sft_rfe_params& p = params[r];
      if (p.method < 0 || p.method > 2) return fail(h, SFT_ERR_ARG, "rfe method must be 0, 1 or 2");
      if (!(p.rate_mx_per_hour >= 0.0) || !std::isfinite(p.rate_mx_per_hour))
        return fail(h, SFT_ERR_ARG, "rfe rate must be finite and >= 0");
      if (std::isnan(p.lifetime_hours)) return fail(h, SFT_ERR_ARG, "rfe lifetime is NaN");
      if (p.origin_given && !std::isfinite(p.origin_hours)) return fail(h, SFT_ERR_ARG, "rfe origin must be finite");
    }
  }
  // the step graphs change shape: drop the cached configurations
  SFT_CUDA(h, cudaStreamSynchronize(h->stream));
  for (auto& w : h->waves) {
    for (auto& c : w.configs) free_config(*c, h->stream);
    w.configs.clear();
  }
  bool any = false;
  for (int r = 0; r < h->n_real && params; ++r)
    any = any || (params[r].method != 0 && params[r].rate_mx_per_hour > 0.0);
  // buffers first: a failed allocation leaves the previous settings in force
  if (any && !h->d_rfe) SFT_CUDA(h, dev_malloc(&h->d_rfe, (size_t)h->n_real * sizeof(RfeStep)));
  if (any && !h->d_rfe_fac) SFT_CUDA(h, dev_malloc(&h->d_rfe_fac, (size_t)h->n_real * 8 * sizeof(double)));
  for (int r = 0; r < h->n_real; ++r) {
    RealInfo& ri = h->reals[r];
    ri.rfe = params ? params[r] : sft_rfe_params{};
    ri.rfe_t0 = ri.rfe.origin_given ? ri.rfe.origin_hours : ri.t;
    ri.rfe_m0 = -1;
  }
  h->any_rfe = any;
  return SFT_OK;
}

sft_status sft_balance_flux(sft_handle h) {
  if (!h) return fail(nullptr, SFT_ERR_ARG, "NULL handle");
  SFT_CUDA(h, cudaSetDevice(h->device));
  AssimArgs aa{nullptr, nullptr, nullptr, nullptr};
  sft_status st;
  if (h->prec == SFT_FP32) {
    st = reduce_fold<float>(h, RED_BALANCE, 0.0, aa);
    if (st != SFT_OK) return st;
    SFT_CUDA(h, launch_apply<float>(RED_BALANCE, h->n_rtiles, h->stream, h->d_rtiles, h->d_desc,
                                    h->d_geod, ptr<float>(h->state), aa, h->d_red));
  } else {
    st = reduce_fold<double>(h, RED_BALANCE, 0.0, aa);
    if (st != SFT_OK) return st;
    SFT_CUDA(h, launch_apply<double>(RED_BALANCE, h->n_rtiles, h->stream, h->d_rtiles, h->d_desc,
                                     h->d_geod, ptr<double>(h->state), aa, h->d_red));
  }
  return SFT_OK;
}

sft_status sft_flux_diagnostics(sft_handle h, double lat_cut_deg, sft_diag* out) {
  NvtxRange nvtx("sft_flux_diagnostics");
  if (!h || !out) return fail(h, SFT_ERR_ARG, "NULL argument");
  SFT_CUDA(h, cudaSetDevice(h->device));
  AssimArgs aa{nullptr, nullptr, nullptr, nullptr};
  const double cut = lat_cut_deg * kPi / 180.0;
  sft_status st = h->prec == SFT_FP32 ? reduce_fold<float>(h, RED_DIAG, cut, aa)
                                      : reduce_fold<double>(h, RED_DIAG, cut, aa);
  if (st != SFT_OK) return st;
  SFT_CUDA(h, cudaMemcpyAsync(h->h_red, h->d_red, (size_t)h->n_real * kDiagFields * sizeof(double),
                              cudaMemcpyDeviceToHost, h->stream));
  SFT_CUDA(h, cudaStreamSynchronize(h->stream));
  const double mx = kRsunCm * kRsunCm;
  const double k3 = 3.0 / (4.0 * kPi);
  for (int r = 0; r < h->n_real; ++r) {
    const double* v = h->h_red + (size_t)r * kDiagFields;
    sft_diag& d = out[r];
    d.flux_signed = v[0] * mx;
    d.flux_pos = v[1] * mx;
    d.flux_neg = v[2] * mx;
    d.flux_pole_n = v[3] * mx;
    d.flux_pole_s = v[4] * mx;
    d.area_pole_n = v[5] * mx;
    d.area_pole_s = v[6] * mx;
    d.dipole_axial = k3 * v[7];
    d.h1 = k3 * v[8];
    d.h2 = k3 * v[9];
    d.nonfinite = (int64_t)v[10];
    d.brmin = v[11];
    d.brmax = v[12];
    d.absmin = v[13];
    d.t_hours = h->reals[r].t;
    d.steps = h->reals[r].steps;
  }
  return check_status_word(h);
}

sft_status sft_get_stats(sft_handle h, sft_stats* out) {
  if (!h || !out) return fail(h, SFT_ERR_ARG, "NULL argument");
  SFT_CUDA(h, cudaSetDevice(h->device));
  SFT_CUDA(h, cudaStreamSynchronize(h->stream));
  *out = h->stats;
  return SFT_OK;
}

sft_status sft_reset_stats(sft_handle h) {
  if (!h) return fail(nullptr, SFT_ERR_ARG, "NULL handle");
  h->stats = sft_stats{};
  return SFT_OK;
}

sft_status sft_set_profiling(sft_handle h, int32_t profile) {
  if (!h) return fail(nullptr, SFT_ERR_ARG, "NULL handle");
  h->profiling = profile != 0;
  return SFT_OK;
}

sft_status sft_set_graphs(sft_handle h, int32_t use_graphs) {
  if (!h) return fail(nullptr, SFT_ERR_ARG, "NULL handle");
  h->use_graphs = use_graphs != 0;
  return SFT_OK;
}

sft_status sft_set_fusion(sft_handle h, int32_t stages_per_pass) {
  if (!h) return fail(nullptr, SFT_ERR_ARG, "NULL handle");
  if (stages_per_pass != 1 && stages_per_pass != fused::K)
    return fail(h, SFT_ERR_ARG, "stages per pass must be 1 or " + std::to_string(fused::K));
  if (stages_per_pass == fused::K && !h->fused_ok)
    return fail(h, SFT_ERR_ARG, "fused RKL2 needs FP32 and grids with ntheta >= " +
                                    std::to_string(2 * fused::K + 4) + ", nphi >= 16");
  h->fused = stages_per_pass == fused::K;
  return SFT_OK;
}

int32_t sft_get_fusion(sft_handle h) { return h ? (h->fused ? fused::K : 1) : 0; }

sft_status sft_set_tile_rows(sft_handle h, int32_t shape_id, int32_t rows) {
  if (!h) return fail(nullptr, SFT_ERR_ARG, "NULL handle");
  if (shape_id < 0 || shape_id >= (int)h->shapes.size()) return fail(h, SFT_ERR_ARG, "bad shape id");
  if (rows != 0 && rows != 1 && rows != 2 && rows != 4 && rows != 8)
    return fail(h, SFT_ERR_ARG, "tile rows must be 0, 1, 2, 4 or 8");
  h->shapes[shape_id].tile_rows = rows;
  return SFT_OK;
}

int32_t sft_get_tile_rows(sft_handle h, int32_t shape_id) {
  if (!h || shape_id < 0 || shape_id >= (int)h->shapes.size()) return 0;
  return h->shapes[shape_id].tile_rows;
}

sft_status sft_set_band_rows(sft_handle h, int32_t shape_id, int32_t rows) {
  if (!h) return fail(nullptr, SFT_ERR_ARG, "NULL handle");
  if (shape_id < 0 || shape_id >= (int)h->shapes.size()) return fail(h, SFT_ERR_ARG, "bad shape id");
  if (rows != 0 && (rows <= fused::K || rows > (1 << 16)))
    return fail(h, SFT_ERR_ARG, "band rows must be 0 or in (" + std::to_string(fused::K) + ", 65536]");
  if (rows == 0) {  // the next step tunes it; until then the default
    sft_status st = set_band(h, shape_id, fused::default_band_rows(h->shapes[shape_id].nt));
    h->shapes[shape_id].band_rows = 0;
    return st;
  }
  return set_band(h, shape_id, rows);
}

int32_t sft_get_band_rows(sft_handle h, int32_t shape_id) {
  if (!h || shape_id < 0 || shape_id >= (int)h->shapes.size()) return 0;
  return h->shapes[shape_id].band_rows;
}

int32_t sft_wave_size(sft_handle h) { return h ? h->wave_size : 0; }

sft_status sft_step_plan(sft_handle h, int32_t r, double dt_hours, double* dt_cfl, double* dt_euler,
                         int32_t* stages) {
  if (!h) return fail(nullptr, SFT_ERR_ARG, "NULL handle");
  if (r < 0 || r >= h->n_real) return fail(h, SFT_ERR_ARG, "realization index out of range");
  if (!h->flows_set) return fail(h, SFT_ERR_STATE, "sft_set_flows first");
  const RealInfo& ri = h->reals[r];
  if (dt_cfl) *dt_cfl = ri.dt_cfl;
  if (dt_euler) *dt_euler = ri.dt_euler;
  if (stages) *stages = sts_stages(ri.fp.diffusion, dt_hours, ri.dt_euler);
  return SFT_OK;
}

sft_status sft_debug_checks(uint64_t* first_failure, uint32_t* failures, int32_t reset) {
  if (!sft::kDebugBuild) return fail(nullptr, SFT_ERR_STATE, "library built without SFT_DEBUG");
  const cudaError_t e = sft::debug_read(first_failure, failures, reset != 0);
  if (e != cudaSuccess) return fail(nullptr, SFT_ERR_CUDA, std::string("sft_debug_checks: ") + cudaGetErrorString(e));
  return SFT_OK;
}

sft_status sft_debug_probe(int32_t site, int64_t value, int64_t lo, int64_t hi) {
  if (!sft::kDebugBuild) return fail(nullptr, SFT_ERR_STATE, "library built without SFT_DEBUG");
  if (site <= 0 || site > 0xffff || lo > hi) return fail(nullptr, SFT_ERR_ARG, "site in 1..65535 and lo <= hi");
  cudaError_t e = sft::launch_debug_probe(site, value, lo, hi, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(nullptr, SFT_ERR_CUDA, std::string("sft_debug_probe: ") + cudaGetErrorString(e));
  return SFT_OK;
}

sft_status sft_debug_fail_alloc(int32_t nth) {
  if (nth < 0) return fail(nullptr, SFT_ERR_ARG, "nth must be >= 0");
  g_fail_alloc.store(nth);
  return SFT_OK;
}

}  // extern "C"
