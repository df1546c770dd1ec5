// sft_device.cuh -- device-side data layout and kernels of libsft.
//
// Layout (all realizations of a handle share one pool per array):
//   map[r](j, k) = pool[desc[r].off + j * pitch + k], j = 0..nt-1 (poles at
//   j = 0 and nt-1, each pole row holding one value), k = 0..np-1 unique
//   longitudes, pitch = np rounded up to 32 elements (128-B rows in FP32).
// Work arrays (advection stage buffers, RKL2 increments) use the same layout
// at desc[r].woff.
//
// Every stage kernel is launched over a table of tiles.  An interior tile is
// TR rows x TC columns of one realization, one thread per V consecutive
// longitudes (V = 4 floats or 2 doubles: one 16-byte vector); a pole tile is
// one block that reduces the ring next to the pole in FP64 and rewrites the
// pole row.  Tiles are ordered so that the realizations still active at a
// given stage form a prefix of the table: a stage launches only that prefix.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sft {

constexpr int kThreads = 256;
constexpr int kAdvRun = 8;  // interior rows one advection thread marches through

// ---- Index checks of the debug build (compiled with -DSFT_DEBUG) ----------
// A kernel checks each index it derives from its tile and descriptor (a row,
// a column, the first and last row of a band) against the closed range
// [lo, hi] inside which every access it makes with that index stays within
// the realization's rows.  A failed check records (site, value) on the device
// (the first failure wins; a counter counts them all) and clamps the index
// into its range, so the accesses that follow stay in bounds and nothing
// traps.  The release build compiles the checks away.  The host-built tables
// the kernels start from (descriptors, tiles) are checked on the host when
// they are built, in every build.
#ifdef SFT_DEBUG
constexpr bool kDebugBuild = true;
#define SFT_DCHECK(site, v, lo, hi) ((v) = ::sft::dbg_check((site), (v), (lo), (hi)))
#else
constexpr bool kDebugBuild = false;
#define SFT_DCHECK(site, v, lo, hi) ((void)0)
#endif

// Check sites (the high 16 bits of the recorded word).
enum DebugSite : int {
  DBG_PROBE = 1,          // sft_debug_probe
  DBG_STAGE_ROW = 2,      // rkl2_stage_kernel interior row j in [1, nt-2]
  DBG_STAGE_COL = 3,      // its first column kc in [0, pitch-V]
  DBG_ADV_ROW = 4,        // adv_stage_kernel interior row
  DBG_ADV_COL = 5,        // its first column
  DBG_FUSED_FIRST = 6,    // rkl2_fused_kernel band: first loaded row in [0, nt-1]
  DBG_FUSED_LAST = 7,     // last loaded row in [first, nt-1]
  DBG_FUSED_COL = 8,      // a lane's first column in [0, np-1] (np-4 when vectorised)
  DBG_FUSED_CAP = 9,      // unused
  DBG_RED_ROWS = 10,      // reduction / RFE tile rows within [0, nt]
};

// Records (site, value) and counts the failure (defined in the debug build).
__device__ void dbg_record(int site, int64_t v);

template <typename I>
__device__ __forceinline__ I dbg_check(int site, I v, I lo, I hi) {
  if (v < lo || v > hi) {
    dbg_record(site, (int64_t)v);
    return v < lo ? lo : hi;
  }
  return v;
}

// Host side of the checks: read (and optionally clear) the record, run one
// check on the device with no memory access (a self-test of the record path).
// Both return cudaErrorNotSupported in the release build.
cudaError_t debug_read(uint64_t* first, uint32_t* count, bool reset);
cudaError_t launch_debug_probe(int site, int64_t v, int64_t lo, int64_t hi, cudaStream_t st);

template <typename T> struct VecT;
template <> struct VecT<float> { using type = float4; static constexpr int N = 4; };
template <> struct VecT<double> { using type = double2; static constexpr int N = 2; };

struct RealDesc {
  int64_t off;     // element offset of row 0 in the state pool
  int64_t woff;    // element offset of row 0 in each work array
  int32_t nt, np, pitch, shape;
  int32_t geo;     // first row of the geometry table (the shape's, or the realization's own
                   // with a grid-based diffusivity folded into cN, cS, cE)
  int32_t flow;    // first row of this realization's flow table
  int32_t col;     // first entry of the shape's cos/sin(phi_k) tables
  int32_t poff;    // offset of this realization's ring-sum partials (doubles, fused RKL2)
  int32_t band;    // rows per band of the fused RKL2 work items (the shape's tuned choice)
};

// Per-row geometry of a shape (uniform grid, Sec. 3.2).
template <typename T> struct RowGeo {
  T cN;        // sin(th_{j-1/2}) / (dth^2 sin th_j)   (Eq. diffusion_matrix a_{j-1,k} / nu)
  T cS;        // sin(th_{j+1/2}) / (dth^2 sin th_j)   (a_{j+1,k} / nu)
  T cE;        // 1 / (dph^2 sin^2 th_j)               (a_{j,k+-1} / nu)
  T cC;        // -(cN + cS + 2 cE) in T               (a_{j,j} / nu); cN..cC are one 16-B vector in FP32
  T inv_sdth;  // 1 / (sin th_j dth)
  T inv_sdph;  // 1 / (sin th_j dph)
  T sdn;       // sin th_{j-1/2}
  T sup;       // sin th_{j+1/2}
};

// Per-row FP64 geometry for the reductions.
struct RowGeoD {
  double area;   // area of one stored entry: sin th_j dth dph, or cap/np on a pole row
  double cos_t;  // cos th_j
  double sin_t;  // sin th_j
  double lat;    // latitude of row j (rad)
};

// Per-row flow of a realization (Eq. dr, Eq. mf, code units).
template <typename T> struct RowFlow {
  T vdn;    // v_theta at face j-1/2
  T vup;    // v_theta at face j+1/2
  T vp;     // v_phi on row j
  T alpha;  // LLF alpha_j = max |v_theta| over faces j-5/2..j+5/2 (App. B)
};

struct ShapeConst {
  double pole_diff;  // sin(dth/2) dph / (dth * cap)  (times nu: diffusion cap operator)
  double pole_adv;   // sin(dth/2) dph / cap          (advection cap operator)
  double dth, dph;
};

// Per-realization parameters of one time step.
struct StepParam {
  double dt;        // hours; 0 = idle this step
  double dt_adv;    // hours of one advection advance: dt (Lie) or dt/2 (Strang)
  double nudt;      // nu * dt (R_sun^2)
  double eps_t;     // WENO eps in the theta sweep
  double eps_p;     // WENO eps in the phi sweep
  double alpha_uw;  // UW/CD factor
  double inv_b0;    // 1 / B_0 of Eq. (flow_attenuation); 0 = no attenuation
  double cap_nu;    // nu at the cap faces relative to nudt: 1 (constant nu), nu_g(theta_1/2) (Eq. diffgrid)
  int32_t s;        // RKL2 stages (0 = no diffusion)
  int32_t coef;     // index of this realization's stage-0 coefficients
  int32_t weno;     // 1 = WENO3-CS(h), 0 = UW
  int32_t adv;      // 1 = advection on for this realization
};

// RKL2 stage coefficients in increment form (see rkl2_stage_kernel).
template <typename T> struct Coef {
  T mu, nu, mut, gsum;  // mu_j, nu_j, mu~_j, mu~_j + gamma~_j
};

// kind & 3: 0 interior, 1 north cap, 2 south cap.  kind >> 8: log2 of the
// threads per tile row (256 threads = TR rows x 256/TR threads), so tiles of
// different heights (one per grid shape) run in the same launch.
struct Tile {
  int32_t r;     // realization
  int32_t j0;    // first row (interior tiles)
  int32_t k0;    // first longitude (interior tiles)
  int32_t kind;
};

// Advection stage: out = a * fn + b * fin - c * dt * F_A(fin)   (Sec. 3.6.2)
template <typename T> struct AdvStage {
  const T* fin;
  const T* fn;
  T* out;
  int fin_work, fn_work, out_work;  // 1: array is a work array (use woff), 0: the state pool
  T a, b, c;
};

// Launch wrappers (defined in sft_kernels.cu).
template <typename T>
cudaError_t launch_rkl2_stage(int n_tiles, cudaStream_t st, const Tile* tiles, const RealDesc* rd,
                              const StepParam* sp, const RowGeo<T>* geo, const ShapeConst* shc,
                              const Coef<T>* coef, T* B, T* G, T* D0, T* D1, int stage,
                              int allow_final, int* status);
template <typename T>
cudaError_t launch_adv_stage(int n_tiles, cudaStream_t st, const Tile* tiles, const RealDesc* rd,
                             const StepParam* sp, const RowGeo<T>* geo, const RowFlow<T>* flow,
                             const ShapeConst* shc, T* state, T* work_base0, T* work_base1,
                             AdvStage<T> s);
// Fused RKL2: K stages per launch (see rkl2_fused_kernel in sft_kernels.cu).
#ifndef SFT_FUSED_K
#define SFT_FUSED_K 8
#endif
#ifndef SFT_FUSED_MINB
#define SFT_FUSED_MINB 2
#endif
#ifndef SFT_FUSED_BAND
#define SFT_FUSED_BAND 256
#endif
namespace fused {
constexpr int K = SFT_FUSED_K;   // RKL2 stages per pass
constexpr int LANES = 32;
constexpr int HL = (K + 3) / 4;  // phi-halo lanes on each side of a strip (4 columns each, >= K)
constexpr int STRIP = 4 * (LANES - 2 * HL);  // output columns of one warp strip (lanes HL..31-HL)
constexpr int WARPS = 4;         // strips per block
constexpr int THREADS = WARPS * LANES;
constexpr int MIN_BLOCKS = SFT_FUSED_MINB;  // blocks per SM the register budget is sized for
#ifndef SFT_FUSED_D
#define SFT_FUSED_D 8
#endif
constexpr int D = SFT_FUSED_D;   // rows of asynchronous-copy lookahead per warp (a power of 2)
// G and coefficient rings: row r in slot r mod RG; slots 0..MG-1 are also
// mirrored after the ring (slot RG + x), so the K rows t-1..t-K a row step
// reads always sit at P - 1 .. P - K for one base slot P (no wrap).
constexpr int RG = D + K;        // ring period: rows t-K .. t+D-1 live at once
constexpr int MG = K - 1;        // mirrored slots
constexpr int GSLOTS = RG + MG;  // slots of the G ring and of the coefficient table
constexpr int RING_F4 = (2 * D + GSLOTS) * LANES;  // float4 slots of one warp's rings (C, A, G)
constexpr int TAB_F4 = (GSLOTS + 1) * 2 * K;       // one warp's table: per slot K levels x (ka, kb), + a spare slot
// Band height of a grid before the autotuner has chosen one: 256 rows from
// 512 rows up (fewer band-overlap rows), 128 below (more work items).
__host__ __device__ constexpr int default_band_rows(int nt) { return nt >= 512 ? SFT_FUSED_BAND : 128; }
constexpr int POLE_F4 = (2 * K + 3) / 4;           // one warp's pole values (north, south)
constexpr size_t kSmemBytes = sizeof(float4) * (RING_F4 + TAB_F4 + POLE_F4) * WARPS;
static_assert((D & (D - 1)) == 0 && RG >= D + K && MG >= K - 1, "ring sizes");
static_assert(4 * K <= LANES, "at most one coefficient of a row per lane");
// Bands of a grid: rows 1 .. nt-2 in bands of `band` rows (>= 2K).
__host__ __device__ constexpr int n_bands(int nt, int band) { return (nt - 2 + band - 1) / band; }
__host__ __device__ constexpr int n_strips(int np) { return (np + STRIP - 1) / STRIP; }
// A grid shape can use the fused path when the K rows next to each pole are
// disjoint and inside one band, and a strip is at least its halo wide.
inline bool shape_ok(int nt, int np) { return nt >= 2 * K + 4 && np >= 16; }
// Per realization, the ring-sum partials of the rows next to the poles
// (doubles): 2 buffers x 2 poles x 2 inputs, then G, x K rows x strips.
inline int64_t part_elems(int np) { return 10ll * K * n_strips(np); }
}  // namespace fused

// Stages j0 .. j0+K-1 of every realization with s >= j0 (fewer, ending with
// the final write B += delta_s, for a realization whose s ends inside the
// launch).  Reads delta_{j0-2} (Dm2, zero when j0 == 2), delta_{j0-1} (Dm1),
// G; writes delta_{j0+K-2} (Om2) and delta_{j0+K-1} (Om1), rows 0 .. nt-1.
// part: ring-sum partials (desc.poff), read from buffer pin, written to
// buffer 1-pin for the next launch.  launch_ring_sums fills buffer 0 and the
// G partials from stage 1's output and G before the first launch of a step
// (tiles: a north and a south tile per realization).
cudaError_t launch_rkl2_fused(int n_tiles, cudaStream_t st, const Tile* tiles, const RealDesc* rd,
                              const StepParam* sp, const RowGeo<float>* geo, const ShapeConst* shc,
                              const Coef<float>* coef, float* B, const float* G, const float* Dm2,
                              const float* Dm1, float* Om2, float* Om1, double* part, int pin, int j0,
                              int* status);
cudaError_t launch_ring_sums(int n_tiles, cudaStream_t st, const Tile* tiles, const RealDesc* rd,
                             const float* D1, const float* G, double* part);
cudaError_t prepare_rkl2_fused();

template <typename T>
cudaError_t launch_fix_poles(int n_real, cudaStream_t st, const RealDesc* rd, T* state, int only_r);

// Reductions: one block per (realization, band of rows); partial results
// per block; a second kernel folds them per realization in a fixed order.
enum RedMode { RED_DIAG = 0, RED_ASSIM = 1, RED_BALANCE = 2 };

// Random flux emergence of one step (Sec. 2.4), per realization: source maps
// m0 .. m0+3 (the map indices of Eq. rfe_s) and their weights in hours, wa
// for the step's first source application, wb for the second (Lie: one
// application after D; Strang: one before the first and one after the second
// advection).  c: Eq. (rfe_m2)'s G/hour per unit normal draw, or for Eq.
// (rfe_m1) the same times the cell area (divided by it per cell).
struct RfeStep {
  int32_t method;   // 0 off (or idle this step), 1 Eq. rfe_m1, 2 Eq. rfe_m2
  int32_t fresh;    // 1: (re)compute the Eq. (fluxbal) factors of maps m0..m0+3 this step
  int64_t m0;
  uint64_t seed;
  double c;
  double wa[4], wb[4];
};
constexpr int kDiagFields = 14;

struct RedTile {
  int32_t r, j0, j1, pad;  // rows [j0, j1)
};

// Observed maps and mu maps in caller layout [nt][np] (pitch np); realization
// r's maps start at element obs_off[r] of obs / mu (all 0 when shared).
struct AssimArgs {
  const void* obs;
  const void* mu;
  const int64_t* obs_off;
  const double* wpar;  // per realization: alpha_mu, mu_lim, lat_lim (rad), balance flag
};

template <typename T>
// cosp / sinp: cos, sin phi_k (FP64); csf: the same as (cos hi, cos lo,
// sin hi, sin lo) float pairs, hi + lo = the FP64 value (FP32 states).
cudaError_t launch_reduce(int mode, int n_tiles, cudaStream_t st, const RedTile* tiles,
                          const RealDesc* rd, const RowGeoD* geod, const double* cosp,
                          const double* sinp, const float4* csf, const T* state, double lat_cut,
                          AssimArgs aa, double* partials);
template <typename T>
cudaError_t launch_rfe_sums(int n_tiles, cudaStream_t st, const RedTile* tiles, const RealDesc* rd,
                            const RowGeoD* geod, const RfeStep* rs, double* partials);
cudaError_t launch_rfe_fold(int n_real, cudaStream_t st, const int* tile_start, const RfeStep* rs,
                            const double* partials, double* fac);
template <typename T>
cudaError_t launch_rfe_apply(int n_tiles, cudaStream_t st, const RedTile* tiles, const RealDesc* rd,
                             const RowGeoD* geod, const RfeStep* rs, const double* fac, int phase, T* state);
cudaError_t launch_fold(int mode, int n_real, cudaStream_t st, const int* tile_start,
                        const double* partials, const double* wpar, double* out);
template <typename T>
cudaError_t launch_apply(int mode, int n_tiles, cudaStream_t st, const RedTile* tiles,
                         const RealDesc* rd, const RowGeoD* geod, T* state, AssimArgs aa,
                         const double* factors);

}  // namespace sft
