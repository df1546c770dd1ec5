/*
 * sft.h -- C-ABI of libsft, a GB300 (sm_103a) implementation of the
 * surface-flux-transport (SFT) time step of HipFT (Caplan et al., "Open-source
 * Flux Transport (OFT) I. HipFT").
 *
 * The library advances the radial photospheric field Br(theta, phi) of many
 * independent realizations, each on its own uniform logically-rectangular
 * grid (Sec. 3.2), by the model of Eq. (main_model) restricted to advection,
 * diffusion and data assimilation:
 *   - advection by analytic differential rotation and meridional flow
 *     (Eq. dr, Eq. mf) with WENO3-CS(h) or upwind face fluxes (Sec. 3.6.1,
 *     App. B) and SSPRK(4,3) / SSPRK(3,3) / forward-Euler stages (Sec. 3.6.2);
 *   - diffusion with the 5-point operator of Eq. (diffusion_op) advanced by
 *     RKL2 super time stepping (Sec. 3.7.2);
 *   - finite-volume polar caps (App. A) and a periodic phi boundary;
 *   - Lie operator splitting A then D (Eq. num_opsplit_nostrang) or Strang
 *     splitting (Eq. num_opsplit_strang) with the time-step controller of
 *     Sec. 3.4;
 *   - optional flow attenuation (Eq. flow_attenuation), grid-based
 *     diffusivity (Eq. diffgrid) and random flux emergence (Sec. 2.4);
 *   - the weighted, optionally flux-balanced assimilation blend of Sec. 2.3
 *     (Eq. data_assim, data_assim_f, data_assim_deltab, fluxbal);
 *   - the analysis quantities of Sec. 2.6.
 *
 * Conventions for every call:
 *   - Maps are row-major [ntheta][nphi], phi contiguous, in the handle's
 *     precision (float for SFT_FP32, double for SFT_FP64).  ntheta counts
 *     theta points INCLUDING both poles (theta_j = j*pi/(ntheta-1)); nphi
 *     counts unique longitudes (phi_k = k*2*pi/nphi).  Rows 0 and ntheta-1
 *     are the poles; the library reads a pole's value from its k = 0 entry
 *     and always writes the whole pole row with one value.
 *   - Units are the paper's code units (Sec. 3.3): R_sun = 6.96e8 m,
 *     time in hours, Br in Gauss.
 *   - Pointers flagged on_device = 1 are CUDA device pointers of the current
 *     device; on_device = 0 means host memory.  The library copies caller
 *     arrays and never retains a caller pointer.
 *   - The handle owns all device memory it uses (allocated by
 *     sft_create_grid, freed by sft_destroy).  After sft_create_grid only
 *     these allocate: sft_step (its cached step configurations and graphs),
 *     sft_set_flows (a larger geometry table for grid-based diffusivity),
 *     sft_set_rfe (its per-realization buffers, once) and sft_assimilate
 *     (its observation buffer, when it grows).  A failed allocation returns
 *     SFT_ERR_OOM and frees what the call had allocated; the call can be
 *     repeated (after a failed sft_set_flows, sft_step waits for one that
 *     succeeds).
 *   - Work is queued on the handle's CUDA stream.  sft_get_state (host
 *     destination), sft_flux_diagnostics, sft_get_stats and sft_step with
 *     profiling on synchronise that stream; the other calls are asynchronous.
 *   - Errors are returned as sft_status codes (never abort or trap);
 *     sft_last_error() gives a one-line description.  A device-side status
 *     word (non-finite values seen by the watchdog) is checked at each
 *     synchronising call and turns into SFT_ERR_UNSTABLE.
 *   - A handle is not thread-safe; distinct handles are independent.
 */
#ifndef SFT_H_
#define SFT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SFT_ABI_VERSION 7

typedef struct sft_grid* sft_handle;

typedef enum {
  SFT_OK = 0,
  SFT_ERR_ARG = 1,      /* invalid argument; the handle is unchanged */
  SFT_ERR_OOM = 2,      /* cudaMalloc failed, or the HBM budget cannot hold one realization */
  SFT_ERR_CUDA = 3,     /* a CUDA runtime call failed (text in sft_last_error) */
  SFT_ERR_UNSTABLE = 4, /* non-finite values seen by the watchdog */
  SFT_ERR_TIMEOUT = 5,  /* reserved for bounded device waits */
  SFT_ERR_STATE = 6     /* calls out of order (e.g. sft_step before sft_set_flows) */
} sft_status;

typedef enum { SFT_FP32 = 0, SFT_FP64 = 1 } sft_prec;

/* advection spatial scheme (Sec. 3.6.1, App. B) */
enum { SFT_ADV_WENO3_CSH = 0, SFT_ADV_UPWIND = 1 };
/* advection time scheme (Sec. 3.6.2) */
enum { SFT_TIME_SSPRK43 = 0, SFT_TIME_SSPRK33 = 1, SFT_TIME_FE = 2 };
/* diffusion time scheme (Sec. 3.7.2): the RKL2 super time stepper
 * (s = min{s >= 2 : dt <= dt_E (s^2+s-2)/4} stages), RKG2(3/2) (the
 * paper's default; s = min{s >= 2 : dt <= dt_E (s^2+3s-4)/6}), or none */
enum { SFT_DIFF_RKL2 = 0, SFT_DIFF_OFF = 1, SFT_DIFF_RKG2 = 2 };
/* operator splitting of one step (Sec. 3.5): Lie, Eq. (num_opsplit_nostrang):
 * A(dt) then D(dt); Strang, Eq. (num_opsplit_strang) with the source the
 * identity: A(dt/2), D(dt), A(dt/2) -- the flow then allows twice the step */
enum { SFT_SPLIT_LIE = 0, SFT_SPLIT_STRANG = 1 };

typedef struct {
  int32_t ntheta; /* >= 5, poles included */
  int32_t nphi;   /* >= 8, unique longitudes */
} sft_shape;

/* Per-realization model and method parameters (Sec. 2.1, 2.2, 2.5, 3.6, 3.7). */
typedef struct {
  double d0, d2, d4;  /* Eq. (dr): v_phi = (d0 + d2 cos^2 + d4 cos^4) sin(theta), m/s */
  double m1, m3, m5;  /* Eq. (mf): v_theta = -(m1 cos + m3 cos^3 + m5 cos^5) sin(theta), m/s */
  double nu;          /* diffusivity, km^2/s (constant per realization), >= 0; unused when
                         nu_grid_alpha > 0 */
  double alpha_uw;    /* upwind factor of the UW/CD flux (Sec. 3.6.1); 1 = upwind */
  double cfl_safety;  /* safety factor on the flow CFL limit (Sec. 3.6.2), e.g. 0.9 */
  double eps_w;       /* WENO epsilon: <= 0 selects eps_w = h (WENO3-CS(h)), > 0 a constant */
  int32_t adv_space;  /* SFT_ADV_*  (may differ between realizations) */
  int32_t adv_time;   /* SFT_TIME_* (must be the same for all realizations) */
  int32_t diffusion;  /* SFT_DIFF_* (must be the same for all realizations) */
  int32_t advection;  /* 1 = advection on, 0 = off (then dt is limited only by the target) */
  double atten_b0;    /* Eq. (flow_attenuation): the flow is scaled by 1 - tanh(|B_r| / atten_b0)
                         where it meets the field (each flux term v B_i becomes v a_i B_i; the
                         LLF bound and the CFL limit keep the unattenuated flow), G; 0 = off,
                         otherwise > 0 (the paper's default is 500 G) */
  int32_t splitting;  /* SFT_SPLIT_* (must be the same for all realizations) */
  int32_t reserved;   /* 0 */
  double nu_grid_alpha; /* > 0: the grid-based diffusivity of Eq. (diffgrid),
                           nu_g = nu_grid_alpha [(dtheta)^2 + (dphi sin theta)^2] at the theta
                           faces of the operator (1/hour; the map smoother of Sec. 2.2), in
                           place of nu; 0 = the constant nu */
} sft_flow_params;

/* Random flux emergence of a realization (Sec. 2.4). */
typedef struct {
  int32_t method;          /* 0 off, 1 Eq. (rfe_m1): uniform unsigned flux per cell, 2 Eq. (rfe_m2):
                              uniform unsigned flux per unit area (the paper's default) */
  int32_t origin_given;    /* 0: source map 0 belongs to the realization's time at sft_set_rfe;
                              1: to origin_hours (resuming a run from a checkpoint) */
  double rate_mx_per_hour; /* total unsigned flux per hour of the source maps, Mx/hour, >= 0 */
  double lifetime_hours;   /* tau of Eq. (rfe_s), the time between source maps; <= 0 or inf: one
                              map for ever */
  uint64_t seed;           /* of the counter-based normal draws */
  double origin_hours;     /* t0 when origin_given = 1 */
} sft_rfe_params;

/* Assimilation weight and balance options (Sec. 2.3). */
typedef struct {
  double alpha_mu;    /* exponent of mu in Eq. (data_assim_f) */
  double mu_lim;      /* F = 0 unless mu > mu_lim */
  double lat_lim_deg; /* F = 0 unless |latitude| < lat_lim_deg */
  int32_t flux_balance; /* 1: balance Delta B by Eq. (fluxbal) before adding it */
  int32_t reserved;
} sft_assim_params;

/* Analysis quantities of one realization (Sec. 2.6), all accumulated in FP64. */
typedef struct {
  double flux_signed, flux_pos, flux_neg; /* Mx */
  double flux_pole_n, flux_pole_s;        /* Mx, |latitude| >= lat_cut */
  double area_pole_n, area_pole_s;        /* cm^2 */
  double brmin, brmax, absmin;            /* G */
  double dipole_axial, h1, h2;            /* G: D and h1, h2 of Eq. (eqdipole1) */
  double t_hours;                         /* the realization's simulated time */
  int64_t steps;                          /* time steps taken by the realization */
  int64_t nonfinite;                      /* number of non-finite map entries */
} sft_diag;

/* Work counters since creation or the last sft_reset_stats. */
typedef struct {
  int64_t global_steps;      /* iterations of the sft_step loop */
  int64_t realization_steps; /* sum over realizations of time steps taken */
  double cell_updates;       /* sum over realizations of ntheta*nphi*steps */
  double adv_cell_stages;    /* ntheta*nphi x advection stages executed */
  double diff_cell_stages;   /* ntheta*nphi x RKL2 stages executed */
  int64_t kernel_launches;   /* library kernels launched (graph nodes included) */
  int64_t graph_launches;    /* CUDA graph launches */
  double diff_ms;            /* with profiling on: device time of the RKL2 stages (stage 1 to the
                                last stage, both launch chains of the fused passes) */
  double adv_ms;             /* with profiling on: device time of the advection stage kernels */
  int64_t diff_launches;     /* with profiling on: RKL2 passes timed (stage 1, then one per
                                fused pass of K stages whatever the number of launch chains;
                                one per stage on the single-stage path) */
  int64_t adv_launches;      /* with profiling on: advection stage kernels timed */
  double diff_bytes;         /* algorithmic HBM bytes of the timed RKL2 stage kernels */
  double adv_bytes;          /* algorithmic HBM bytes of the timed advection stage kernels */
} sft_stats;

/*
 * Create a batch of n_real realizations; shapes[r] is realization r's grid
 * (shapes may differ: an uneven batch).  prec is the state precision.
 * hbm_budget_bytes bounds the device memory of the handle (0 = no bound):
 * the state of every realization stays resident and the time-stepping work
 * buffers are sized for the largest group of realizations ("wave") that fits
 * the rest of the budget; sft_step then advances the waves one after another.
 * SFT_ERR_OOM if the budget cannot hold the state plus one realization's
 * work buffers.  cuda_stream is the cudaStream_t all work is queued on; NULL
 * makes the handle create its own blocking stream (ordered with the legacy
 * default stream).  Maps start at zero and simulated times at 0 h.
 */
sft_status sft_create_grid(const sft_shape* shapes, int32_t n_real, sft_prec prec,
                           size_t hbm_budget_bytes, void* cuda_stream, sft_handle* out);

/* Release every device resource of the handle.  NULL is accepted. */
sft_status sft_destroy(sft_handle h);

/* Copy realization r's map in (caller layout [ntheta][nphi]).  Pole rows are
 * taken from their k = 0 entries. */
sft_status sft_set_state(sft_handle h, int32_t r, const void* br, int32_t on_device);

/* Copy realization r's map out (caller layout [ntheta][nphi]). */
sft_status sft_get_state(sft_handle h, int32_t r, void* br, int32_t on_device);

/* Set the simulated time (hours) of realization r, or of every realization
 * when r = -1 (checkpoint/resume). */
sft_status sft_set_time(sft_handle h, int32_t r, double t_hours);

/* Batched forms of sft_set_state / sft_get_state / sft_set_time for a subset
 * of realizations (an ensemble member subset, Sec. 2.5): idx[0..n) are
 * realization indices (host array, distinct for sft_set_states), all of one
 * grid shape; maps is one packed array of n maps in caller layout, map q
 * (for realization idx[q]) at element q * ntheta * nphi, on the device when
 * on_device, else in host memory; t_hours[q] (host) is idx[q]'s time.  One
 * call issues every copy on the handle's stream and, for sft_set_states, one
 * pole fix-up launch; sft_get_states with host memory synchronises.  The
 * first bad index or argument fails the call before any copy
 * (SFT_ERR_ARG). */
sft_status sft_set_states(sft_handle h, int32_t n, const int32_t* idx, const void* maps, int32_t on_device);

/* The maps of realizations idx[0..n) into the packed array maps (see above). */
sft_status sft_get_states(sft_handle h, int32_t n, const int32_t* idx, void* maps, int32_t on_device);

/* The times of realizations idx[0..n) to t_hours[0..n) (see above). */
sft_status sft_set_times(sft_handle h, int32_t n, const int32_t* idx, const double* t_hours);

/* Per-realization simulated times (host array of n_real doubles). */
sft_status sft_get_time(sft_handle h, double* t_hours);

/* Set every realization's parameters (host array of n_real structs).
 * Builds the per-realization flow tables (Eq. dr, mf), the flow CFL limit
 * (Eq. ssprk43_dt / advection_timestep times cfl_safety) and the explicit
 * diffusion limit (Gershgorin bound of the Eq. diffusion_matrix operator). */
sft_status sft_set_flows(sft_handle h, const sft_flow_params* params);

/*
 * Advance every realization to t_target_hours (Sec. 3.4, 3.5): each time
 * step is dt_r = min(t_target - t_r, CFL limit of r); advection then the
 * super time stepped diffusion (RKL2 or RKG2(3/2), s_r stages as above).
 * All realizations step in lockstep (one batched launch per stage); a
 * realization that has reached the target idles.  max_steps > 0 stops after
 * that many loop iterations.  *steps_taken (may be NULL) receives the number
 * of loop iterations.
 */
sft_status sft_step(sft_handle h, double t_target_hours, int32_t max_steps, int32_t* steps_taken);

/*
 * Assimilate observations (Sec. 2.3).  br_obs and mu are maps in the
 * handle's precision: one map per realization (obs_per_realization = 1,
 * concatenated in realization order), one map per grid shape
 * (obs_per_realization = 2, concatenated in shape order, the order of first
 * appearance in sft_create_grid's shapes), or one map shared by every
 * realization (obs_per_realization = 0; all realizations must then have the
 * same shape).  F = mu^alpha_mu where mu > mu_lim and |lat| < lat_lim, else
 * 0 (Eq. data_assim_f); Delta B = F (B_obs - B) (Eq. data_assim_deltab),
 * balanced by Eq. (fluxbal) when requested (skipped for a realization whose
 * Delta B has no positive or no negative part); then B += Delta B.
 * params: host array of n_real structs.
 */
sft_status sft_assimilate(sft_handle h, const void* br_obs, const void* mu,
                          int32_t obs_per_realization, int32_t on_device,
                          const sft_assim_params* params);

/* Multiplicatively flux-balance every realization's map (the input-map
 * option of Sec. 5.1): B > 0 divided by sqrt(r), B <= 0 multiplied by
 * sqrt(r), r = |Phi+ / Phi-| (Eq. fluxbal applied to B). */
sft_status sft_balance_flux(sft_handle h);

/* Analysis quantities of Sec. 2.6 for every realization (host array of
 * n_real structs), accumulated in FP64.  lat_cut_deg bounds the polar
 * regions.  Synchronises. */
sft_status sft_flux_diagnostics(sft_handle h, double lat_cut_deg, sft_diag* out);

/* Work counters; synchronises so profiled times are complete. */
sft_status sft_get_stats(sft_handle h, sft_stats* out);

/* Zeroes the work counters (the step state is untouched). */
sft_status sft_reset_stats(sft_handle h);

/* profile != 0: sft_step records CUDA events around its advection and RKL2
 * stage kernels on the handle's stream and accumulates their device time in
 * sft_stats (each step then synchronises). */
sft_status sft_set_profiling(sft_handle h, int32_t profile);

/* use_graphs != 0 (default): sft_step replays one captured CUDA graph per
 * distinct step configuration (captured on the configuration's second use;
 * its first use launches directly); 0: plain launches. */
sft_status sft_set_graphs(sft_handle h, int32_t use_graphs);

/* RKL2 stages per kernel launch: 1 (one launch per stage) or 8 (temporal
 * blocking: eight stages per pass through HBM; bands of rows marched by
 * warps with an eight-point halo; per pole, one block evaluates the pole
 * values of the pass over the whole ring).  The fused path needs FP32 and
 * every grid with ntheta >= 20 and nphi >= 16; it is the default when
 * available.  Both paths compute the same stages (the fused path folds the
 * stencil into per-row coefficients: another rounding order, agreement to
 * FP32 rounding). */
sft_status sft_set_fusion(sft_handle h, int32_t stages_per_pass);

/* Current RKL2 stages per launch (1 or 8). */
int32_t sft_get_fusion(sft_handle h);

/* Tile rows per block of the stage kernels for realizations of shape index
 * shape_id (order of first appearance in shapes[]); 0 lets the built-in
 * autotuner choose on the first step.  Valid values: 1, 2, 4, 8. */
sft_status sft_set_tile_rows(sft_handle h, int32_t shape_id, int32_t rows);

/* The tile rows chosen for shape_id (after autotuning), or 0 if not yet. */
int32_t sft_get_tile_rows(sft_handle h, int32_t shape_id);

/* Rows per band of the fused RKL2 work items for shape_id (a warp marches
 * one band of one strip): 0 = chosen by the built-in autotuner on the first
 * step (one timed launch per candidate 64, 128, 256, 512), else rows > 8.
 * Results do not depend on it. */
sft_status sft_set_band_rows(sft_handle h, int32_t shape_id, int32_t rows);

/* The band rows chosen for shape_id (after autotuning), or 0 if not yet. */
int32_t sft_get_band_rows(sft_handle h, int32_t shape_id);

/* Number of realizations per wave for the handle's HBM budget. */
int32_t sft_wave_size(sft_handle h);

/* The flow CFL limit of one advection advance (hours; a Strang step may be
 * twice as long, its two advances being half steps) and the RKL2 stage count
 * for a step of dt hours of realization r, as sft_step would use them.
 * Host-only computation. */
sft_status sft_step_plan(sft_handle h, int32_t r, double dt_hours, double* dt_cfl, double* dt_euler,
                         int32_t* stages);

/*
 * Flux diagnostics of one map that the caller keeps in its own device memory,
 * without allocating any device memory.  No counterpart in the paper: this
 * exists for callers that cannot call cudaMalloc while they run (a solver
 * coupled into a model that has already reserved the device memory through
 * its own pool, or a real-time pipeline that forbids allocation after
 * start-up because cudaMalloc can stall the device).
 *
 * br_device: device pointer to a [ntheta][nphi] map (pitch nphi) in
 * precision prec; the grid convention is that of every other call.  The
 * result (the sft_diag of sft_flux_diagnostics, with t_hours = steps = 0) is
 * written to the host struct *out; the call synchronises cuda_stream (NULL =
 * legacy default stream).
 * Scratch: one fixed file-scope device array of SFT_NOALLOC_SCRATCH_BYTES
 * (held by every GPU that loads the library until the process exits).  A map
 * whose tables and partial sums do not fit is rejected with SFT_ERR_ARG
 * (roughly up to 8192 x 16384).  Every call looks up the array's address in
 * the current context (cudaGetSymbolAddress, which allocates nothing).  With
 * lazy module loading (CUDA's default) the first call in a context also
 * loads the library's device code and commits the array's memory: make one
 * call at start-up, before a memory pool reserves the device, or set
 * CUDA_MODULE_LOADING=EAGER.  All calls share the array, so calls that
 * overlap on the GPU race; errors are reported through sft_last_error(NULL).
 */
#define SFT_NOALLOC_SCRATCH_BYTES (4u << 20)

/* Flux diagnostics of one caller-owned device map without device allocation
 * (no counterpart in the paper), as described above. */
sft_status sft_flux_diagnostics_noalloc(const void* br_device, int32_t ntheta, int32_t nphi,
                                        sft_prec prec, double lat_cut_deg, void* cuda_stream,
                                        sft_diag* out);

/* One-line description of the last error on h (or of the last failed
 * sft_create_grid or handle-free call when h is NULL).  Valid until the next
 * call on h. */
const char* sft_last_error(sft_handle h);

/*
 * Random flux emergence (Sec. 2.4), params[r] per realization (NULL: off for
 * all).  Source map k of a realization is Eq. (rfe_m1) or Eq. (rfe_m2) from
 * standard normal draws (counter-based in seed, map and cell: the SplitMix64
 * output function of two states per cell and Box-Muller; each polar cap is
 * one cell), flux balanced as Eq. (fluxbal); map k belongs to time
 * t0 + k tau with t0 the realization's time at this call (or origin_hours),
 * and Eq. (rfe_s)
 * interpolates linearly between maps.  Every step adds the exact time
 * integral of that source over the step: after the diffusion advance (Lie),
 * or half before the first and half after the second advection advance
 * (Strang).  A finite lifetime caps the time step at tau.  Nothing is stored
 * per map: each step regenerates the (at most four) maps it needs, so a run
 * resumed from a checkpoint (state, time, and these parameters with the
 * original origin) continues bit for bit.
 */
sft_status sft_set_rfe(sft_handle h, const sft_rfe_params* params);

/* ---- Debug build and host fault injection ------------------------------
 * The library built with -DSFT_DEBUG (libsft_debug.so) checks, inside the
 * stepping and reduction kernels, every index a kernel derives from its
 * tile and realization descriptor (row, first column, first and last row
 * of a fused band, rows of a reduction tile) against the range that keeps
 * all its accesses inside the realization.  A failed check records the
 * check site and the offending value on the device and clamps or skips the
 * access; nothing traps.  The release build compiles the checks away, and
 * both builds check the host-built descriptor and tile tables whenever
 * they are built (SFT_ERR_STATE on an inconsistency, before any launch).
 */

/* Reads the device record: *first_failure = (site << 48) | (value mod 2^48)
 * of the first failed check, 0 when none; *failures = number of failed
 * checks (either pointer may be NULL).  reset != 0 clears the record.
 * Synchronises the device.  SFT_ERR_STATE in a release build. */
sft_status sft_debug_checks(uint64_t* first_failure, uint32_t* failures, int32_t reset);

/* Runs one check on the device, value against [lo, hi], with no memory
 * access: a self-test of the record path (site 1..65535, lo <= hi).
 * Synchronises the device.  SFT_ERR_STATE in a release build. */
sft_status sft_debug_probe(int32_t site, int64_t value, int64_t lo, int64_t hi);

/* Host fault injection, in every build: the nth device or pinned allocation
 * made by an sft_* call from now on (1 = the next) reports an allocation
 * failure without allocating; the call that makes it returns SFT_ERR_OOM
 * and frees what it had allocated, and the same call made again succeeds
 * (sft_step after a failed sft_set_flows waits for a successful one).
 * 0 disarms.  Process-wide. */
sft_status sft_debug_fail_alloc(int32_t nth);

/* SFT_ABI_VERSION of the loaded library. */
int32_t sft_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SFT_H_ */
