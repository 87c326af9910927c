/* imexds: explicit-implicit domain splitting for 1-D isothermal two-phase flow with phase transition
 * (May & Thein, arXiv 2211.00705), on one NVIDIA GB300 (sm_103a), FP64 throughout.
 *
 * One time step (Algorithm 1) is: the CFL time step (Eq. cfl_cond:unif); an explicit HLL sweep over
 * every cell away from the tiny cells (Algorithm 1, Step 1); and, on the neighbourhood {k-1, k, k+1}
 * of every tiny cell k next to a phase boundary, dual time stepping (Algorithm 2, Eq. dual time tau
 * diff) with the phase-boundary Riemann solver of App. A at the implicit faces, followed by the
 * conservative re-flux of Algorithm 2 Part 2 on the moving grid (Eq. godunov_meth:nonunif, Sec. 3.4).
 * Grid management (merge/split of cells next to a boundary, Sec. 2.3/3.4) and phase creation
 * (App. B) run inside the step.
 *
 * Units: SI. Phase labels: 0 = vapour, 1 = liquid. A state is (rho, m = rho u) per cell.
 *
 * Conventions of every call:
 *   - every function returns an imexds_status; nothing throws across this interface;
 *   - host pointers belong to the caller and are only read/written during the call;
 *   - device memory is owned by the context (allocated in imexds_create, freed in imexds_destroy);
 *   - the library works on the CUDA stream given to imexds_create (0 = the legacy default stream)
 *     and returns after the work is complete unless a function says otherwise;
 *   - a context is used by one host thread at a time.
 */
#ifndef IMEXDS_H
#define IMEXDS_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct imexds_ctx imexds_ctx; /* opaque, owned by the library */

typedef enum {
  IMEXDS_OK = 0,
  IMEXDS_ERR_ARG = 1,          /* invalid argument (sizes, a fixed face off the lattice, NULL) */
  IMEXDS_ERR_CUDA = 2,         /* a CUDA call failed; imexds_last_error_string() has the text */
  IMEXDS_ERR_NONPHYSICAL = 3,  /* rho <= 0, width <= 0 or a non-finite state after a step */
  IMEXDS_ERR_PB_NOCONV = 4,    /* the phase-boundary (or phase-creation) Newton iteration failed */
  IMEXDS_WARN_DTS_MAXITER = 5, /* dual time stepping hit l_max (the last iterate was used) */
  IMEXDS_ERR_VANISH = 6,       /* a cell between two phase boundaries would vanish (not treated) */
  IMEXDS_ERR_TIMEOUT = 7,      /* a bounded device wait gave up */
  IMEXDS_ERR_STATE = 8,        /* call order (e.g. step before set_states) */
  IMEXDS_ERR_CAPACITY = 9      /* a zone or the zone pool of an instance is full */
} imexds_status;

/* Equation of state of one phase (Sec. 4, Eq. eos:isoT_idgas and eos:isoT_lintait):
 *   kind 0 (ideal gas):   p = a2 * rho
 *   kind 1 (linear Tait): p = p0 + a2 * (rho - rho0)       (a2 = K0 / rho0)
 * a2 is the squared isothermal sound speed. */
typedef struct {
  int kind;
  double a2, p0, rho0;
} imexds_eos;

/* Two-phase fluid. p_sat is the saturation pressure, where both Gibbs energies g = a2 ln(rho/rho_sat)
 * vanish (Sec. 2.1: the Maxwell construction makes them equal there). p_min / p_tilde are the
 * cavitation / nucleation thresholds of App. B (Table tab:max_vap_lintait363). */
typedef struct {
  imexds_eos vapour, liquid;
  double p_sat, p_min, p_tilde;
} imexds_fluid;

/* Scheme options. NULL in imexds_create selects the defaults listed. */
typedef struct {
  double cfl;          /* C_CFL of Eq. cfl_cond:unif (0.5) */
  double theta_nb;     /* theta of Alg. 2 for cells of width h; theta_i = min(theta_nb, h_i/h) (0.9, Sec. 4) */
  double tol_nb, tol_k;/* dual-time stop tolerances of Sec. 4 for neighbours / tiny cells (1e-3, 1e-1) */
  int res_mode;        /* 0: residual as printed in Sec. 4 (1/s); 1: residual times dt (0) */
  int l_max;           /* cap on dual-time iterations per block and step (10000) */
  double newton_tol;   /* relative step tolerance of the phase-boundary Newton iteration (1e-12) */
  int newton_itmax;    /* cap on Newton iterations (50) */
  double alpha_min;    /* a boundary cell predicted below max(alpha_min h, h_i/2) is merged (1e-8) */
  double split_ratio;  /* a boundary cell wider than split_ratio * h is split (2) */
  int creation;        /* 1: detect cavitation / nucleation at same-phase faces (App. B) (0) */
  int zone_capacity;   /* zone records per instance (0 = automatic: 4 + 2 * phase boundaries) */
  int schedule;        /* 0 automatic, 1 one launch per kernel and step (graph of 8 steps), 2 instance
                          groups advanced by one resident launch in lockstep, 3 instance groups whose
                          instances advance independently inside the resident launch (0) */
  int group_cells;     /* lattice cells per instance group (0 = 16384, or total cells / SMs when the batch
                          is too small to fill every SM with 16384-cell groups) */
  int group_threads;   /* threads per group CTA, a multiple of 32 from 64 to 256 (0 = 128): warp 0 runs
                          the per-instance work, the other warps sweep; above 128 one CTA per SM (the
                          independent-group schedule 3 takes at most 128) */
  int block_solver;    /* solver of each implicit block's system of Algorithm 2 Part 1: 0 dual time stepping
                          (Alg. 2, Eq. dual time tau diff); 1 Newton's method on the same system with the same
                          stop test of Sec. 4 (the outlook of Sec. 5), the iteration counters then counting
                          Newton steps (0) */
} imexds_options;

/* A batch of independent 1-D problems on [x_left[i], x_right[i]] with n_lattice[i] background
 * cells of width h_i = (x_right - x_left)/n_lattice and kinetic coefficient tau[i] > 0 of the kinetic
 * relation z = tau p_V [[g + e_kin]] (Eq. isoT:kin_rel1). Arrays have n_inst entries. */
typedef struct {
  int32_t n_inst;
  const int32_t* n_lattice;
  const double* x_left;
  const double* x_right;
  const double* tau;
  imexds_fluid fluid;
} imexds_problem;

/* Create a context on the current CUDA device. `stream` is a cudaStream_t (NULL = default stream).
 * Copies everything it needs from `prob`/`opts`. On error *out is NULL. */
imexds_status imexds_create(const imexds_problem* prob, const imexds_options* opts, void* stream,
                            imexds_ctx** out);

/* Load the initial cell lists (host arrays). Instance i owns cells [cell_offsets[i], cell_offsets[i+1])
 * of widths/rho/m/phase. A face between cells of different phase is a phase boundary (Sec. 2.3); every
 * other face must lie on the background lattice (face positions accumulate the widths from the last
 * fixed face; tolerance 1e-9 h), and a cell with two fixed faces must be one background cell.
 * cell_offsets[0] = 0 and every instance holds at least one cell; rho > 0 and finite, m finite, widths
 * > 0, phase 0 (vapour) or 1 (liquid). Sets t = t0 for all instances and resets statistics.
 * IMEXDS_ERR_ARG on a malformed list (nothing is changed then). */
imexds_status imexds_set_states(imexds_ctx* ctx, const int32_t* cell_offsets, const double* widths,
                                const double* rho, const double* m, const uint8_t* phase, double t0);

/* Number of cells of every instance now (host array of n_inst entries). IMEXDS_ERR_STATE before
 * imexds_set_states. */
imexds_status imexds_cell_counts(imexds_ctx* ctx, int32_t* counts);

/* Copy the cell lists back (host arrays sized from imexds_cell_counts; cell_offsets has n_inst+1
 * entries). t and inst_status have n_inst entries; inst_status holds an imexds_status per instance: an
 * instance that met an error (IMEXDS_ERR_NONPHYSICAL, _PB_NOCONV, _VANISH, _CAPACITY) stopped in the
 * step where it occurred; its states are then not meaningful. IMEXDS_ERR_STATE before
 * imexds_set_states. The lists are packed on the device into a staging buffer the context keeps (allocated on
 * the first call, 25 B per cell) and copied once; pinned host arrays copy fastest. */
imexds_status imexds_get_states(imexds_ctx* ctx, int32_t* cell_offsets, double* widths, double* rho,
                                double* m, uint8_t* phase, double* t, int32_t* inst_status);

/* Advance every instance by n_steps time steps of Algorithm 1 (each with the CFL time step of
 * Eq. cfl_cond:unif over the instance's cells, Algorithm 2 on every implicit neighbourhood, grid
 * management and, with options.creation, phase creation of App. B), without clipping to an end time.
 * Instances that met an error stop and report it through imexds_get_states; the call itself returns
 * IMEXDS_OK unless an argument, the call order (IMEXDS_ERR_STATE before imexds_set_states) or CUDA
 * failed. */
imexds_status imexds_step(imexds_ctx* ctx, int32_t n_steps);

/* Advance every instance until t = t_end: the steps of imexds_step, the last step of each instance
 * shortened to land on t_end (its time step is min(C h / S_max, t_end - t)). Finished instances idle.
 * IMEXDS_ERR_TIMEOUT if some instance has not arrived after 2e7 steps; errors otherwise as imexds_step. */
imexds_status imexds_run_to(imexds_ctx* ctx, double t_end);

/* Per-instance counters (n_inst x 10, int64, row-major): steps, dual-time iterations, max dual-time
 * iterations in one step, Newton iterations, merges, splits, creations, l_max warnings, boundary
 * solves, kernel launches of the last call (same value in every row). */
imexds_status imexds_get_stats(imexds_ctx* ctx, int64_t* stats);

/* Device-resident variant of imexds_set_states for callers that keep the cell lists in GPU memory: the
 * same arguments as device pointers (cell_offsets stays a host array, checked before any copy:
 * cell_offsets[0] = 0 and at least one cell per instance, else IMEXDS_ERR_ARG). The copies run on the
 * context's stream; the lists are then checked as by imexds_set_states. */
imexds_status imexds_set_states_device(imexds_ctx* ctx, const int32_t* cell_offsets_host,
                                       const double* widths_d, const double* rho_d, const double* m_d,
                                       const uint8_t* phase_d, double t0);

/* Device-resident variant of imexds_get_states: the cell lists are written into DEVICE arrays widths_d, rho_d,
 * m_d, phase_d (sized from imexds_cell_counts) by kernels on the context's stream, in the order of
 * imexds_get_states; cell_offsets (n_inst + 1), t and inst_status (n_inst) are host arrays. No per-cell data
 * passes through the host. Returns after the copies are complete. */
imexds_status imexds_get_states_device(imexds_ctx* ctx, int32_t* cell_offsets, double* widths_d, double* rho_d,
                                       double* m_d, uint8_t* phase_d, double* t, int32_t* inst_status);

/* Restore the states (and t0) given to the last imexds_set_states, on the device (device-to-device
 * copies only). */
imexds_status imexds_reset(imexds_ctx* ctx);

/* Measurement of the group schedule (timing mode): SM clock cycles per phase of the resident kernel, for
 * the group whose launch took the most cycles (slowest6) and summed over all groups (sum6). Arrays of 6:
 * 0 boundary solves + plan, 1 sweep (first sweep warp), 2 dual time or Newton (warp 0), 3 grid management,
 * 4 the concurrent phase of 1 and 2 (barrier to barrier), 5 the whole launch. With the lockstep groups,
 * 0 + 4 + 3 equals 5 up to the loop's own instructions and, by design, 1, 2 <= 4; with Newton on the blocks
 * at full size 1 has been measured above 4 by about 3 (the wait for the longer sweep appears to be counted in 3), so
 * there the split between 4 and 3 is not reliable, while 5 is; with the independent groups (schedule
 * 3) each entry is the maximum over the group's instances, 4 being dual time plus the wait for the sweep.
 * The counters accumulate over the timing-mode calls since the last imexds_set_kernel_timing. */
imexds_status imexds_get_group_phase_cycles(imexds_ctx* ctx, int64_t* slowest6, int64_t* sum6);

/* Choose the schedule for the next calls (values of imexds_options.schedule, 0..3). */
imexds_status imexds_set_schedule(imexds_ctx* ctx, int32_t schedule);

/* Measurement: with on != 0, steps are launched without the step graph and CUDA events are recorded
 * around each kernel; imexds_get_kernel_times returns, per kernel (0 pre-solve, 1 plan, 2 sweep,
 * 3 dual time, 4 post, 5 group-resident kernel), the summed duration in ms and the number of timed
 * launches since timing was switched on. Arrays have 6 entries. Every call of imexds_set_kernel_timing zeroes
 * those durations and counts and the group phase cycles. With a group schedule (2, 3) timing changes no launch
 * (events around the resident kernel; its phase counters are written at its end); the first timed call of a
 * context allocates the counters. */
imexds_status imexds_set_kernel_timing(imexds_ctx* ctx, int32_t on);
imexds_status imexds_get_kernel_times(imexds_ctx* ctx, double* total_ms, int64_t* launches);

/* One explicit time step that allocates no GPU memory, for callers that cannot call cudaMalloc: code
 * running inside a memory-pool-restricted or pre-reserved environment, or a host program that must not
 * grow its GPU footprint after start-up. The paper has no counterpart: this is the library's explicit
 * HLL sweep and CFL time step, restricted to instances that contain no phase boundary (one phase in
 * every cell), with the same arithmetic as imexds_step.
 *
 * Arguments: fluid and cfl as in imexds_create; n_lattice, x_left, x_right: HOST arrays of n_inst
 * entries (instance i has n_lattice[i] >= 2 cells of width (x_right - x_left)/n_lattice); rho_in, m_in,
 * phase: DEVICE arrays of the concatenated cells (instance after instance); rho_out, m_out: DEVICE
 * arrays of the same size receiving the states after one step (they must not overlap the inputs);
 * dt_out: DEVICE array of n_inst receiving each instance's time step; stream: a cudaStream_t (NULL =
 * default stream).
 *
 * The call is synchronous: it copies the host arrays with cudaMemcpyAsync, launches its kernels, reads an
 * error flag back and waits for the stream before it returns. None of these is allowed while a stream is
 * being captured, so never make this call during a stream capture.
 *
 * Errors: IMEXDS_ERR_ARG (imexds_last_error_string says which) for a NULL pointer, cfl <= 0, n_inst <= 0,
 * an instance with fewer than 2 cells or x_right <= x_left, and, found on the device, a phase byte above 1,
 * a density that is not positive and finite, a non-finite momentum, or an instance holding cells of both
 * phases. When the device check fails, rho_out and m_out are not written (dt_out is, but is meaningless).
 *
 * Scratch: a fixed device array of about 0.7 MB inside the library, which every GPU that loads the
 * library holds until the process exits; it limits n_inst to 16384 (larger batches are rejected with
 * IMEXDS_ERR_CAPACITY before any work, see imexds_last_error_string). The first call on a device looks
 * up that array's address (cudaGetSymbolAddress) with the device current. Every call reuses the same
 * array and leaves its contents behind, so calls that may overlap on the GPU (other streams, other host
 * threads) race: serialise them. */
imexds_status imexds_step_uniform_noalloc(const imexds_fluid* fluid, double cfl, int32_t n_inst,
                                          const int32_t* n_lattice, const double* x_left, const double* x_right,
                                          const double* rho_in, const double* m_in, const uint8_t* phase,
                                          double* rho_out, double* m_out, double* dt_out, void* stream);

/* Diagnostic: the library's quotient a / b (a times the Newton-Raphson-refined reciprocal of b, used for
 * the lattice velocity and the HLL weights) and CUDA's division on n host pairs; results in fast and ref. */
imexds_status imexds_check_div(int32_t n, const double* a, const double* b, double* fast, double* ref);

/* Diagnostic: the library's dual-time stop test of one component, |d| < lim max(|w|, 1) (Sec. 4's residual
 * test with the tolerance folded into lim > 0), decided on IEEE bit patterns in integer instructions, and the
 * same test in FP64 comparisons, on n host triples (d, w, lim); 0/1 results in fast and ref. The two agree
 * for every non-NaN d and w and finite lim > 0. */
imexds_status imexds_check_tol(int32_t n, const double* d, const double* w, const double* lim, uint8_t* fast,
                               uint8_t* ref);

/* Diagnostic: evaluate the library's table-driven logarithm (Tang's method, used in the boundary
 * solves) and CUDA's log on n host values x > 0; results in the host arrays fast and ref. */
imexds_status imexds_check_log(int32_t n, const double* x, double* fast, double* ref);

/* ---- discrete adjoint ----
 * Gradient of a loss J of the final cell states of the last forward run (the imexds_step / imexds_run_to
 * calls since the last imexds_set_states or imexds_reset) with respect to the initial cell states, the
 * initial widths (which place the phase boundaries) and the kinetic coefficient tau of each instance.
 * The paper has no adjoint; this differentiates its discrete scheme (Algorithm 1 / Algorithm 2 with the
 * App. A boundary solver) along the replayed trajectory, with every decision frozen (CFL argmax cell,
 * merges, implicit blocks, splits): the explicit sweep by its transposed HLL Jacobians, each block's
 * converged dual-time system by one transposed solve (implicit function theorem, not by unrolling the
 * pseudo-iterations), the boundary flux by the implicit function theorem on the 2x2 system of
 * Eq. 2p_RP:ex_sys, phase creation (App. B) through the created cell, the per-side fluxes and moving
 * faces at the creation face and the implicit function theorem on the 3x3 creation system, forward states
 * checkpointed every k steps and recomputed per segment. The gradient is that of the converged implicit
 * system: use tight dual-time tolerances when it is compared with finite differences of the forward run.
 * An instance whose replay does not reproduce the forward run (steps, cells, or a grid event of its
 * reverse) reports IMEXDS_ERR_STATE (imexds_adjoint_replay says where).
 *
 * Inputs (host arrays in imexds_get_states order, sized from imexds_cell_counts): dJ_drho_T, dJ_dm_T
 * and dJ_dw_T (may be NULL: J independent of the widths). Outputs (host arrays in imexds_set_states
 * order): dJ_drho0, dJ_dm0, dJ_dw0 (may be NULL; zero for cells with two fixed faces, whose width is
 * the lattice's; for a cell next to a boundary it moves that boundary with the width), dJ_dtau
 * (n_inst), inst_status (n_inst, may be NULL): IMEXDS_OK, or why the instance has no gradient (its
 * entries are NaN). The replay uses the context's options; device memory for the checkpoints and the
 * tape of one segment is allocated on the first call and kept (about (38 n_ck + 26 k) bytes per cell
 * slot). */
imexds_status imexds_adjoint(imexds_ctx* ctx, const double* dJ_dw_T, const double* dJ_drho_T,
                             const double* dJ_dm_T, double* dJ_dw0, double* dJ_drho0, double* dJ_dm0,
                             double* dJ_dtau, int32_t* inst_status);
/* Device-resident variant of imexds_adjoint: the seeds dJ_dw_T (may be NULL), dJ_drho_T, dJ_dm_T and the outputs
 * dJ_dw0 (may be NULL), dJ_drho0, dJ_dm0, dJ_dtau are DEVICE arrays in the same orders and sizes; inst_status is
 * a host array (may be NULL). The seeds are scattered, the replay is checked and the gradients are assembled by
 * kernels, so no per-cell data passes through the host (the library uploads its own copy of the initial lists
 * of the last imexds_set_states, as imexds_adjoint does). imexds_adjoint_replay then reports the stop sites
 * only (its cell lists are empty). Returns after the gradients are complete. */
imexds_status imexds_adjoint_device(imexds_ctx* ctx, const double* dJ_dw_T, const double* dJ_drho_T,
                                    const double* dJ_dm_T, double* dJ_dw0, double* dJ_drho0, double* dJ_dm0,
                                    double* dJ_dtau, int32_t* inst_status);
/* Checkpoint interval k of the adjoint (default 64). The adjoint replays the forward run, keeping a copy of the
 * cell lists every k steps, and recomputes each k-step segment with a tape before reversing it; the last segment
 * is taped during the replay. Device memory grows with k (per instance and taped step about 26 B per cell slot
 * plus a 1.7 KB step record; per checkpoint about 54 B per slot); with k at least the run's step count the run
 * is taped once and nothing is recomputed (1024 instances x 565 slots x 2000 steps: 35 GB). */
imexds_status imexds_set_adjoint_checkpoint(imexds_ctx* ctx, int32_t every);
/* The last imexds_adjoint: device time of its kernel (ms), the largest relative deviation of its
 * replayed final states from the forward run's (rho and m relative to max|rho|, widths relative to h),
 * and the cell-steps it replayed (initial cells x steps, per instance, summed). Any may be NULL. */
imexds_status imexds_adjoint_info(imexds_ctx* ctx, double* kernel_ms, double* replay_err, int64_t* cell_steps);
/* The last imexds_adjoint's replayed final cell lists (host arrays; cell_offsets has n_inst+1 entries,
 * the others are sized from cell_offsets[n_inst], which may exceed the forward's total when a replay
 * diverged; any array but cell_offsets may be NULL) and, per instance, where a replay was stopped:
 * 0 not stopped, 1 its program ended early in a recomputed segment, 2/4 its grid events did not
 * reverse to the taped list, 3 a block system was singular, 5 its final cell count differs from the
 * forward run's, 6 its step count differs, 7 its final cell count differs (host check). */
imexds_status imexds_adjoint_replay(imexds_ctx* ctx, int32_t* cell_offsets, double* widths, double* rho,
                                    double* m, int32_t* stop_site);

/* Free the context and its device memory (NULL is ignored). */
void imexds_destroy(imexds_ctx* ctx);
const char* imexds_status_string(imexds_status s);
/* Text of the last CUDA error seen by any context of this process (thread-unsafe, static storage). */
const char* imexds_last_error_string(void);

#ifdef __cplusplus
}
#endif
#endif
