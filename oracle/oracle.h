/* Oracle for the explicit-implicit domain-splitting scheme (May & Thein, arXiv 2211.00705).
 *
 * TEST INFRASTRUCTURE ONLY. This is a plain, slow FP64 CPU implementation of the scheme,
 * written from the paper, that the tests, the smoke check and the CPU baseline of the
 * benchmark compare the CUDA library against. Nothing in the product library links it,
 * includes it or calls it, and it shares no code with the CUDA path.
 *
 * Pins (tests/test_oracle_pins.py, test_oracle_scheme.py, test_oracle_tangent.py): the boundary solver and
 * the creation solver against the paper's printed star states, the saturation table, closed forms and
 * special cases; the scheme against conservation, preserved equilibria, the exact Riemann solution and a
 * fully explicit run; the tangent mode against central differences. The HLL wave-speed estimate (Davis)
 * is a reading — the paper names HLL only — pinned by consistency, upwind limits and Toro's integral
 * consistency (the HLL state equals the average of the exact two-rarefaction solution over the fan),
 * not by printed values.
 *
 * Modes: plain (double), tangent (forward-mode dual numbers, oracle/dual.h) and operation counting
 * (oracle/counted.h); the scheme is one template on the scalar type, so all three run the same code.
 *
 * Conventions (shared in meaning, not in code, with the product C-ABI):
 *   phase 0 = vapour, phase 1 = liquid.
 *   [[X]] = X_right - X_left at any discontinuity (Sec. 2.1).
 *   A state is (rho, m = rho*u) per cell; cells carry a width and a phase label.
 */
#ifndef IMEXDS_ORACLE_H
#define IMEXDS_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int kind;    /* 0: ideal gas p = a2*rho (Eq. eos:isoT_idgas); 1: linear Tait p = p0 + a2*(rho - rho0) (Eq. eos:isoT_lintait) */
  double a2;   /* squared isothermal sound speed (k T0 / m for the vapour, K0/rho0 for the liquid) */
  double p0;   /* Tait reference pressure (saturation pressure); unused for kind 0 */
  double rho0; /* Tait reference density (saturation liquid density); unused for kind 0 */
} orc_eos;

typedef struct {
  orc_eos ph[2];   /* [0] vapour, [1] liquid */
  double p_sat;    /* saturation pressure: common zero of both Gibbs energies */
  double p_min;    /* minimum liquid pressure (cavitation threshold, App. B) */
  double p_tilde;  /* maximum vapour pressure (nucleation threshold, App. B) */
} orc_fluid;

typedef struct {
  double cfl;          /* C_CFL of Eq. cfl_cond:unif */
  double theta_nb;     /* theta of the regular neighbours in Alg. 2 (0.9 in Sec. 4) */
  double tol_nb, tol_k;/* stop tolerances of Sec. 4 (1e-3 neighbours, 1e-1 tiny cells) */
  int res_mode;        /* 0: residual as printed in Sec. 4 (1/s); 1: residual times dt (dimensionless) */
  int l_max;           /* cap on dual-time iterations per block */
  double newton_tol;   /* relative step tolerance of the phase-boundary Newton iteration */
  int newton_itmax;    /* cap on Newton iterations */
  double alpha_min;    /* merge floor: a cell predicted below alpha_min*h is merged */
  double split_ratio;  /* a phase-boundary cell wider than split_ratio*h is split (2 in Sec. 3.4) */
  int creation;        /* 1: detect cavitation/nucleation at same-phase faces (App. B) */
  int block_solver;    /* solver of each block's implicit system: 0 = dual time stepping (Alg. 2, the
                          paper's); 1 = Newton with a central-difference Jacobian (the paper's outlook):
                          same system, same stop test (the Sec. 4 residual of the iterate), l_max caps
                          its iterations; dts_iters then counts Newton iterations */
} orc_opts;

/* statuses (same numbering as the product library) */
enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_NONPHYSICAL = 3, ORC_ERR_PB_NOCONV = 4,
       ORC_ERR_VANISH = 6, ORC_ERR_CAPACITY = 9 };

void orc_default_opts(orc_opts* o);

/* ---- pointwise pieces (unit tests and pins) ---- */
/* HLL flux (Toro) at a same-phase face; F[2] = (mass, momentum) flux. */
void orc_hll(const orc_fluid* fl, int ph, double rl, double ml, double rr, double mr, double F[2]);
/* Evaluate the phase-boundary system G of Eq. 2p_RP:ex_sys at given star pressures (pl, pr) of
 * the left and right side. out[0..1] = G, out[2] = z (kinetic relation), out[3..6] = DG row-major. */
void orc_pb_system(const orc_fluid* fl, double tau, int phl, double rl, double ul, int phr, double rr,
                   double ur, double pls, double prs, double out[7]);
/* Solve the phase-boundary Riemann problem (App. A). out: [0] p_l*, [1] p_r*, [2] rho_l*, [3] rho_r*,
 * [4] u_l*, [5] u_r*, [6] z, [7] w, [8] F_mass, [9] F_mom, [10] newton iterations. Returns status. */
int orc_pb_solve(const orc_fluid* fl, const orc_opts* o, double tau, int phl, double rl, double ul,
                 int phr, double rr, double ur, double out[11]);
/* Star pressure of the same-phase Riemann problem without phase transition. */
double orc_nopt_star(const orc_fluid* fl, int ph, double rl, double ul, double rr, double ur);
/* Single-phase Riemann problem with phase creation (App. B): parent phase ph, created phase 1-ph.
 * out: [0] p_parent_left*, [1] p_created*, [2] p_parent_right*, [3] rho_created, [4] u_created,
 * [5] z_left_PB, [6] z_right_PB, [7] w_left, [8] w_right, [9] u_parent_left*, [10] u_parent_right*,
 * [11] newton iterations. Returns status. */
int orc_creation_solve(const orc_fluid* fl, const orc_opts* o, double tau, int ph, double rl, double ul,
                       double rr, double ur, double out[12]);
/* Exact solution of the two-phase Riemann problem sampled at n similarity coordinates xi = x/t. */
int orc_exact_sample(const orc_fluid* fl, const orc_opts* o, double tau, int phl, double rl, double ul,
                     int phr, double rr, double ur, int n, const double* xi, double* rho, double* u, int* ph);

/* ---- batched instances ---- */
void* orc_create(int n_inst, const int* n_lattice, const double* x_left, const double* x_right,
                 const double* tau, const orc_fluid* fl, const orc_opts* o);
void orc_destroy(void* H);
/* Cell lists per instance, concatenated; cell_offsets has n_inst+1 entries. */
int orc_set_states(void* H, const int* cell_offsets, const double* widths, const double* rho,
                   const double* m, const unsigned char* phase, double t0);
int orc_n_cells(void* H, int* cell_counts);
int orc_get_states(void* H, int* cell_offsets, double* widths, double* rho, double* m,
                   unsigned char* phase, double* t, int* status);
/* Phase-boundary positions of every instance (n_pb per instance, concatenated). */
int orc_get_pbs(void* H, int* pb_offsets, double* x_pb);
/* per instance 10 counters: steps, dts_iters, dts_max, newton, merges, splits, creations,
 * maxiter_warnings, pb_solves, last_dt_bits(unused=0) */
int orc_get_stats(void* H, long long* stats);
int orc_run_to(void* H, double t_end, int n_threads);
int orc_step(void* H, int n_steps, int n_threads);
/* Fully explicit reference (brute force): every cell explicit, dt limited by the smallest cell. */
int orc_explicit_run_to(void* H, double t_end, int n_threads);
/* Residual of the implicit system G(W) = 0 (Sec. 3.3) of the last step's blocks, max over blocks;
 * recorded when the dual-time loop ends (diagnostic for tests). */
double orc_last_implicit_residual(void* H, int inst);

/* ---- tangent-linear (forward-mode) derivative: the oracle's own derivative of the scheme ----
 * Re-runs every instance from its current states through the same code with dual numbers (value +
 * 8 directional derivatives per pass, more directions in further passes) and keeps the derivatives
 * of the final cell states. Branch decisions (CFL argmax, merges, blocks, splits, stop tests) are
 * frozen; iterations (Newton, dual time) are differentiated as computed. Seeds are laid out
 * [n_dir][total cells] for widths, rho and m and [n_dir][n_inst] for tau; any may be NULL (zero).
 * Seeding the widths of the two cells next to a phase boundary with +d and -d moves the boundary by
 * d. The program is a list of calls: kind 0 = step(arg) steps, kind 1 = run_to(arg). Afterwards
 * the instances hold the final states (as if the program had run). */
int orc_tangent(void* H, int n_dir, const double* seed_w, const double* seed_rho, const double* seed_m,
                const double* seed_tau, int n_prog, const int* prog_kind, const double* prog_arg, int n_threads);
/* Direction dir of the last orc_tangent: final-state derivatives, in orc_get_states order. */
int orc_get_tangent(void* H, int dir, double* d_w, double* d_rho, double* d_m);

/* Operation count of a program (kinds as in orc_tangent), run on copies of the instances with a
 * counting scalar (oracle/counted.h): the instances keep their states. counts[7]: adds and subtracts,
 * multiplies, divides, square roots, logarithms, exponentials, and cell-steps (cells at the start of
 * every step, summed over steps and instances). */
int orc_count_ops(void* H, int n_prog, const int* prog_kind, const double* prog_arg, long long* counts);

#ifdef __cplusplus
}
#endif
#endif
