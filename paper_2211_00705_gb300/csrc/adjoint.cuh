// Discrete adjoint of the explicit-implicit splitting scheme (arXiv 2211.00705): gradients of a loss of
// the final cell states with respect to the initial states, the initial boundary positions (through the
// widths) and the kinetic coefficient tau of every instance.
//
// Design (up to AWARPS instances per CTA, one warp each, all instances in one launch):
//   * Warp w advances instance base + w through the data-parallel parts of a step (fluxes, updates, list copies,
//     reductions); lane l of warp 0 runs the one-thread parts of instance base + l (boundary solves and grid
//     management, Algorithm 2 on the blocks, created cells and splits; in reverse the transposed block solves),
//     so that the serial chains of the CTA's instances issue their FP64 instructions together (GB300 issues a
//     one-lane FP64 warp instruction at the cost of a full one). The instances of a CTA step in lockstep; an
//     instance that has finished or failed sits out the remaining steps.
//   * Replay: the step of Algorithm 1 / Algorithm 2 runs again on a plain cell list of the instance
//     (the paper's moving grid: one entry per cell, faces with their kind), from the initial states of
//     the last forward call, with the same device physics as the forward kernels. Every k steps the
//     whole list is written to a checkpoint.
//   * Reverse: for the checkpoint segments from last to first, the segment is recomputed from its
//     checkpoint while each step's pre-step list and its decisions (dt, the CFL argmax cell, merges,
//     blocks, the last dual-time iterate of each block, the converged boundary pressures, splits) are
//     taped; then the steps are reversed one by one:
//       splits^T -> boundary positions^T -> per block: the converged implicit system differentiated by
//       the implicit function theorem (one transposed solve of (I - dg/dW)^T mu = lambda_W, not an
//       unrolled dual-time loop) -> explicit sweep^T (HLL Jacobians at U^n) -> merges^T -> dt^T through
//       the argmax cell (or t^T for a step clipped to an end time).
//   * Face Jacobians come from forward-mode dual numbers (adjoint_local.cuh); the boundary flux is
//     differentiated at the converged star pressures by the implicit function theorem.
// Decisions (merges, blocks, splits, the argmax cell, dual-time stop) are frozen: the gradient is that
// of the discrete map along the replayed trajectory. Phase creation (App. B) is differentiated too: the
// created cell's insertion, the per-side fluxes and moving faces at the creation face, and the creation
// system itself by the implicit function theorem.
#pragma once
#include "adjoint_local.cuh"

namespace imexds {
namespace adj {

constexpr int AWARPS = 8;      // instances per CTA at most, one warp each
constexpr int ATHREADS = 32 * AWARPS;
constexpr int AMAXPB = 16;   // phase boundaries per instance
constexpr int AMAXBLK = 8;   // blocks per step
constexpr int AMAXB = 8;     // cells per block
constexpr int AMAXBC = 32;   // block cells per step, all blocks
constexpr int AMAXEV = 8;    // merges and splits per step
constexpr int ACAP_PAD = 64; // cells a list may grow by (splits, created cells) beyond its initial count
constexpr int AMAXCR = 4;    // phase creations per step

struct StepRec {
  double dt;
  int clipped, kmax, n_merge, n_blk, n_split, n_pbf;
  int mg_a[AMAXEV], mg_b[AMAXEV];
  double mg_v[AMAXEV][6];  // w_a, r_a, m_a, w_b, r_b, m_b before the merge
  int blo[AMAXBLK], bhi[AMAXBLK];
  double Wr[AMAXBC], Wm[AMAXBC];  // last dual-time iterate of each block cell, block after block
  double ppl[AMAXPB], ppr[AMAXPB];  // converged star pressures at that iterate, interior boundary faces in order
  int sp_i[AMAXEV], sp_case[AMAXEV];
  int n_cr, cr_g[AMAXCR], cr_P[AMAXCR];  // creation faces (post-merge numbering) and parent phases
  double cr_x[AMAXCR][3];                // converged (p_P-, p_C, p_P+)
  double cr_o[AMAXCR][7];                // z1, z2, u_C, p_C, rho_C, w1, w2
};

struct AInst {
  long long off;  // first slot of this instance in every per-cell / per-face array (stride cap + 1)
  long long done; // steps done inside the current program call
  int M, cap, status, pc;
  int nsteps, M_seed, site, nexp;  // site: where an instance was stopped (1..5, see k_adjoint); nexp: steps
                                  // of the forward run, which the replay is expected to repeat
  double h, xL, tau, t;
  double lam_t, lam_tau;
};

struct ACk {
  long long done;
  int M, status, pc, pad;
  double t;
};

struct ADev {
  AInst* I;
  int n_inst, k, n_ck, n_prog;
  long long stride;
  const int* pk;     // program: 0 = step(arg), 1 = run_to(arg)
  const double* pa;
  // working cell list and faces (pwl/pwr: last converged star pressures at a boundary face, the start of
  // its next solve, as in the forward kernels)
  double *w, *r, *m, *fx, *pwl, *pwr;
  unsigned char *ph, *fpb, *cdet;  // cdet: creation detected at a face (App. B)
  int* fj;
  // face scratch
  double *F0, *F1, *LF0, *LF1, *CL0, *CL1, *CR0, *CR1;
  // post-merge list (reverse)
  double *pw, *pr, *pm;
  unsigned char *pph, *pfpb;
  // adjoints (current) and accumulators
  double *lw, *lr, *lm, *lx, *nw, *nr, *nm, *nx;
  // checkpoints
  double *ck_w, *ck_r, *ck_m, *ck_fx, *ck_pwl, *ck_pwr;
  unsigned char *ck_ph, *ck_fpb;
  int* ck_fj;
  ACk* ck_h;
  // final replay states
  double *fin_w, *fin_r, *fin_m;
  unsigned char* fin_ph;
  int* fin_M;
  // tape
  double *tp_w, *tp_r, *tp_m;
  unsigned char *tp_ph, *tp_fpb;
  int* tp_M;
  StepRec* rec;
};

__device__ inline void afail(AInst& I, int code, int site = 0) {
  if (I.status == 0) {
    I.status = code;
    I.site = site;
  }
}

// ------------------------------------------------------------------------------ list helpers
// copy n cells (and n + 1 faces when faces) between two lists of the same layout, whole warp
__device__ inline void cta_copy_d(double* dst, const double* src, int n) {
  for (int i = threadIdx.x & 31; i < n; i += 32) dst[i] = src[i];
}
__device__ inline void cta_copy_b(unsigned char* dst, const unsigned char* src, int n) {
  for (int i = threadIdx.x & 31; i < n; i += 32) dst[i] = src[i];
}
__device__ inline void cta_copy_i(int* dst, const int* src, int n) {
  for (int i = threadIdx.x & 31; i < n; i += 32) dst[i] = src[i];
}
__device__ inline void cta_zero(double* dst, int n) {
  for (int i = threadIdx.x & 31; i < n; i += 32) dst[i] = 0.0;
}

// one thread: erase cell b (and face b) of a list
__device__ void list_erase(double* w, double* r, double* m, unsigned char* ph, unsigned char* fpb, int* fj,
                           double* fx, double* pl, double* pr, int M, int b) {
  for (int i = b; i + 1 < M; ++i) {
    w[i] = w[i + 1];
    r[i] = r[i + 1];
    m[i] = m[i + 1];
    ph[i] = ph[i + 1];
  }
  for (int g = b; g < M; ++g) {
    fpb[g] = fpb[g + 1];
    if (fj) fj[g] = fj[g + 1];
    if (fx) fx[g] = fx[g + 1];
    if (pl) pl[g] = pl[g + 1];
    if (pr) pr[g] = pr[g + 1];
  }
}
// one thread: open a slot at cell p (cells p.. and faces p.. move one up)
__device__ void list_open(double* w, double* r, double* m, unsigned char* ph, unsigned char* fpb, int* fj,
                          double* fx, double* pl, double* pr, int M, int p) {
  for (int i = M - 1; i >= p; --i) {
    w[i + 1] = w[i];
    r[i + 1] = r[i];
    m[i + 1] = m[i];
    ph[i + 1] = ph[i];
  }
  for (int g = M; g >= p; --g) {
    fpb[g + 1] = fpb[g];
    if (fj) fj[g + 1] = fj[g];
    if (fx) fx[g + 1] = fx[g];
    if (pl) pl[g + 1] = pl[g];
    if (pr) pr[g + 1] = pr[g];
  }
}
// adjoint lists: erase / open cell b of (lw, lr, lm) and face b of lx
__device__ void lam_erase(double* lw, double* lr, double* lm, double* lx, int M, int b) {
  for (int i = b; i + 1 < M; ++i) {
    lw[i] = lw[i + 1];
    lr[i] = lr[i + 1];
    lm[i] = lm[i + 1];
  }
  for (int g = b; g < M; ++g) lx[g] = lx[g + 1];
}
__device__ void lam_open(double* lw, double* lr, double* lm, double* lx, int M, int p) {
  for (int i = M - 1; i >= p; --i) {
    lw[i + 1] = lw[i];
    lr[i + 1] = lr[i];
    lm[i + 1] = lm[i];
  }
  for (int g = M; g >= p; --g) lx[g + 1] = lx[g];
}

// Per-instance state of the current step, in shared memory (one entry per warp of the CTA).
struct SharedStep {
  double dt, lam, lam_dt;  // lam_dt: d(dt) contributions of a reverse step (lane 0 of the instance's warp and
                           // the instance's lane of warp 0 add to it in turn)
  int M, kmax, clipped, done, bad, act;  // act: the instance takes part in this step
  int n_pb, pb[AMAXPB];
  int n_blk, blo[AMAXBLK], bhi[AMAXBLK];
  int n_cr, cr_g[AMAXCR], cr_P[AMAXCR];
  double cr_o[AMAXCR][7];
  double t_end;
  double hp[AMAXBC];  // predicted widths of the block cells (block after block)
  int tiny[AMAXBC];   // tiny flags of the block cells
  StepRec* rec;       // where this step's decisions are taped (nullptr: not taped)
  int slot;           // tape slot of the pre-step list
};

// creation event at face g of this step, or -1
__device__ inline int cr_at(const SharedStep& S, int g) {
  for (int k = 0; k < S.n_cr; ++k)
    if (S.cr_g[k] == g) return k;
  return -1;
}

// The explicit update of cell i (Eq. godunov_meth:nonunif): the fluxes it sees at its right and left faces
// and its new width. At a creation face the cell on each side sees that side's flux (mass flux z1 on the
// left, z2 on the right) and the face moves with w1 / w2; elsewhere F0/F1 hold the face flux.
struct CellUpd {
  double fr0, fr1, fl0, fl1, wl, wr, h1;
};
__device__ inline CellUpd cell_upd(const double* F0, const double* F1, const SharedStep& S, int i, double w,
                                   double dt) {
  CellUpd c;
  c.fr0 = F0[i + 1];
  c.fr1 = F1[i + 1];
  c.fl0 = F0[i];
  c.fl1 = F1[i];
  c.wl = c.wr = 0.0;
  if (S.n_cr) {
    const int kr = cr_at(S, i + 1), kl = cr_at(S, i);
    if (kr >= 0) {
      const double* e = S.cr_o[kr];
      c.fr0 = -e[0];
      c.fr1 = -e[0] * e[2] + e[3];
      c.wl = e[5];
    }
    if (kl >= 0) {
      const double* e = S.cr_o[kl];
      c.fl0 = -e[1];
      c.fl1 = -e[1] * e[2] + e[3];
      c.wr = e[6];
    }
  }
  c.h1 = w + (c.wl - c.wr) * dt;
  return c;
}

__device__ inline bool in_block(const SharedStep& S, int i) {
  for (int b = 0; b < S.n_blk; ++b)
    if (i >= S.blo[b] && i <= S.bhi[b]) return true;
  return false;
}
__device__ inline bool face_in_block(const SharedStep& S, int g) {
  for (int b = 0; b < S.n_blk; ++b)
    if (g > S.blo[b] && g <= S.bhi[b]) return true;
  return false;
}

// warp max of v (first index among equal maxima); every lane gets the result
__device__ inline void warp_argmax(double& v, int& idx) {
  for (int o = 16; o > 0; o >>= 1) {
    const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
    const int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
    if (v2 > v || (v2 == v && i2 < idx)) {
      v = v2;
      idx = i2;
    }
  }
}
// warp sum in a fixed order (the same bits on every lane)
__device__ inline double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// collect the phase-boundary faces of a list (ascending) into S.pb, whole warp; false if there are too many
__device__ bool collect_pbs(SharedStep& S, const unsigned char* fpb, int M) {
  const int lane = threadIdx.x & 31;
  if (lane == 0) S.n_pb = 0;
  __syncwarp();
  for (int g = 1 + lane; g < M; g += 32)
    if (fpb[g]) {
      int q = atomicAdd(&S.n_pb, 1);
      if (q < AMAXPB) S.pb[q] = g;
    }
  __syncwarp();
  const bool ok = S.n_pb <= AMAXPB;
  if (lane == 0 && ok) {
    for (int a = 1; a < S.n_pb; ++a) {  // insertion sort of a handful of faces
      int v = S.pb[a], b = a - 1;
      while (b >= 0 && S.pb[b] > v) {
        S.pb[b + 1] = S.pb[b];
        --b;
      }
      S.pb[b + 1] = v;
    }
  }
  __syncwarp();
  return ok;
}

// ------------------------------------------------------------------------------ forward step
// Program position: advance past finished calls; returns false when the instance has no step left.
__device__ bool prog_next(const ADev& A, AInst& I, double& t_end) {
  while (I.pc < A.n_prog) {
    if (A.pk[I.pc] == 0) {
      if (I.done < (long long)A.pa[I.pc]) break;
    } else {
      if (I.t < A.pa[I.pc]) break;
    }
    I.pc++;
    I.done = 0;
  }
  if (I.pc >= A.n_prog || I.status) return false;
  t_end = (A.pk[I.pc] == 1) ? A.pa[I.pc] : -1.0;
  return true;
}

// Algorithm 2 on one block of the list (one thread: the instance's lane of warp 0). U^n of the block cells is
// still in the list (the sweep does not touch them); FL/FR are the explicit fluxes at faces lo and hi+1. Writes
// the last iterate and converged boundary pressures to the step record (when rec != nullptr) and the Part 2
// result to out_*.
__device__ bool dts_block(const ADev& A, AInst& I, const SharedStep& S, int lo, int hi, const double* hp,
                          const int* tiny, double FL0, double FL1, double FR0, double FR1, StepRec* rec,
                          int& rec_cell, int& rec_pbf, double* out_r, double* out_m, double* out_w, double* wcf) {
  const long long o = I.off;
  const double dt = S.dt, h = I.h, tau = I.tau;
  const int nb = hi - lo + 1;
  double Ur[AMAXB], Um[AMAXB], Uw[AMAXB], Wr[AMAXB], Wm[AMAXB], th[AMAXB];
  double F0[AMAXB + 1], F1[AMAXB + 1], wc[AMAXB + 1], hl[AMAXB], gl[AMAXB + 1], gr[AMAXB + 1];
  int ph[AMAXB], fp[AMAXB + 1];
  for (int q = 0; q < nb; ++q) {
    Ur[q] = Wr[q] = A.r[o + lo + q];
    Um[q] = Wm[q] = A.m[o + lo + q];
    Uw[q] = A.w[o + lo + q];
    ph[q] = A.ph[o + lo + q];
    th[q] = fmin(c_opts.theta_nb, hp[q] / h);
  }
  for (int q = 0; q <= nb; ++q) {
    fp[q] = (q > 0 && q < nb) ? A.fpb[o + lo + q] : 0;
    gl[q] = fp[q] ? A.pwl[o + lo + q] : 0.0;
    gr[q] = fp[q] ? A.pwr[o + lo + q] : 0.0;
  }
  FaceJac fj[AMAXB + 1];  // boundary faces' Jacobians (Newton block solver)
  const bool newton_solver = (c_opts.block_solver == 1);
  auto fluxes = [&]() -> int {  // 0 ok, 1 boundary solve failed, 2 non-positive width
    F0[0] = FL0;
    F1[0] = FL1;
    F0[nb] = FR0;
    F1[nb] = FR1;
    wc[0] = wc[nb] = 0.0;
    for (int q = 1; q < nb; ++q) {
      if (fp[q]) {
        PBOut R = newton_solver ? pb_solve_core<true>(c_fluid, c_opts, tau, ph[q - 1], Wr[q - 1], Wm[q - 1], ph[q],
                                                      Wr[q], Wm[q], gl[q], gr[q], &fj[q])
                                : pb_solve_warm(c_fluid, c_opts, tau, ph[q - 1], Wr[q - 1], Wm[q - 1], ph[q], Wr[q],
                                                Wm[q], gl[q], gr[q]);
        if (!R.ok) return 1;
        F0[q] = R.F0;
        F1[q] = R.F1;
        wc[q] = R.w;
      } else {
        hll_fast(c_fluid.ph[ph[q]], Wr[q - 1], Wm[q - 1], Wr[q], Wm[q], F0[q], F1[q]);
        wc[q] = 0.0;
      }
    }
    for (int q = 0; q < nb; ++q) hl[q] = __fma_rn(wc[q + 1] - wc[q], dt, Uw[q]);
    for (int q = 0; q < nb; ++q)
      if (!pos_finite_bits(hl[q])) return 2;
    return 0;
  };
  bool stop = false;
  if (newton_solver) {
    // Newton on the block's system R(W) = W - T(W) with the stop test of Sec. 4 (the forward kernels'
    // newton_simple / newton_general): fluxes at W, T(W), the test, then (I - dT/dW) dW = T(W) - W
    const double dtr = (c_opts.res_mode == 1) ? 1.0 : dt;
    double corr_prev = INFINITY;
    for (int l = 0; l < c_opts.l_max; ++l) {
      int e = fluxes();
      if (e) {
        afail(I, e == 1 ? IMEXDS_ERR_PB_NOCONV : IMEXDS_ERR_VANISH);
        return false;
      }
      double Tr[AMAXB], Tm[AMAXB], ih[AMAXB];
      stop = true;
      for (int q = 0; q < nb; ++q) {
        ih[q] = rcp_nr(hl[q]);
        Tr[q] = __fma_rn(-dt, F0[q + 1] - F0[q], Uw[q] * Ur[q]) * ih[q];
        Tm[q] = __fma_rn(-dt, F1[q + 1] - F1[q], Uw[q] * Um[q]) * ih[q];
        const double lim = (tiny[q] ? c_opts.tol_k : c_opts.tol_nb) * dtr;
        stop = stop && below_tol(Tr[q] - Wr[q], Wr[q], lim) && below_tol(Tm[q] - Wm[q], Wm[q], lim);
      }
      if (stop) break;
      for (int q = 1; q < nb; ++q)
        if (!fp[q]) hll_jac(c_fluid.ph[ph[q]], Wr[q - 1], Wm[q - 1], Wr[q], Wm[q], fj[q]);
      double dr[AMAXB], dmv[AMAXB];
      if (!newton_block_step(nb, dt, ih, Tr, Tm, Wr, Wm, fj, dr, dmv)) {
        afail(I, IMEXDS_ERR_PB_NOCONV);
        return false;
      }
      const double corr = newton_corr(nb, Wr, Wm, dr, dmv);
      const bool at_floor = newton_at_floor(corr, corr_prev);
      corr_prev = corr;
      for (int q = 0; q < nb; ++q) {
        Wr[q] += dr[q];
        Wm[q] += dmv[q];
      }
      if (at_floor) break;
    }
  }
  // Algorithm 2 Part 1 in the forward kernels' arithmetic (dts_simple, dts_zone_general), so that the replay
  // takes the same stop decisions: the Sec. 4 test of a component, (1 + theta)|W^{l+1} - W^l| / (theta dt
  // max(|W^l|, 1)) (x dt in the res dt mode) below tol, as |W^{l+1} - W^l| < lim max(|W^l|, 1)
  double ith[AMAXB], lim[AMAXB];
  {
    const double dtr = (c_opts.res_mode == 1) ? 1.0 : dt;
    for (int q = 0; q < nb; ++q) {
      ith[q] = 1.0 / (1.0 + th[q]);
      lim[q] = (tiny[q] ? c_opts.tol_k : c_opts.tol_nb) * th[q] * dtr * ith[q];
    }
  }
  for (int l = 0; !newton_solver && l < c_opts.l_max && !stop; ++l) {
    int e = fluxes();
    if (e) {
      afail(I, e == 1 ? IMEXDS_ERR_PB_NOCONV : IMEXDS_ERR_VANISH);
      return false;
    }
    stop = true;
    for (int q = 0; q < nb; ++q) {
      const double t = th[q], ih = rcp_nr(hl[q]);
      const double tr = __fma_rn(-dt, F0[q + 1] - F0[q], Uw[q] * Ur[q]) * ih;
      const double tm = __fma_rn(-dt, F1[q + 1] - F1[q], Uw[q] * Um[q]) * ih;
      const double nr = __fma_rn(t, tr, Wr[q]) * ith[q];
      const double nm = __fma_rn(t, tm, Wm[q]) * ith[q];
      stop = stop && below_tol(nr - Wr[q], Wr[q], lim[q]) && below_tol(nm - Wm[q], Wm[q], lim[q]);
      Wr[q] = nr;
      Wm[q] = nm;
    }
  }
  int e = fluxes();  // Part 2 at the last iterate
  if (e) {
    afail(I, e == 1 ? IMEXDS_ERR_PB_NOCONV : IMEXDS_ERR_VANISH);
    return false;
  }
  for (int q = 0; q < nb; ++q) {
    out_r[q] = (Uw[q] * Ur[q] - dt * (F0[q + 1] - F0[q])) / hl[q];
    out_m[q] = (Uw[q] * Um[q] - dt * (F1[q + 1] - F1[q])) / hl[q];
    out_w[q] = hl[q];
  }
  for (int q = 0; q <= nb; ++q) wcf[q] = wc[q];
  for (int q = 1; q < nb; ++q)
    if (fp[q]) {
      A.pwl[o + lo + q] = gl[q];
      A.pwr[o + lo + q] = gr[q];
    }
  if (rec) {
    if (rec_cell + nb > AMAXBC) {
      afail(I, IMEXDS_ERR_CAPACITY);
      return false;
    }
    for (int q = 0; q < nb; ++q) {
      rec->Wr[rec_cell + q] = Wr[q];
      rec->Wm[rec_cell + q] = Wm[q];
    }
    rec_cell += nb;
    for (int q = 1; q < nb; ++q)
      if (fp[q]) {
        if (rec_pbf >= AMAXPB) {
          afail(I, IMEXDS_ERR_CAPACITY);
          return false;
        }
        rec->ppl[rec_pbf] = gl[q];
        rec->ppr[rec_pbf] = gr[q];
        rec_pbf++;
      }
  }
  return true;
}

// Grid management of one instance at the start of a step (one thread: the instance's lane of warp 0).
__device__ __noinline__ void serial_grid(const ADev& A, AInst& I, SharedStep& S) {
  const long long o = I.off;
  StepRec* rec = S.rec;
  // (2) grid management: boundary solves at U^n, marks, merges (the list is short-edited)
  const double dt = S.dt;
  double wf[AMAXPB];
  int nmk = 0, mk[2 * AMAXPB];
  bool ok = true;
  for (int q = 0; q < S.n_pb && ok; ++q) {
    int g = S.pb[q];
    PBOut R = pb_solve_warm(c_fluid, c_opts, I.tau, A.ph[o + g - 1], A.r[o + g - 1], A.m[o + g - 1], A.ph[o + g],
                            A.r[o + g], A.m[o + g], A.pwl[o + g], A.pwr[o + g]);
    if (!R.ok) {
      afail(I, IMEXDS_ERR_PB_NOCONV);
      ok = false;
    }
    wf[q] = R.w;
  }
  // candidate cells: both neighbours of every boundary, ascending, without repeats
  for (int q = 0; q < S.n_pb && ok; ++q)
    for (int s = 0; s < 2; ++s) {
      int i = S.pb[q] - 1 + s;
      if (nmk > 0 && mk[nmk - 1] >= i) continue;
      int ql = -1, qr = -1;  // boundary indices on the left / right face of i
      for (int p = 0; p < S.n_pb; ++p) {
        if (S.pb[p] == i) ql = p;
        if (S.pb[p] == i + 1) qr = p;
      }
      double wl = ql >= 0 ? wf[ql] : 0.0, wr = qr >= 0 ? wf[qr] : 0.0;
      double hp = A.w[o + i] + (wr - wl) * dt;
      if (hp < fmax(c_opts.alpha_min * I.h, 0.5 * A.w[o + i])) mk[nmk++] = i;
    }
  // merges in ascending order with the index shifts of earlier merges
  int nmerge = 0, shift = 0;
  bool any = false;
  for (int q = 0; q < nmk && ok; ++q) {
    if (mk[q] < 0) continue;  // consumed by the merge before it
    int i = mk[q] - shift;
    int Mi = S.M;
    bool left_fixed = (i > 0) && !A.fpb[o + i];
    bool right_fixed = (i + 1 < Mi) && !A.fpb[o + i + 1];
    int a, b;
    if (left_fixed) {
      a = i - 1;
      b = i;
    } else if (right_fixed) {
      a = i;
      b = i + 1;
      // the right neighbour is consumed: a later mark on it is dropped
      if (q + 1 < nmk && mk[q + 1] - shift == i + 1) mk[q + 1] = -1000000;
    } else {
      afail(I, IMEXDS_ERR_VANISH);
      ok = false;
      break;
    }
    if (nmerge >= AMAXEV) {
      afail(I, IMEXDS_ERR_CAPACITY);
      ok = false;
      break;
    }
    double wa = A.w[o + a], ra = A.r[o + a], ma = A.m[o + a];
    double wb = A.w[o + b], rb = A.r[o + b], mb = A.m[o + b];
    double wm = wa + wb;
    A.r[o + a] = (wa * ra + wb * rb) / wm;
    A.m[o + a] = (wa * ma + wb * mb) / wm;
    A.w[o + a] = wm;
    list_erase(A.w + o, A.r + o, A.m + o, A.ph + o, A.fpb + o, A.fj + o, A.fx + o, A.pwl + o, A.pwr + o, Mi, b);
    S.M = Mi - 1;
    if (rec) {
      rec->mg_a[nmerge] = a;
      rec->mg_b[nmerge] = b;
      double* v = rec->mg_v[nmerge];
      v[0] = wa, v[1] = ra, v[2] = ma, v[3] = wb, v[4] = rb, v[5] = mb;
    }
    nmerge++;
    shift++;
    any = true;
    for (int p = 0; p < S.n_pb; ++p)
      if (S.pb[p] > b) S.pb[p]--;
  }
  if (rec) rec->n_merge = nmerge;
  // predicted widths on the merged grid (boundary speeds at U^n of the merged cells)
  if (ok && any)
    for (int q = 0; q < S.n_pb && ok; ++q) {
      int g = S.pb[q];
      PBOut R = pb_solve_warm(c_fluid, c_opts, I.tau, A.ph[o + g - 1], A.r[o + g - 1], A.m[o + g - 1],
                              A.ph[o + g], A.r[o + g], A.m[o + g], A.pwl[o + g], A.pwr[o + g]);
      if (!R.ok) {
        afail(I, IMEXDS_ERR_PB_NOCONV);
        ok = false;
      }
      wf[q] = R.w;
    }
  // (3) blocks {k-1, k, k+1} around the tiny cell of every boundary, joined where they overlap
  int nbk = 0;
  const int Mm = S.M;
  for (int q = 0; q < S.n_pb && ok; ++q) {
    int g = S.pb[q];
    int k = (A.w[o + g - 1] < A.w[o + g]) ? g - 1 : g;
    int lo = max(k - 1, 0), hi = min(k + 1, Mm - 1);
    if (nbk > 0 && lo <= S.bhi[nbk - 1]) {
      S.bhi[nbk - 1] = max(S.bhi[nbk - 1], hi);
    } else {
      if (nbk >= AMAXBLK) {
        afail(I, IMEXDS_ERR_CAPACITY);
        ok = false;
        break;
      }
      S.blo[nbk] = lo;
      S.bhi[nbk] = hi;
      nbk++;
    }
  }
  S.n_blk = ok ? nbk : 0;
  // per block cell: predicted width and tiny flag (block cells numbered block after block)
  int c = 0;
  for (int b = 0; b < S.n_blk && ok; ++b) {
    if (S.bhi[b] - S.blo[b] + 1 > AMAXB || c + S.bhi[b] - S.blo[b] + 1 > AMAXBC) {
      afail(I, IMEXDS_ERR_CAPACITY);
      ok = false;
      break;
    }
    for (int i = S.blo[b]; i <= S.bhi[b]; ++i, ++c) {
      double wl = 0.0, wr = 0.0;
      int tiny = 0;
      for (int q = 0; q < S.n_pb; ++q) {
        int g = S.pb[q];
        if (g == i) wl = wf[q];
        if (g == i + 1) wr = wf[q];
        int k = (A.w[o + g - 1] < A.w[o + g]) ? g - 1 : g;
        if (k == i) tiny = 1;
      }
      S.hp[c] = A.w[o + i] + (wr - wl) * S.dt;
      S.tiny[c] = tiny;
    }
  }
  if (rec && ok) {
    rec->n_blk = S.n_blk;
    for (int b = 0; b < S.n_blk; ++b) {
      rec->blo[b] = S.blo[b];
      rec->bhi[b] = S.bhi[b];
    }
  }
  if (!ok) S.bad = 1;
}

// Algorithm 2 on every block of one instance, Part 2 and the boundary positions, created cells, splits and
// the instance's new time (one thread: the instance's lane of warp 0).
__device__ __noinline__ void serial_blocks(const ADev& A, AInst& I, SharedStep& S) {
  const long long o = I.off;
  StepRec* rec = S.rec;
  const double t_end = S.t_end;
  // (6) Algorithm 2 on every block, Part 2, boundary positions; (8) splits
  bool ok = true;
  int rc = 0, rp = 0, c = 0;
  for (int b = 0; b < S.n_blk && ok; ++b) {
    const int lo = S.blo[b], hi = S.bhi[b], nb = hi - lo + 1;
    double orr[AMAXB], om[AMAXB], ow[AMAXB], wc[AMAXB + 1];
    ok = dts_block(A, I, S, lo, hi, S.hp + c, S.tiny + c, A.F0[o + lo], A.F1[o + lo], A.F0[o + hi + 1],
                   A.F1[o + hi + 1], rec, rc, rp, orr, om, ow, wc);
    c += nb;
    if (!ok) break;
    for (int q = 0; q < nb; ++q) {
      A.r[o + lo + q] = orr[q];
      A.m[o + lo + q] = om[q];
      A.w[o + lo + q] = ow[q];
    }
    for (int q = 1; q < nb; ++q)
      if (A.fpb[o + lo + q]) A.fx[o + lo + q] += wc[q] * S.dt;
  }
  if (rec) rec->n_pbf = rp;
  // (7) created cells (App. B), highest face first: width (w2 - w1) dt between two new boundaries at
  //     x_g + w1 dt and x_g + w2 dt, state (rho_C, rho_C u_C), the other phase
  for (int k = S.n_cr - 1; k >= 0 && ok; --k) {
    const int g = S.cr_g[k];
    const double* e = S.cr_o[k];
    const int Mi = S.M;
    if (Mi + 1 > I.cap || S.n_pb + 2 > AMAXPB) {
      afail(I, IMEXDS_ERR_CAPACITY);
      ok = false;
      break;
    }
    const double xg = I.xL + (double)A.fj[o + g] * I.h;
    list_open(A.w + o, A.r + o, A.m + o, A.ph + o, A.fpb + o, A.fj + o, A.fx + o, A.pwl + o, A.pwr + o, Mi, g);
    S.M = Mi + 1;
    A.w[o + g] = (e[6] - e[5]) * S.dt;
    A.r[o + g] = e[4];
    A.m[o + g] = e[4] * e[2];
    A.ph[o + g] = (unsigned char)(1 - S.cr_P[k]);
    A.fpb[o + g] = 1;
    A.fx[o + g] = xg + e[5] * S.dt;
    A.fpb[o + g + 1] = 1;
    A.fx[o + g + 1] = xg + e[6] * S.dt;
    A.pwl[o + g] = A.pwr[o + g] = A.pwl[o + g + 1] = A.pwr[o + g + 1] = 0.0;
    // boundary list: faces at or after g move one up; the two new boundaries join it (kept sorted)
    int np = 0, tmp[AMAXPB];
    bool put = false;
    for (int p = 0; p < S.n_pb; ++p) {
      int f = S.pb[p] >= g ? S.pb[p] + 1 : S.pb[p];
      if (!put && f > g) {
        tmp[np++] = g;
        tmp[np++] = g + 1;
        put = true;
      }
      tmp[np++] = f;
    }
    if (!put) {
      tmp[np++] = g;
      tmp[np++] = g + 1;
    }
    for (int p = 0; p < np; ++p) S.pb[p] = tmp[p];
    S.n_pb = np;
  }
  // splits of boundary cells wider than split_ratio h (Sec. 3.4), keeping fixed faces on the lattice
  int nsp = 0;
  if (ok) {
    int Mi = S.M;
    int last = -1;
    for (int q = 0; q < S.n_pb && ok; ++q)
      for (int s = 0; s < 2; ++s) {
        int i = S.pb[q] - 1 + s + nsp;  // boundary faces shift by the cells inserted so far
        if (i <= last) continue;
        last = i;
        bool lpb = A.fpb[o + i], rpb = A.fpb[o + i + 1];
        if (!(lpb || rpb) || !(A.w[o + i] > c_opts.split_ratio * I.h)) continue;
        double w1, w2;
        int jc, cs;
        if (!lpb) {
          jc = A.fj[o + i] + 1;
          w1 = I.h;
          w2 = A.w[o + i] - I.h;
          cs = 1;
        } else if (!rpb) {
          jc = A.fj[o + i + 1] - 1;
          w2 = I.h;
          w1 = A.w[o + i] - I.h;
          cs = 2;
        } else {
          double xm = 0.5 * (A.fx[o + i] + A.fx[o + i + 1]);
          jc = (int)llround((xm - I.xL) / I.h);
          w1 = (I.xL + (double)jc * I.h) - A.fx[o + i];
          w2 = A.w[o + i] - w1;
          cs = 3;
          if (!(w1 > 0.0) || !(w2 > 0.0)) continue;
        }
        if (Mi + 1 > I.cap || nsp >= AMAXEV) {
          afail(I, IMEXDS_ERR_CAPACITY);
          ok = false;
          break;
        }
        list_open(A.w + o, A.r + o, A.m + o, A.ph + o, A.fpb + o, A.fj + o, A.fx + o, A.pwl + o, A.pwr + o, Mi,
                  i + 1);
        Mi++;
        A.fpb[o + i + 1] = 0;
        A.fj[o + i + 1] = jc;
        A.fx[o + i + 1] = 0.0;
        A.pwl[o + i + 1] = A.pwr[o + i + 1] = 0.0;
        A.w[o + i] = w1;
        A.w[o + i + 1] = w2;
        A.r[o + i + 1] = A.r[o + i];  // both parts keep the state of the split cell
        A.m[o + i + 1] = A.m[o + i];
        A.ph[o + i + 1] = A.ph[o + i];
        if (rec) {
          rec->sp_i[nsp] = i;
          rec->sp_case[nsp] = cs;
        }
        nsp++;
        last = i + 1;  // the new cell is not examined in this step
      }
    S.M = Mi;
  }
  if (rec) rec->n_split = nsp;
  if (!ok) S.bad = 1;
  I.M = S.M;
  I.t = S.clipped ? t_end : I.t + S.dt;
  I.done++;
}

// One time step of the replay for the instances of this CTA that take part (S.act). Warp w advances instance
// base + w through the data-parallel parts; lane l of warp 0 runs the one-thread parts of instance base + l
// (serial_grid, serial_blocks). Tapes the pre-step list into tape slot S.slot and the decisions into *S.rec
// when S.rec != nullptr. Every thread of the CTA calls it.
__device__ void fwd_step_grp(const ADev& A, SharedStep* SS, int base, int G) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = lane;
  SharedStep& S = SS[w];
  const bool mine = S.act != 0;
  if (mine) {
    AInst& I = A.I[base + w];
    const long long o = I.off;
    StepRec* rec = S.rec;
    const int slot = S.slot;
    const double t_end = S.t_end;
    if (lane == 0) {
      S.M = I.M;
      S.bad = 0;
    }
    __syncwarp();
    int M = S.M;
    if (rec) {
      const long long to = (long long)slot * A.stride + o;
      cta_copy_d(A.tp_w + to, A.w + o, M);
      cta_copy_d(A.tp_r + to, A.r + o, M);
      cta_copy_d(A.tp_m + to, A.m + o, M);
      cta_copy_b(A.tp_ph + to, A.ph + o, M);
      cta_copy_b(A.tp_fpb + to, A.fpb + o, M + 1);
      if (lane == 0) A.tp_M[(long long)slot * A.n_inst + (int)(&I - A.I)] = M;
    }
    // (1) CFL time step (Eq. cfl_cond:unif) over all cells, with the argmax cell
    {
      double v = -1.0;
      int idx = 0x7fffffff;
      for (int i = tid; i < M; i += 32) {
        double s = fabs(A.m[o + i] / A.r[o + i]) + c_fluid.ph[A.ph[o + i]].a;
        if (s > v) {
          v = s;
          idx = i;
        }
      }
      warp_argmax(v, idx);
      if (lane == 0) {
        double dt = c_opts.cfl * I.h / v;
        int clipped = 0;
        if (t_end > 0.0 && t_end - I.t <= dt) {
          dt = t_end - I.t;
          clipped = 1;
        }
        S.dt = dt;
        S.lam = dt / I.h;
        S.kmax = idx;
        S.clipped = clipped;
        if (rec) {
          rec->dt = dt;
          rec->clipped = clipped;
          rec->kmax = idx;
          rec->n_merge = rec->n_blk = rec->n_split = rec->n_pbf = 0;
        }
      }
    }
    if (!collect_pbs(S, A.fpb + o, M) && lane == 0) {
      afail(I, IMEXDS_ERR_CAPACITY);
      S.bad = 1;
    }
    __syncwarp();
  }
  __syncthreads();
  if (w == 0 && lane < G && SS[lane].act && !SS[lane].bad) serial_grid(A, A.I[base + lane], SS[lane]);
  __syncthreads();
  if (mine && !S.bad) {
    AInst& I = A.I[base + w];
    const long long o = I.off;
    StepRec* rec = S.rec;
    int M = S.M;
    // (4) phase creation (App. B) at same-phase faces between two explicit cells: detection by the
    //     no-transition star pressure, a face whose left neighbour face is also detected is not used
    if (lane == 0) S.n_cr = 0;
    __syncwarp();
    if (c_opts.creation) {
      for (int g = tid; g <= M; g += 32) {
        unsigned char det = 0;
        if (g >= 1 && g < M && !A.fpb[o + g] && !in_block(S, g - 1) && !in_block(S, g)) {
          det = creation_detect(c_fluid, A.ph[o + g], A.r[o + g - 1], div_nr(A.m[o + g - 1], A.r[o + g - 1]),
                                A.r[o + g], div_nr(A.m[o + g], A.r[o + g]));
        }
        A.cdet[o + g] = det;
      }
      __syncwarp();
      for (int g = 1 + tid; g < M; g += 32)
        if (A.cdet[o + g] && !A.cdet[o + g - 1]) {
          const int q = atomicAdd(&S.n_cr, 1);
          if (q < AMAXCR) S.cr_g[q] = g;
        }
      __syncwarp();
      if (lane == 0) {
        if (S.n_cr > AMAXCR) {
          afail(I, IMEXDS_ERR_CAPACITY);
          S.bad = 1;
          S.n_cr = 0;
        }
        for (int a = 1; a < S.n_cr; ++a) {
          int v = S.cr_g[a], b = a - 1;
          while (b >= 0 && S.cr_g[b] > v) {
            S.cr_g[b + 1] = S.cr_g[b];
            --b;
          }
          S.cr_g[b + 1] = v;
        }
        for (int k = 0; k < S.n_cr && !S.bad; ++k) {
          const int g = S.cr_g[k];
          const int P = A.ph[o + g];
          CreateOut R = creation_solve(c_fluid, c_opts, I.tau, P, A.r[o + g - 1], A.m[o + g - 1], A.r[o + g], A.m[o + g]);
          if (!R.ok) {
            afail(I, IMEXDS_ERR_PB_NOCONV);
            S.bad = 1;
            break;
          }
          S.cr_P[k] = P;
          const double out[7] = {R.z1, R.z2, R.uC, R.pC, R.rhoC, R.w1, R.w2};
          for (int q = 0; q < 7; ++q) S.cr_o[k][q] = out[q];
          if (rec) {
            rec->cr_g[k] = g;
            rec->cr_P[k] = P;
            rec->cr_x[k][0] = R.pPl;
            rec->cr_x[k][1] = R.pC;
            rec->cr_x[k][2] = R.pPr;
            for (int q = 0; q < 7; ++q) rec->cr_o[k][q] = out[q];
          }
        }
      }
      __syncwarp();
    }
    if (!S.bad) {
      if (rec && lane == 0) rec->n_cr = S.n_cr;
      // (5) explicit fluxes from U^n at every face outside the blocks, then the explicit update
      for (int g = tid; g <= M; g += 32) {
        if (face_in_block(S, g)) continue;
        if (S.n_cr && cr_at(S, g) >= 0) continue;  // creation faces: the per-side fluxes of the event
        double f0, f1;
        if (g == 0)
          phys_flux_fast(c_fluid.ph[A.ph[o]], A.r[o], A.m[o], f0, f1);
        else if (g == M)
          phys_flux_fast(c_fluid.ph[A.ph[o + M - 1]], A.r[o + M - 1], A.m[o + M - 1], f0, f1);
        else
          hll_fast(c_fluid.ph[A.ph[o + g]], A.r[o + g - 1], A.m[o + g - 1], A.r[o + g], A.m[o + g], f0, f1);
        A.F0[o + g] = f0;
        A.F1[o + g] = f1;
      }
      __syncwarp();
      for (int i = tid; i < M; i += 32) {
        if (in_block(S, i)) continue;
        const double wi = A.w[o + i];
        if (S.n_cr && (cr_at(S, i) >= 0 || cr_at(S, i + 1) >= 0)) {
          const CellUpd c = cell_upd(A.F0 + o, A.F1 + o, S, i, wi, S.dt);
          A.r[o + i] = (wi * A.r[o + i] - S.dt * (c.fr0 - c.fl0)) / c.h1;
          A.m[o + i] = (wi * A.m[o + i] - S.dt * (c.fr1 - c.fl1)) / c.h1;
          A.w[o + i] = c.h1;
        } else if (wi == I.h) {
          A.r[o + i] = __fma_rn(-S.lam, A.F0[o + i + 1] - A.F0[o + i], A.r[o + i]);
          A.m[o + i] = __fma_rn(-S.lam, A.F1[o + i + 1] - A.F1[o + i], A.m[o + i]);
        } else {
          A.r[o + i] = (wi * A.r[o + i] - S.dt * (A.F0[o + i + 1] - A.F0[o + i])) / wi;
          A.m[o + i] = (wi * A.m[o + i] - S.dt * (A.F1[o + i + 1] - A.F1[o + i])) / wi;
        }
      }
      __syncwarp();
    }
  }
  __syncthreads();
  if (w == 0 && lane < G && SS[lane].act && !SS[lane].bad) serial_blocks(A, A.I[base + lane], SS[lane]);
  __syncthreads();
  if (mine && A.I[base + w].status == 0) {
    AInst& I = A.I[base + w];
    const long long o = I.off;
    const int M = S.M;
    int badc = 0;
    for (int i = lane; i < M; i += 32) {
      double ri = A.r[o + i], mi = A.m[o + i], wi = A.w[o + i];
      if (!(ri > 0.0) || !isfinite(ri) || !isfinite(mi) || !(wi > 0.0)) badc = 1;
    }
    badc = __any_sync(0xffffffffu, badc);
    if (lane == 0 && badc) afail(I, IMEXDS_ERR_NONPHYSICAL);
  }
  __syncwarp();
}

// ------------------------------------------------------------------------------ reverse step
// Transposed solve (I - Aw)^T mu = b for a block of nb cells (2 nb unknowns), partial pivoting.
__device__ bool solve_T(int n, double (*Aw)[2 * AMAXB], const double* b, double* mu) {
  double Mx[2 * AMAXB][2 * AMAXB + 1];
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) Mx[i][j] = (i == j ? 1.0 : 0.0) - Aw[j][i];
    Mx[i][n] = b[i];
  }
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(Mx[r][c]) > fabs(Mx[p][c])) p = r;
    if (!(Mx[p][c] != 0.0) || !isfinite(Mx[p][c])) return false;
    if (p != c)
      for (int j = 0; j <= n; ++j) {
        double t = Mx[p][j];
        Mx[p][j] = Mx[c][j];
        Mx[c][j] = t;
      }
    for (int r = c + 1; r < n; ++r) {
      double f = Mx[r][c] / Mx[c][c];
      if (f != 0.0)
        for (int j = c; j <= n; ++j) Mx[r][j] -= f * Mx[c][j];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = Mx[i][n];
    for (int j = i + 1; j < n; ++j) s -= Mx[i][j] * mu[j];
    mu[i] = s / Mx[i][i];
  }
  return true;
}

// Adjoint of one block (one thread: the instance's lane of warp 0): reads lambda of the outputs (lw, lr, lm, lx
// in post-merge numbering), writes the accumulators of the block cells' U^n and widths, the face adjoints of
// F_left/F_right and the boundary faces' positions, and returns the dt and tau contributions.
__device__ __noinline__ bool block_adjoint(const ADev& A, AInst& I, const StepRec& R, int lo, int hi, int cell0,
                                           int& pbf, double dt, double& lam_dt, double& lam_tau) {
  const long long o = I.off;
  const int nb = hi - lo + 1, n = 2 * nb;
  double Ur[AMAXB], Um[AMAXB], Uw[AMAXB], Wr[AMAXB], Wm[AMAXB], hl[AMAXB], gv[AMAXB][2];
  double Fv[AMAXB + 1][2], wcv[AMAXB + 1];
  double DF[AMAXB + 1][3][5];  // per interior face: d(F0, F1, w)/d(W_l r, W_l m, W_r r, W_r m, tau)
  int ph[AMAXB];
  for (int q = 0; q < nb; ++q) {
    Ur[q] = A.pr[o + lo + q];
    Um[q] = A.pm[o + lo + q];
    Uw[q] = A.pw[o + lo + q];
    ph[q] = A.pph[o + lo + q];
    Wr[q] = R.Wr[cell0 + q];
    Wm[q] = R.Wm[cell0 + q];
  }
  Fv[0][0] = A.F0[o + lo];
  Fv[0][1] = A.F1[o + lo];
  Fv[nb][0] = A.F0[o + hi + 1];
  Fv[nb][1] = A.F1[o + hi + 1];
  wcv[0] = wcv[nb] = 0.0;
  for (int q = 1; q < nb; ++q) {
    Dual<5> rl = dvar<5>(Wr[q - 1], 0), ml = dvar<5>(Wm[q - 1], 1), rr = dvar<5>(Wr[q], 2), mr = dvar<5>(Wm[q], 3);
    Dual<5> ta = dvar<5>(I.tau, 4);
    Dual<5> f0, f1, wq;
    if (A.pfpb[o + lo + q]) {
      if (!pb_face_d<5>(c_fluid, ph[q - 1], ph[q], rl, ml, rr, mr, ta, R.ppl[pbf], R.ppr[pbf], f0, f1, wq))
        return false;
      pbf++;
    } else {
      hll_d<5>(c_fluid.ph[ph[q]], rl, ml, rr, mr, f0, f1);
      wq = dconst<5>(0.0);
    }
    Fv[q][0] = f0.v;
    Fv[q][1] = f1.v;
    wcv[q] = wq.v;
    for (int k = 0; k < 5; ++k) {
      DF[q][0][k] = f0.d[k];
      DF[q][1][k] = f1.d[k];
      DF[q][2][k] = wq.d[k];
    }
  }
  for (int q = 0; q < nb; ++q) {
    hl[q] = __fma_rn(wcv[q + 1] - wcv[q], dt, Uw[q]);
    gv[q][0] = (Uw[q] * Ur[q] - dt * (Fv[q + 1][0] - Fv[q][0])) / hl[q];
    gv[q][1] = (Uw[q] * Um[q] - dt * (Fv[q + 1][1] - Fv[q][1])) / hl[q];
  }
  // lambda of the outputs
  double lwq[AMAXB], lu[AMAXB][2], lxf[AMAXB + 1], lwc_out[AMAXB + 1];
  for (int q = 0; q < nb; ++q) {
    lwq[q] = A.lw[o + lo + q];
    lu[q][0] = A.lr[o + lo + q];
    lu[q][1] = A.lm[o + lo + q];
  }
  for (int q = 0; q <= nb; ++q) {
    lxf[q] = (q > 0 && q < nb && A.pfpb[o + lo + q]) ? A.lx[o + lo + q] : 0.0;
    lwc_out[q] = (q > 0 && q < nb) ? dt * (lwq[q - 1] - lwq[q] + lxf[q]) : 0.0;
  }
  // Aw = dg/dW and b = lambda_W
  double Aw[2 * AMAXB][2 * AMAXB], b[2 * AMAXB], mu[2 * AMAXB];
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) Aw[i][j] = 0.0;
    b[i] = lu[i >> 1][i & 1];
  }
  for (int q = 1; q < nb; ++q) {
    const int il = q - 1, ir = q;
    const double cl = dt / hl[il], cr = dt / hl[ir];
    for (int c = 0; c < 2; ++c)
      for (int k = 0; k < 4; ++k) {
        const int col = 2 * (il + (k >> 1)) + (k & 1);  // k 0,1 -> W_il; 2,3 -> W_ir
        Aw[2 * il + c][col] += -cl * DF[q][c][k] - gv[il][c] * cl * DF[q][2][k];
        Aw[2 * ir + c][col] += cr * DF[q][c][k] + gv[ir][c] * cr * DF[q][2][k];
      }
    for (int k = 0; k < 4; ++k) b[2 * (il + (k >> 1)) + (k & 1)] += lwc_out[q] * DF[q][2][k];
  }
  if (!solve_T(n, Aw, b, mu)) return false;
  // parameter adjoints
  for (int q = 0; q < nb; ++q) {
    const double s = Uw[q] / hl[q];
    A.nr[o + lo + q] += s * mu[2 * q];
    A.nm[o + lo + q] += s * mu[2 * q + 1];
    A.nw[o + lo + q] += lwq[q] + (mu[2 * q] * (Ur[q] - gv[q][0]) + mu[2 * q + 1] * (Um[q] - gv[q][1])) / hl[q];
    const double dwc = wcv[q + 1] - wcv[q];
    lam_dt += (mu[2 * q] * (-(Fv[q + 1][0] - Fv[q][0]) - gv[q][0] * dwc) +
               mu[2 * q + 1] * (-(Fv[q + 1][1] - Fv[q][1]) - gv[q][1] * dwc)) /
                  hl[q] +
              lwq[q] * dwc;
  }
  A.LF0[o + lo] += dt / hl[0] * mu[0];
  A.LF1[o + lo] += dt / hl[0] * mu[1];
  A.LF0[o + hi + 1] += -dt / hl[nb - 1] * mu[2 * nb - 2];
  A.LF1[o + hi + 1] += -dt / hl[nb - 1] * mu[2 * nb - 1];
  for (int q = 1; q < nb; ++q) {
    const int il = q - 1, ir = q;
    const double cl = dt / hl[il], cr = dt / hl[ir];
    double lf0 = -cl * mu[2 * il] + cr * mu[2 * ir];
    double lf1 = -cl * mu[2 * il + 1] + cr * mu[2 * ir + 1];
    double lwc = -cl * (mu[2 * il] * gv[il][0] + mu[2 * il + 1] * gv[il][1]) +
                 cr * (mu[2 * ir] * gv[ir][0] + mu[2 * ir + 1] * gv[ir][1]) + lwc_out[q];
    lam_tau += lf0 * DF[q][0][4] + lf1 * DF[q][1][4] + lwc * DF[q][2][4];
    if (A.pfpb[o + lo + q]) {
      lam_dt += lxf[q] * wcv[q];
      A.nx[o + lo + q] += lxf[q];
    }
  }
  return true;
}

// The blocks of one reverse step (one thread: the instance's lane of warp 0): block_adjoint on each, in the
// order the forward step solved them.
__device__ __noinline__ void serial_rev_blocks(const ADev& A, AInst& I, SharedStep& S) {
  const StepRec& R = *S.rec;
  const double dt = R.dt;
  int cell0 = 0, pbf = 0;
  double ltau = 0.0;
  for (int b = 0; b < S.n_blk; ++b) {
    if (!block_adjoint(A, I, R, S.blo[b], S.bhi[b], cell0, pbf, dt, S.lam_dt, ltau)) {
      S.bad = 1;
      afail(I, IMEXDS_ERR_STATE, 3);
      break;
    }
    cell0 += S.bhi[b] - S.blo[b] + 1;
  }
  I.lam_tau += ltau;
}

// One reverse step for the instances of this CTA that take part (S.act), the step taped in slot S.slot with the
// record *S.rec. Warp w runs the data-parallel parts of instance base + w; lane l of warp 0 the transposed block
// solves of instance base + l (serial_rev_blocks). Every thread of the CTA calls it.
__device__ void rev_step_grp(const ADev& A, SharedStep* SS, int base, int G) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = lane;
  SharedStep& S = SS[w];
  const bool mine = S.act != 0;
  double lcr[AMAXCR][7];  // lane 0: adjoints of the creation outputs z1, z2, u_C, p_C, rho_C, w1, w2
  if (mine) {
    AInst& I = A.I[base + w];
    const StepRec& R = *S.rec;
    const long long o = I.off;
    const long long to = (long long)S.slot * A.stride + o;
    const int Mn = A.tp_M[(long long)S.slot * A.n_inst + base + w];
    const double dt = R.dt;
    // (a) splits^T on the adjoint list, then the created cells leave it (insertion^T)
    if (lane == 0) {
      S.lam_dt = 0.0;
      int Mc = I.M;
      for (int q = R.n_split - 1; q >= 0; --q) {
        const int i = R.sp_i[q];
        A.lr[o + i] += A.lr[o + i + 1];
        A.lm[o + i] += A.lm[o + i + 1];
        if (R.sp_case[q] == 1) {
          A.lw[o + i] = A.lw[o + i + 1];
        } else if (R.sp_case[q] == 3) {
          A.lx[o + i] += -A.lw[o + i] + A.lw[o + i + 1];
          A.lw[o + i] = A.lw[o + i + 1];
        }
        lam_erase(A.lw + o, A.lr + o, A.lm + o, A.lx + o, Mc, i + 1);
        Mc--;
      }
      S.n_cr = R.n_cr;
      for (int k = 0; k < R.n_cr; ++k) {
        S.cr_g[k] = R.cr_g[k];
        S.cr_P[k] = R.cr_P[k];
        for (int q = 0; q < 7; ++q) {
          S.cr_o[k][q] = R.cr_o[k][q];
          lcr[k][q] = 0.0;
        }
      }
      // the created cell of event k sits at g_k + k (each earlier event shifted it by one): highest first.
      // w_C = (w2 - w1) dt, rho_C, m_C = rho_C u_C, boundaries at x_g + w1 dt and x_g + w2 dt
      for (int k = R.n_cr - 1; k >= 0; --k) {
        const int p = R.cr_g[k] + k;
        const double* e = R.cr_o[k];
        const double lwC = A.lw[o + p], lrC = A.lr[o + p], lmC = A.lm[o + p];
        const double lxl = A.lx[o + p], lxr = A.lx[o + p + 1];
        lcr[k][5] += (-lwC + lxl) * dt;
        lcr[k][6] += (lwC + lxr) * dt;
        lcr[k][4] += lrC + lmC * e[2];
        lcr[k][2] += lmC * e[4];
        S.lam_dt += lwC * (e[6] - e[5]) + lxl * e[5] + lxr * e[6];
        lam_erase(A.lw + o, A.lr + o, A.lm + o, A.lx + o, Mc, p);
        Mc--;
        A.lx[o + p] = 0.0;  // the fixed face the boundaries were created at
      }
      S.M = Mc;  // post-merge count
      S.n_blk = R.n_blk;
      for (int b = 0; b < R.n_blk; ++b) {
        S.blo[b] = R.blo[b];
        S.bhi[b] = R.bhi[b];
      }
      S.bad = 0;
    }
    __syncwarp();
    // (b) the post-merge list: the taped pre-step list with the recorded merges applied
    cta_copy_d(A.pw + o, A.tp_w + to, Mn);
    cta_copy_d(A.pr + o, A.tp_r + to, Mn);
    cta_copy_d(A.pm + o, A.tp_m + to, Mn);
    cta_copy_b(A.pph + o, A.tp_ph + to, Mn);
    cta_copy_b(A.pfpb + o, A.tp_fpb + to, Mn + 1);
    __syncwarp();
    if (lane == 0) {
      int Mc = Mn;
      for (int q = 0; q < R.n_merge; ++q) {
        const int a = R.mg_a[q], b = R.mg_b[q];
        const double* v = R.mg_v[q];
        double wm = v[0] + v[3];
        A.pr[o + a] = (v[0] * v[1] + v[3] * v[4]) / wm;
        A.pm[o + a] = (v[0] * v[2] + v[3] * v[5]) / wm;
        A.pw[o + a] = wm;
        list_erase(A.pw + o, A.pr + o, A.pm + o, A.pph + o, A.pfpb + o, nullptr, nullptr, nullptr, nullptr, Mc, b);
        Mc--;
      }
      if (Mc != S.M) S.bad = 1;
    }
    __syncwarp();
    if (S.bad) {
      if (lane == 0) afail(I, IMEXDS_ERR_STATE, 2);
    } else {
      const int M = S.M;
      // (c) zero the accumulators; explicit fluxes at U^n (post-merge)
      cta_zero(A.nw + o, M);
      cta_zero(A.nr + o, M);
      cta_zero(A.nm + o, M);
      cta_zero(A.nx + o, M + 1);
      cta_zero(A.LF0 + o, M + 1);
      cta_zero(A.LF1 + o, M + 1);
      for (int g = tid; g <= M; g += 32) {
        if (face_in_block(S, g)) continue;
        if (S.n_cr && cr_at(S, g) >= 0) continue;
        double f0, f1;
        if (g == 0)
          phys_flux_fast(c_fluid.ph[A.pph[o]], A.pr[o], A.pm[o], f0, f1);
        else if (g == M)
          phys_flux_fast(c_fluid.ph[A.pph[o + M - 1]], A.pr[o + M - 1], A.pm[o + M - 1], f0, f1);
        else
          hll_fast(c_fluid.ph[A.pph[o + g]], A.pr[o + g - 1], A.pm[o + g - 1], A.pr[o + g], A.pm[o + g], f0, f1);
        A.F0[o + g] = f0;
        A.F1[o + g] = f1;
      }
    }
    __syncwarp();
  }
  __syncthreads();
  if (w == 0 && lane < G && SS[lane].act && !SS[lane].bad) serial_rev_blocks(A, A.I[base + lane], SS[lane]);
  __syncthreads();
  if (mine && !S.bad) {
    AInst& I = A.I[base + w];
    const StepRec& R = *S.rec;
    const long long o = I.off;
    const long long to = (long long)S.slot * A.stride + o;
    const int Mn = A.tp_M[(long long)S.slot * A.n_inst + base + w];
    const double dt = R.dt;
    const int M = S.M;
    // (e) explicit sweep^T: face adjoints from the explicit cells, then the face Jacobians at U^n
    for (int g = tid; g <= M; g += 32) {
      if (face_in_block(S, g)) continue;
      if (S.n_cr && cr_at(S, g) >= 0) {  // a creation face: its adjoint goes to the event (lane 0, below)
        A.CL0[o + g] = A.CL1[o + g] = A.CR0[o + g] = A.CR1[o + g] = 0.0;
        continue;
      }
      double l0 = A.LF0[o + g], l1 = A.LF1[o + g];
      if (g > 0 && !in_block(S, g - 1)) {
        const double c = dt / cell_upd(A.F0 + o, A.F1 + o, S, g - 1, A.pw[o + g - 1], dt).h1;
        l0 -= c * A.lr[o + g - 1];
        l1 -= c * A.lm[o + g - 1];
      }
      if (g < M && !in_block(S, g)) {
        const double c = dt / cell_upd(A.F0 + o, A.F1 + o, S, g, A.pw[o + g], dt).h1;
        l0 += c * A.lr[o + g];
        l1 += c * A.lm[o + g];
      }
      double cl0 = 0.0, cl1 = 0.0, cr0 = 0.0, cr1 = 0.0;
      if (g == 0 || g == M) {
        const int i = (g == 0) ? 0 : M - 1;
        Dual<2> rr = dvar<2>(A.pr[o + i], 0), mm = dvar<2>(A.pm[o + i], 1), f0, f1;
        phys_flux_d<2>(c_fluid.ph[A.pph[o + i]], rr, mm, f0, f1);
        const double a0 = l0 * f0.d[0] + l1 * f1.d[0], a1 = l0 * f0.d[1] + l1 * f1.d[1];
        if (g == 0) {
          cr0 = a0;
          cr1 = a1;
        } else {
          cl0 = a0;
          cl1 = a1;
        }
      } else {
        Dual<4> rl = dvar<4>(A.pr[o + g - 1], 0), ml = dvar<4>(A.pm[o + g - 1], 1);
        Dual<4> rr = dvar<4>(A.pr[o + g], 2), mr = dvar<4>(A.pm[o + g], 3), f0, f1;
        hll_d<4>(c_fluid.ph[A.pph[o + g]], rl, ml, rr, mr, f0, f1);
        cl0 = l0 * f0.d[0] + l1 * f1.d[0];
        cl1 = l0 * f0.d[1] + l1 * f1.d[1];
        cr0 = l0 * f0.d[2] + l1 * f1.d[2];
        cr1 = l0 * f0.d[3] + l1 * f1.d[3];
      }
      A.CL0[o + g] = cl0;
      A.CL1[o + g] = cl1;
      A.CR0[o + g] = cr0;
      A.CR1[o + g] = cr1;
    }
    double ldt_part = 0.0;
    for (int i = tid; i < M; i += 32) {
      if (in_block(S, i)) continue;
      const double wi = A.pw[o + i], lr = A.lr[o + i], lm = A.lm[o + i];
      const CellUpd c = cell_upd(A.F0 + o, A.F1 + o, S, i, wi, dt);
      const double dF = (c.fr0 - c.fl0) * lr + (c.fr1 - c.fl1) * lm;
      if (c.wl == 0.0 && c.wr == 0.0) {
        A.nr[o + i] += lr;
        A.nm[o + i] += lm;
        A.nw[o + i] += A.lw[o + i] + dt * dF / (wi * wi);
        ldt_part -= dF / wi;
      } else {  // next to a creation face: the width moves with w1 / w2
        const double r1 = (wi * A.pr[o + i] - dt * (c.fr0 - c.fl0)) / c.h1;
        const double m1 = (wi * A.pm[o + i] - dt * (c.fr1 - c.fl1)) / c.h1;
        const double sc = wi / c.h1, dw = c.wl - c.wr;
        A.nr[o + i] += lr * sc;
        A.nm[o + i] += lm * sc;
        A.nw[o + i] += A.lw[o + i] + (lr * (A.pr[o + i] - r1) + lm * (A.pm[o + i] - m1)) / c.h1;
        ldt_part += (-dF - (lr * r1 + lm * m1) * dw) / c.h1 + A.lw[o + i] * dw;
      }
    }
    __syncwarp();
    // (f) gather the face contributions into the cells (faces inside a block contribute nothing here)
    for (int i = tid; i < M; i += 32) {
      double a0 = 0.0, a1 = 0.0;
      if (!face_in_block(S, i)) {
        a0 += A.CR0[o + i];
        a1 += A.CR1[o + i];
      }
      if (!face_in_block(S, i + 1)) {
        a0 += A.CL0[o + i + 1];
        a1 += A.CL1[o + i + 1];
      }
      A.nr[o + i] += a0;
      A.nm[o + i] += a1;
    }
    const double tot = warp_sum(ldt_part);
    __syncwarp();
    // (g') creation faces^T (lane 0): the two cells beside each creation face see its per-side fluxes and
    //      move its faces; the event's outputs go back to the adjacent states and tau through the implicit
    //      function theorem on the creation system
    if (lane == 0) {
      for (int k = 0; k < S.n_cr; ++k) {
        const int g = S.cr_g[k];
        const double* e = S.cr_o[k];
        double* L = lcr[k];
        for (int side = 0; side < 2; ++side) {
          const int i = g - 1 + side;
          const double wi = A.pw[o + i], lr = A.lr[o + i], lm = A.lm[o + i], lw = A.lw[o + i];
          const CellUpd c = cell_upd(A.F0 + o, A.F1 + o, S, i, wi, dt);
          const double r1 = (wi * A.pr[o + i] - dt * (c.fr0 - c.fl0)) / c.h1;
          const double m1 = (wi * A.pm[o + i] - dt * (c.fr1 - c.fl1)) / c.h1;
          const double sgn = side ? 1.0 : -1.0;  // the flux enters the right face of cell g-1, the left of cell g
          const double a0 = sgn * dt / c.h1 * lr, a1 = sgn * dt / c.h1 * lm;
          const double zs = side ? e[1] : e[0];
          L[side] += -a0 - a1 * e[2];  // (-z, -z u_C + p_C)
          L[2] += -a1 * zs;
          L[3] += a1;
          L[5 + side] += -sgn * dt * (lw - (lr * r1 + lm * m1) / c.h1);  // h1 = w + (w_l - w_r) dt
        }
        Dual<5> rl = dvar<5>(A.pr[o + g - 1], 0), ml = dvar<5>(A.pm[o + g - 1], 1);
        Dual<5> rr = dvar<5>(A.pr[o + g], 2), mr = dvar<5>(A.pm[o + g], 3), ta = dvar<5>(I.tau, 4);
        Dual<5> out[7];
        if (!creation_d<5>(c_fluid, S.cr_P[k], rl, ml, rr, mr, ta, R.cr_x[k], out)) {
          afail(I, IMEXDS_ERR_STATE, 3);
          break;
        }
        double lt[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int q = 0; q < 7; ++q)
          for (int kk = 0; kk < 5; ++kk) lt[kk] += L[q] * out[q].d[kk];
        A.nr[o + g - 1] += lt[0];
        A.nm[o + g - 1] += lt[1];
        A.nr[o + g] += lt[2];
        A.nm[o + g] += lt[3];
        I.lam_tau += lt[4];
      }
    }
    // (g) merges^T and (h) dt^T (lane 0)
    if (lane == 0) {
      double lam_dt = S.lam_dt + tot;
      int Mc = M;
      for (int q = R.n_merge - 1; q >= 0; --q) {
        const int a = R.mg_a[q], b = R.mg_b[q];
        const double* v = R.mg_v[q];
        const double wm = v[0] + v[3];
        const double rm = (v[0] * v[1] + v[3] * v[4]) / wm, mm = (v[0] * v[2] + v[3] * v[5]) / wm;
        const double Lw = A.nw[o + a], Lr = A.nr[o + a], Lm = A.nm[o + a];
        lam_open(A.nw + o, A.nr + o, A.nm + o, A.nx + o, Mc, b);
        Mc++;
        A.nx[o + b] = 0.0;
        A.nr[o + a] = Lr * v[0] / wm;
        A.nm[o + a] = Lm * v[0] / wm;
        A.nw[o + a] = Lw + (Lr * (v[1] - rm) + Lm * (v[2] - mm)) / wm;
        A.nr[o + b] = Lr * v[3] / wm;
        A.nm[o + b] = Lm * v[3] / wm;
        A.nw[o + b] = Lw + (Lr * (v[4] - rm) + Lm * (v[5] - mm)) / wm;
      }
      if (R.clipped) {
        I.lam_t = -lam_dt;
      } else {
        lam_dt += I.lam_t;
        const int k = R.kmax;
        const double rk = A.tp_r[to + k], mk = A.tp_m[to + k];
        const double S_ = fabs(mk / rk) + c_fluid.ph[A.tp_ph[to + k]].a;
        const double lS = -lam_dt * dt / S_;
        const double sg = (mk > 0.0) ? 1.0 : ((mk < 0.0) ? -1.0 : 0.0);
        A.nm[o + k] += lS * sg / rk;
        A.nr[o + k] += -lS * sg * mk / (rk * rk);
      }
      I.M = Mc;
      if (Mc != Mn) afail(I, IMEXDS_ERR_STATE, 4);
    }
    __syncwarp();
    // lambda^n <- accumulators
    cta_copy_d(A.lw + o, A.nw + o, Mn);
    cta_copy_d(A.lr + o, A.nr + o, Mn);
    cta_copy_d(A.lm + o, A.nm + o, Mn);
    cta_copy_d(A.lx + o, A.nx + o, Mn + 1);
  }
  __syncwarp();
}

__device__ void save_list(const ADev& A, AInst& I, long long dst_off, double* w, double* r, double* m,
                          unsigned char* ph, unsigned char* fpb, int* fj, double* fx, double* pl, double* pr) {
  const long long o = I.off;
  cta_copy_d(w + dst_off, A.w + o, I.M);
  cta_copy_d(r + dst_off, A.r + o, I.M);
  cta_copy_d(m + dst_off, A.m + o, I.M);
  cta_copy_b(ph + dst_off, A.ph + o, I.M);
  if (fpb) cta_copy_b(fpb + dst_off, A.fpb + o, I.M + 1);
  if (fj) cta_copy_i(fj + dst_off, A.fj + o, I.M + 1);
  if (fx) cta_copy_d(fx + dst_off, A.fx + o, I.M + 1);
  if (pl) cta_copy_d(pl + dst_off, A.pwl + o, I.M + 1);
  if (pr) cta_copy_d(pr + dst_off, A.pwr + o, I.M + 1);
}
__device__ void load_list(const ADev& A, AInst& I, long long src_off, int M) {
  const long long o = I.off;
  cta_copy_d(A.w + o, A.ck_w + src_off, M);
  cta_copy_d(A.r + o, A.ck_r + src_off, M);
  cta_copy_d(A.m + o, A.ck_m + src_off, M);
  cta_copy_b(A.ph + o, A.ck_ph + src_off, M);
  cta_copy_b(A.fpb + o, A.ck_fpb + src_off, M + 1);
  cta_copy_i(A.fj + o, A.ck_fj + src_off, M + 1);
  cta_copy_d(A.fx + o, A.ck_fx + src_off, M + 1);
  cta_copy_d(A.pwl + o, A.ck_pwl + src_off, M + 1);
  cta_copy_d(A.pwr + o, A.ck_pwr + src_off, M + 1);
}

// The whole adjoint of the CTA's instances, base + w for warp w < G (G = blockDim.x / 32): replay with
// checkpoints, then the segments from last to first, recomputed (all but the last, taped during the replay) and
// reversed. The instances step in lockstep; one that has finished its program, or failed, sits out.
__global__ void __launch_bounds__(ATHREADS, 2) k_adjoint(ADev A) {
  const int G = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int base = blockIdx.x * G, ii = base + w;
  __shared__ SharedStep SS[AWARPS];
  __shared__ int s_max[AWARPS];
  SharedStep& S = SS[w];
  const bool valid = ii < A.n_inst;
  // CTA-wide maximum of a value that is uniform within each warp; every thread calls it
  auto cta_max = [&](int v) -> int {
    __syncthreads();
    if (lane == 0) s_max[w] = v;
    __syncthreads();
    int m = s_max[0];
    for (int q = 1; q < G; ++q) m = max(m, s_max[q]);
    return m;
  };
  // phase A: replay from the initial states, a checkpoint every k steps. The steps of the last segment (as the
  // forward run's step count places it) are taped on the way, so that segment needs no recompute; with k at
  // least the run's length the whole adjoint is one taped replay and one reverse sweep.
  int n = 0, taped = 0, tape_from = 0;
  bool run = valid;
  if (valid) {
    const int ne = A.I[ii].nexp;
    tape_from = (ne > 0) ? ((ne - 1) / A.k) * A.k : 0;
  }
  for (;;) {
    if (run && n % A.k == 0) {
      AInst& I = A.I[ii];
      const int c = n / A.k;
      if (c >= A.n_ck) {
        if (lane == 0) afail(I, IMEXDS_ERR_CAPACITY);
        run = false;
      } else {
        save_list(A, I, (long long)c * A.stride + I.off, A.ck_w, A.ck_r, A.ck_m, A.ck_ph, A.ck_fpb, A.ck_fj, A.ck_fx,
                  A.ck_pwl, A.ck_pwr);
        if (lane == 0) {
          ACk& h = A.ck_h[(long long)c * A.n_inst + ii];
          h.done = I.done;
          h.M = I.M;
          h.status = I.status;
          h.pc = I.pc;
          h.t = I.t;
        }
      }
      __syncwarp();
    }
    if (lane == 0) {
      int go = 0;
      double te = -1.0;
      if (run) go = prog_next(A, A.I[ii], te) ? 1 : 0;
      const bool tape = go && n >= tape_from && n - tape_from < A.k;
      S.act = go;
      S.t_end = te;
      S.rec = tape ? A.rec + (long long)(n - tape_from) * A.n_inst + ii : nullptr;
      S.slot = n - tape_from;
    }
    __syncwarp();
    run = S.act != 0;
    if (!__syncthreads_or(run ? 1 : 0)) break;
    fwd_step_grp(A, SS, base, G);
    if (run) {
      if (S.rec) ++taped;
      ++n;
    }
  }
  bool alive = false;
  if (valid) {
    AInst& I = A.I[ii];
    if (lane == 0) I.nsteps = n;
    save_list(A, I, I.off, A.fin_w, A.fin_r, A.fin_m, A.fin_ph, nullptr, nullptr, nullptr, nullptr, nullptr);
    if (lane == 0) A.fin_M[ii] = I.M;
    __syncwarp();
    alive = I.status == 0;
    if (alive && I.M != I.M_seed) {
      if (lane == 0) afail(I, IMEXDS_ERR_STATE, 5);
      alive = false;
    }
    __syncwarp();
  }
  // phase B: segments from last to first
  const int n_seg = alive ? (n + A.k - 1) / A.k : 0;
  const int max_seg = cta_max(n_seg);
  for (int sg = max_seg - 1; sg >= 0; --sg) {
    const int first = sg * A.k;
    const bool part = alive && sg < n_seg;
    const int last = part ? min(n, first + A.k) - 1 : -1;
    // the last segment, taped whole during the replay, which left the list at the state after its last step
    const bool taped_whole = part && sg == n_seg - 1 && first == tape_from && taped == last - first + 1;
    bool rerun = part && !taped_whole;
    const int Mlam = part ? A.I[ii].M : 0;  // the adjoint list length (cells of the state after step last)
    if (rerun) {
      AInst& I = A.I[ii];
      const ACk& h = A.ck_h[(long long)sg * A.n_inst + ii];
      load_list(A, I, (long long)sg * A.stride + I.off, h.M);
      if (lane == 0) {
        I.M = h.M;
        I.t = h.t;
        I.pc = h.pc;
        I.done = h.done;
      }
      __syncwarp();
    }
    const int last_rerun = cta_max(rerun ? last : -1);
    for (int s = first; s <= last_rerun; ++s) {
      const bool go = rerun && s <= last;
      if (lane == 0) {
        int ok = 0;
        double te = -1.0;
        if (go) {
          ok = prog_next(A, A.I[ii], te) ? 1 : 0;
          if (!ok) afail(A.I[ii], IMEXDS_ERR_STATE, 1);
          S.rec = A.rec + (long long)(s - first) * A.n_inst + ii;
          S.slot = s - first;
        }
        S.act = ok;
        S.t_end = te;
      }
      __syncwarp();
      if (go && !S.act) {  // the program ended early in a recomputed segment
        alive = false;
        rerun = false;
      }
      __syncthreads();
      fwd_step_grp(A, SS, base, G);
      if (go && alive && A.I[ii].status) {
        alive = false;
        rerun = false;
      }
    }
    const bool rpart = part && alive;
    if (rpart && lane == 0) A.I[ii].M = Mlam;
    __syncwarp();
    const int last_rev = cta_max(rpart ? last : -1);
    for (int s = last_rev; s >= first; --s) {
      const bool go = rpart && alive && s <= last;
      if (lane == 0) {
        S.act = go ? 1 : 0;
        if (go) {
          S.rec = A.rec + (long long)(s - first) * A.n_inst + ii;
          S.slot = s - first;
        }
      }
      __syncthreads();
      rev_step_grp(A, SS, base, G);
      if (go && A.I[ii].status) alive = false;
    }
  }
}

}  // namespace adj
}  // namespace imexds
