// imexds: CUDA kernels and C-ABI of the explicit-implicit domain-splitting scheme for 1-D isothermal
// two-phase flow with phase transition (May & Thein, arXiv 2211.00705), FP64, sm_103a.
//
// Device layout (per instance, batched):
//   * background lattice: rho[], m[] and the velocity u[] = m/rho (double buffered, parity per
//     instance), phase[] (uint8), own[] (int32: zone slot that currently owns the lattice cell, -1 if
//     it is an explicit cell);
//   * zones: fixed-capacity records holding the irregular cells next to phase boundaries (a maximal
//     run of cells whose faces are not all on the lattice) with their widths, phases, face kinds and
//     boundary positions. Zones are kept at least ZONE_GAP lattice cells apart (closer zones are
//     joined), so every step's work on a zone touches no other zone.
//
// One time step, per-step schedule = five kernels (replayed from a CUDA graph by the host loop):
//   k_pre    (thread per zone)  phase-boundary solves at U^n -> predicted widths -> merge marks (Sec. 3.4)
//   k_plan   (thread per zone)  merges, tiny cells, implicit blocks {k-1,k,k+1} (Sec. 3.2), owned range
//   k_sweep  (30-cell tile per warp) Algorithm 1 Step 1: HLL fluxes and explicit update of every free
//                               lattice cell; phase-creation detection at free same-phase faces (App. B)
//   k_dts    (thread per zone)  Algorithm 2 (dual time stepping + Part 2) on the zone's blocks with the
//                               App. A boundary solver at the implicit faces and the moving widths
//   k_post   (thread per instance) splits, release of regular cells, creation, t += dt, next dt
// k_sweep and k_dts read U^n only and write disjoint cells of U^{n+1}. Group schedule: k_group, one
// resident CTA per group of instances for the whole call, runs the same device functions (warp 0 one
// instance per lane: solves, plan, dual time, grid management; the other warps the sweep tiles).
// Adjoint: k_adjoint (adjoint.cuh), up to eight instances per CTA, one warp each.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "../../include/imexds.h"
#include "physics.cuh"

using namespace imexds;

namespace {

constexpr int ZC = 16;            // max cells per zone
constexpr int ZB = ZC + 2;        // block index space: zone cells plus one pulled lattice cell per side
constexpr int MAXBLK = ZC;        // max blocks per zone
constexpr int ZONE_GAP = 4;       // minimum number of lattice cells between two zones
constexpr int EV_CAP = 4;         // creation events per instance and step
constexpr int N_STATS = 9;
constexpr long long kRunToMaxSteps = 20000000;  // run_to gives up (IMEXDS_ERR_TIMEOUT) after this many steps

struct Zone {
  int alive, inst, A, B, nc;
  int changed;                   // footprint changed in this step (merge, release, split, creation)
  int merge_mask;
  int pullL, pullR, oA, oB;
  int nblk;
  int blo[MAXBLK], bhi[MAXBLK];  // block ranges in the extended index space (-1 .. nc)
  unsigned tiny_mask;            // bit (e + 1) set for a tiny extended index e
  int ph[ZC];
  int fpb[ZC + 1];               // face k between cells k-1 and k: 1 = phase boundary
  int fj[ZC + 1];                // lattice index of a fixed face
  double w[ZC], r[ZC], m[ZC];
  double fx[ZC + 1];             // position of a phase-boundary face
  double eL0, eL1, eR0, eR1;     // U^n of the first / last owned cell (read by neighbouring sweep cells)
  double wpre[ZC + 1];           // boundary speeds from the solves at U^n (k_pre)
  double pwl[ZC + 1], pwr[ZC + 1]; // last converged star pressures at a boundary face (Newton start)
  double hp[ZC];                 // widths predicted for t^{n+1} on the merged grid (theta of Alg. 2)
};

struct Inst {
  int N, lat_off, zone_off, zone_cap;
  double xL, h, tau;
  double t, dt, lam;  // lam = dt / h (set with dt)
  int status, active, parity, clipped;
  unsigned long long smax_bits;
  int n_ev;
  int n_work;  // entries of the work list of post_inst
  long long stats[N_STATS];  // steps, dts_iters, dts_max, newton, merges, splits, creations, maxiter, pb_solves
};

struct Event {
  int face;
  double w1, w2, rhoC, mC, hl, hr;
  int phC;
};

struct Ctrl {
  double t_end;
  int clip;
  int n_active;
};

struct Dev {
  double* rho[2];
  double* m[2];
  double* u[2];  // u = m / rho of every lattice cell, written by whoever writes the cell (saves a division)
  // The buffers of parity p, selected rather than indexed: a run-time index into the arrays of this
  // struct (a kernel parameter) makes the compiler copy the whole struct to local memory in every thread.
  __device__ __forceinline__ double* R(int p) const { return p ? rho[1] : rho[0]; }
  __device__ __forceinline__ double* M(int p) const { return p ? m[1] : m[0]; }
  __device__ __forceinline__ double* U(int p) const { return p ? u[1] : u[0]; }
  unsigned char* phase;
  int* own;
  Zone* zones;
  Inst* inst;
  Event* ev;
  int2* tiles;  // (instance, first lattice cell)
  int* work;    // per instance (zone_off ..): zones for post_inst (n_work of them)
  Ctrl* ctrl;
};

__constant__ Fluid c_fluid;
__constant__ Opts c_opts;

__device__ inline void set_status(Inst& I, int code) { atomicCAS(&I.status, 0, code); }

__device__ inline unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }

// ------------------------------------------------------------------------------------------ k_pre
// Phase-boundary solves at U^n predict the widths of the cells next to each boundary; a cell that would
// fall below max(alpha_min h, h_i / 2) is marked for merging (Sec. 2.3, Sec. 3.4).
__device__ __noinline__ void pre_zone(const Dev& d, int zi) {
  Zone& Z = d.zones[zi];
  Z.merge_mask = 0;
  if (!Z.alive) return;
  Inst& I = d.inst[Z.inst];
  if (!I.active || I.status) return;
  double dt = I.dt;
  double wf[ZC + 1];
  for (int k = 0; k <= Z.nc; ++k) wf[k] = 0.0;
  long long newton = 0, solves = 0;
  for (int k = 1; k < Z.nc; ++k) {
    if (!Z.fpb[k]) continue;
    PBOut R = pb_solve_warm(c_fluid, c_opts, I.tau, Z.ph[k - 1], Z.r[k - 1], Z.m[k - 1], Z.ph[k], Z.r[k], Z.m[k],
                            Z.pwl[k], Z.pwr[k]);
    newton += R.iters;
    solves++;
    if (!R.ok) {
      set_status(I, IMEXDS_ERR_PB_NOCONV);
      return;
    }
    wf[k] = R.w;
  }
  for (int k = 0; k <= Z.nc; ++k) Z.wpre[k] = wf[k];
  int mask = 0;
  for (int i = 0; i < Z.nc; ++i) {
    if (!(Z.fpb[i] || Z.fpb[i + 1])) continue;
    double hp = Z.w[i] + (wf[i + 1] - wf[i]) * dt;
    if (hp < fmax(c_opts.alpha_min * I.h, 0.5 * Z.w[i])) mask |= 1 << i;
  }
  Z.merge_mask = mask;
  atomicAdd((unsigned long long*)&I.stats[3], (unsigned long long)newton);
  atomicAdd((unsigned long long*)&I.stats[8], (unsigned long long)solves);
}

// remove cell index b of a zone (faces shift down; face b is removed)
__device__ inline void zone_erase_cell(Zone& Z, int b) {
  for (int i = b; i + 1 < Z.nc; ++i) {
    Z.w[i] = Z.w[i + 1];
    Z.r[i] = Z.r[i + 1];
    Z.m[i] = Z.m[i + 1];
    Z.ph[i] = Z.ph[i + 1];
  }
  for (int k = b; k < Z.nc; ++k) {
    Z.fpb[k] = Z.fpb[k + 1];
    Z.fj[k] = Z.fj[k + 1];
    Z.fx[k] = Z.fx[k + 1];
    Z.pwl[k] = Z.pwl[k + 1];
    Z.pwr[k] = Z.pwr[k + 1];
  }
  Z.nc--;
}

// insert an empty cell at index pos of a zone (cells pos.. and faces pos+1.. move up; face pos+1 is a copy of
// face pos); 0 when the zone is full
__device__ inline int zone_insert_cell(Zone& Z, int pos) {
  if (Z.nc >= ZC) return 0;
  for (int i = Z.nc; i > pos; --i) {
    Z.w[i] = Z.w[i - 1];
    Z.r[i] = Z.r[i - 1];
    Z.m[i] = Z.m[i - 1];
    Z.ph[i] = Z.ph[i - 1];
  }
  for (int k = Z.nc + 1; k > pos; --k) {
    Z.fpb[k] = Z.fpb[k - 1];
    Z.fj[k] = Z.fj[k - 1];
    Z.fx[k] = Z.fx[k - 1];
    Z.pwl[k] = Z.pwl[k - 1];
    Z.pwr[k] = Z.pwr[k - 1];
  }
  Z.nc++;
  return 1;
}

// ------------------------------------------------------------------------------------------ k_plan
// Merges (left to right, a marked cell joins its neighbour across its fixed face), then the implicit
// neighbourhoods: at every boundary the smaller adjacent cell is the tiny cell k; {k-1, k, k+1} are
// joined where they overlap. Cells outside the zone taking part (one lattice cell per side) are
// "pulled": the sweep skips them and k_dts updates them.
__device__ __noinline__ void plan_zone(const Dev& d, int zi) {
  Zone& Z = d.zones[zi];
  if (!Z.alive) return;
  Inst& I = d.inst[Z.inst];
  if (!I.active || I.status) return;
  const int cur = I.parity;
  const double* lr = d.R(cur) + I.lat_off;
  const double* lm = d.M(cur) + I.lat_off;
  int mark[ZC];
  for (int i = 0; i < Z.nc; ++i) mark[i] = (Z.merge_mask >> i) & 1;
  long long merges = 0;
  for (int i = 0; i < Z.nc; ++i) {
    if (!mark[i]) continue;
    bool left_fixed = !Z.fpb[i] && !(i == 0 && Z.A == 0);
    bool right_fixed = !Z.fpb[i + 1] && !(i == Z.nc - 1 && Z.B == I.N);
    if (left_fixed) {
      if (i == 0) {  // join the lattice cell A-1 (free: zones are ZONE_GAP apart)
        int j = Z.A - 1;
        double wl = I.h, rl = lr[j], ml = lm[j];
        double wm = wl + Z.w[0];
        double rm = (wl * rl + Z.w[0] * Z.r[0]) / wm;
        double mm = (wl * ml + Z.w[0] * Z.m[0]) / wm;
        Z.w[0] = wm;
        Z.r[0] = rm;
        Z.m[0] = mm;
        Z.A = j;
        Z.fj[0] = j;
        mark[0] = 0;
      } else {
        int a = i - 1;
        double wm = Z.w[a] + Z.w[i];
        double rm = (Z.w[a] * Z.r[a] + Z.w[i] * Z.r[i]) / wm;
        double mm = (Z.w[a] * Z.m[a] + Z.w[i] * Z.m[i]) / wm;
        Z.w[a] = wm;
        Z.r[a] = rm;
        Z.m[a] = mm;
        zone_erase_cell(Z, i);
        for (int q = i; q < Z.nc; ++q) mark[q] = mark[q + 1];
        mark[a] = 0;
        --i;
      }
    } else if (right_fixed) {
      if (i == Z.nc - 1) {  // join the lattice cell B
        int j = Z.B;
        double wr = I.h, rr = lr[j], mr = lm[j];
        double wm = Z.w[i] + wr;
        double rm = (Z.w[i] * Z.r[i] + wr * rr) / wm;
        double mm = (Z.w[i] * Z.m[i] + wr * mr) / wm;
        Z.w[i] = wm;
        Z.r[i] = rm;
        Z.m[i] = mm;
        Z.B = j + 1;
        Z.fj[Z.nc] = j + 1;
      } else {
        int b = i + 1;
        double wm = Z.w[i] + Z.w[b];
        double rm = (Z.w[i] * Z.r[i] + Z.w[b] * Z.r[b]) / wm;
        double mm = (Z.w[i] * Z.m[i] + Z.w[b] * Z.m[b]) / wm;
        Z.w[i] = wm;
        Z.r[i] = rm;
        Z.m[i] = mm;
        zone_erase_cell(Z, b);
        for (int q = b; q < Z.nc; ++q) mark[q] = mark[q + 1];
      }
      mark[i] = 0;
    } else {
      set_status(I, IMEXDS_ERR_VANISH);
      return;
    }
    merges++;
  }
  if (merges) {
    atomicAdd((unsigned long long*)&I.stats[4], (unsigned long long)merges);
    Z.changed = 1;
  }
  // widths predicted for t^{n+1} (Sec. 3.1 treats the implicit neighbourhood on the mesh at t^{n+1});
  // after a merge the boundary speeds are solved again from the merged states
  {
    double wf[ZC + 1];
    for (int k = 0; k <= Z.nc; ++k) wf[k] = 0.0;
    for (int k = 1; k < Z.nc; ++k) {
      if (!Z.fpb[k]) continue;
      if (merges) {
        PBOut R = pb_solve_warm(c_fluid, c_opts, I.tau, Z.ph[k - 1], Z.r[k - 1], Z.m[k - 1], Z.ph[k], Z.r[k], Z.m[k],
                                Z.pwl[k], Z.pwr[k]);
        atomicAdd((unsigned long long*)&I.stats[3], (unsigned long long)R.iters);
        if (!R.ok) {
          set_status(I, IMEXDS_ERR_PB_NOCONV);
          return;
        }
        wf[k] = R.w;
      } else {
        wf[k] = Z.wpre[k];
      }
    }
    for (int i = 0; i < Z.nc; ++i) Z.hp[i] = Z.w[i] + (wf[i + 1] - wf[i]) * I.dt;
  }
  // implicit neighbourhoods in the extended index space
  int emin = (Z.A > 0) ? -1 : 0;
  int emax = (Z.B < I.N) ? Z.nc : Z.nc - 1;
  int nblk = 0;
  unsigned tiny = 0;
  for (int k = 1; k < Z.nc; ++k) {
    if (!Z.fpb[k]) continue;
    int kt = (Z.w[k - 1] < Z.w[k]) ? k - 1 : k;
    tiny |= 1u << (kt + 1);
    int lo = max(kt - 1, emin), hi = min(kt + 1, emax);
    if (nblk > 0 && lo <= Z.bhi[nblk - 1]) {
      Z.bhi[nblk - 1] = max(Z.bhi[nblk - 1], hi);
    } else {
      if (nblk == MAXBLK) {
        set_status(I, IMEXDS_ERR_CAPACITY);
        return;
      }
      Z.blo[nblk] = lo;
      Z.bhi[nblk] = hi;
      nblk++;
    }
  }
  Z.nblk = nblk;
  Z.tiny_mask = tiny;
  Z.pullL = (nblk > 0 && Z.blo[0] == -1) ? 1 : 0;
  Z.pullR = (nblk > 0 && Z.bhi[nblk - 1] == Z.nc) ? 1 : 0;
  Z.oA = Z.A - Z.pullL;
  Z.oB = Z.B + Z.pullR;
  if (Z.pullL) {
    Z.eL0 = lr[Z.A - 1];
    Z.eL1 = lm[Z.A - 1];
  } else {
    Z.eL0 = Z.r[0];
    Z.eL1 = Z.m[0];
  }
  if (Z.pullR) {
    Z.eR0 = lr[Z.B];
    Z.eR1 = lm[Z.B];
  } else {
    Z.eR0 = Z.r[Z.nc - 1];
    Z.eR1 = Z.m[Z.nc - 1];
  }
  int* own = d.own + I.lat_off;
  for (int j = Z.oA; j < Z.oB; ++j) own[j] = zi;
}

// ------------------------------------------------------------------------------------------ sweep
// Algorithm 1, Step 1 on a tile of one instance, one warp per tile: HLL fluxes from U^n at the faces of
// free lattice cells, the explicit update of Eq. update expl time (Eq. godunov_meth:nonunif next to a
// creation face) and the tile's wave-speed maximum. Lane l owns cell j0+l and the face on its left; the
// right-face flux comes from lane l+1. u = m/rho and the momentum flux are formed once per cell. A face next to a zone sees the zone's edge state.
// CREATION adds detection and the creation solve of App. B at faces between two free cells.
struct CellS {
  int ow, ph;  // owner (-1 free, >= 0 zone slot, -2 outside the domain), phase
  double r, m, u, f1;
};

__device__ inline CellS load_cell(const Dev& d, const Inst& I, int j) {
  // every load is issued unconditionally (index clamped into the instance) and the results are selected,
  // so that the owner, phase and state loads overlap instead of forming a dependent chain
  const bool in = (j >= 0) && (j < I.N);
  const int g = I.lat_off + (in ? j : 0);
  const int ow = d.own[g];
  const int ph = d.phase[g];
  const double r = d.R(I.parity)[g], m = d.M(I.parity)[g], u = d.U(I.parity)[g];
  const bool fr = in && ow < 0;
  CellS c;
  c.ow = in ? ow : -2;
  c.ph = in ? ph : 0;
  c.r = fr ? r : 1.0;
  c.m = fr ? m : 0.0;
  c.u = fr ? u : 0.0;
  c.f1 = fr ? __fma_rn(m, u, pressure_fma(c_fluid.ph[ph], r)) : 0.0;
  return c;
}

__device__ inline CellS shfl_up_cell(const CellS& c) {
  CellS o;
  o.ow = __shfl_up_sync(0xffffffffu, c.ow, 1);
  o.ph = __shfl_up_sync(0xffffffffu, c.ph, 1);
  o.r = __shfl_up_sync(0xffffffffu, c.r, 1);
  o.m = __shfl_up_sync(0xffffffffu, c.m, 1);
  o.u = __shfl_up_sync(0xffffffffu, c.u, 1);
  o.f1 = __shfl_up_sync(0xffffffffu, c.f1, 1);
  return o;
}

// cavitation / nucleation detection at a face between two free cells (App. B)
__device__ inline int detect_face(const CellS& L, const CellS& R) {
  if (L.ow != -1 || R.ow != -1) return 0;
  return creation_detect(c_fluid, R.ph, L.r, L.u, R.r, R.u) ? 1 : 0;
}

struct FaceFlux {
  double F0L, F1L, F0R, F1R, WL, WR;  // seen from the left / right cell; face speeds (creation only)
};

// Flux at face f between cells L and R (at least one of them free). `create`: App. B at this face. The
// common case (two free cells of one phase) is straight-line code; zone edges, domain ends and creation
// adjust inputs or results on their own branches.
template <bool CREATION>
__device__ inline FaceFlux face_flux(const Dev& d, Inst& I, int ii, int f, const CellS& L, const CellS& R, bool create,
                                     bool record) {
  FaceFlux o;
  o.WL = o.WR = 0.0;
  const int P = (L.ow == -1) ? L.ph : R.ph;
  const Phase& E = c_fluid.ph[P];
  double rl = L.r, ml = L.m, ul = L.u, fl1 = L.f1;
  double rr = R.r, mr = R.m, ur = R.u, fr1 = R.f1;
  // a needed face has a free cell on at least one side: a zone edge faces a free cell
  if (L.ow >= 0 && R.ow == -1) {  // a zone's last cell: its state at t^n
    const Zone& Z = d.zones[L.ow];
    rl = Z.eR0;
    ml = Z.eR1;
    ul = div_nr(ml, rl);
    fl1 = __fma_rn(ml, ul, pressure_fma(E, rl));
  }
  if (R.ow >= 0 && L.ow == -1) {
    const Zone& Z = d.zones[R.ow];
    rr = Z.eL0;
    mr = Z.eL1;
    ur = div_nr(mr, rr);
    fr1 = __fma_rn(mr, ur, pressure_fma(E, rr));
  }
  hll_pre(E.a, rl, ml, ul, fl1, rr, mr, ur, fr1, o.F0L, o.F1L);
  if (R.ow == -2) {  // right domain end: transmissive
    o.F0L = L.m;
    o.F1L = L.f1;
  }
  if (L.ow == -2) {  // left domain end: transmissive
    o.F0L = R.m;
    o.F1L = R.f1;
  }
  o.F0R = o.F0L;
  o.F1R = o.F1L;
  if (CREATION && create) {
    // fluxes of Eq. flux:cavitation / flux:nucleation with each boundary's own mass flux
    CreateOut Cr = creation_solve(c_fluid, c_opts, I.tau, P, rl, ml, rr, mr);
    if (record) atomicAdd((unsigned long long*)&I.stats[3], (unsigned long long)Cr.iters);
    if (!Cr.ok) {
      set_status(I, IMEXDS_ERR_PB_NOCONV);
      o.F0L = o.F1L = o.F0R = o.F1R = 0.0;
      return o;
    }
    o.F0L = -Cr.z1;
    o.F1L = -Cr.z1 * Cr.uC + Cr.pC;
    o.F0R = -Cr.z2;
    o.F1R = -Cr.z2 * Cr.uC + Cr.pC;
    o.WL = Cr.w1;
    o.WR = Cr.w2;
    if (record) {
      const double h = I.h, dt = I.dt;
      int k = atomicAdd(&I.n_ev, 1);
      if (k < EV_CAP) {
        Event& Ev = d.ev[ii * EV_CAP + k];
        Ev.face = f;
        Ev.w1 = Cr.w1;
        Ev.w2 = Cr.w2;
        Ev.rhoC = Cr.rhoC;
        Ev.mC = Cr.rhoC * Cr.uC;
        Ev.phC = 1 - P;
        Ev.hl = h + (Cr.w1 - 0.0) * dt;
        Ev.hr = h + (0.0 - Cr.w2) * dt;
      } else {
        set_status(I, IMEXDS_ERR_CAPACITY);
      }
    }
  }
  return o;
}

// One tile of TILE = 30 cells j0 .. j0+29; all 32 lanes of the calling warp take part. Lane l holds cell
// j0 - 1 + l: lane 0 the left neighbour of the tile, lanes 1..30 its cells, lane 31 its right neighbour. Lane
// l >= 1 computes the face on the left of its cell from its own state and lane l-1's, so lanes 1..31 give the
// tile's 31 faces and every cell and face is loaded or formed once per warp; lanes 1..30 update their cells
// (the neighbouring tiles form the same end faces from the same states: identical bits). Compared with 31-cell
// tiles whose lane 0 loaded the left neighbour a second time, this was measured 9 % faster (FP64 bound: one
// warp-wide FP64 instruction costs the same for 30 useful lanes as for 32). The common path is straight-line
// code. The tile's wave-speed maximum is folded into the instance's atomic maximum.
constexpr int TILE = 30;

template <bool CREATION>
__device__ void sweep_tile(const Dev& d, int ii, int j0) {
  const int lane = threadIdx.x & 31;
  Inst& I = d.inst[ii];
  const int N = I.N;
  const int j = j0 - 1 + lane;
  const CellS C = load_cell(d, I, j);
  const CellS Lc = shfl_up_cell(C);  // cell j - 1 (lane 0: its own cell, not used)
  int det_j = 0, det_jm1 = 0;
  if (CREATION) {
    // detection at face j (left of cell j); lane 0 examines face j0 - 1 for lane 1's left-neighbour rule
    CellS L0 = Lc;
    if (lane == 0) L0 = load_cell(d, I, j0 - 2);
    det_j = (j <= N) ? detect_face(L0, C) : 0;
    det_jm1 = __shfl_up_sync(0xffffffffu, det_j, 1);
  }
  // face j (left face of cell j): needed by cell j (updated by lanes 1..TILE) and by cell j-1 (lanes 2..31)
  const bool upd = (lane >= 1) && (lane <= TILE) && (C.ow == -1) && (j < N);
  const bool need = (lane >= 1) && (j <= N) && (((lane <= TILE) && (C.ow == -1)) || (lane >= 2 && Lc.ow == -1));
  // computed in every lane (unneeded lanes hold finite placeholder states); a creation event is recorded by
  // the lane that updates the cell right of the face (lane 31's face is the next tile's lane 1 face)
  const FaceFlux fj = face_flux<CREATION>(d, I, ii, j, Lc, C, CREATION && need && det_j && !det_jm1,
                                          lane >= 1 && lane <= TILE);
  // right face of cell j
  const double G0 = __shfl_down_sync(0xffffffffu, fj.F0L, 1);
  const double G1 = __shfl_down_sync(0xffffffffu, fj.F1L, 1);
  const double GW = CREATION ? __shfl_down_sync(0xffffffffu, fj.WL, 1) : 0.0;
  const double lam = I.lam;
  double r1 = __fma_rn(-lam, G0 - fj.F0R, C.r);
  double m1 = __fma_rn(-lam, G1 - fj.F1R, C.m);
  if (CREATION && upd && (nonzero_bits(GW) || nonzero_bits(fj.WR))) {
    const double h = I.h, dt = I.dt;
    const double hnp1 = h + (GW - fj.WR) * dt;
    r1 = (h * C.r - dt * (G0 - fj.F0R)) / hnp1;
    m1 = (h * C.m - dt * (G1 - fj.F1R)) / hnp1;
  }
  const double u1 = div_nr(m1, r1);
  unsigned long long sbits = 0ull;
  if (upd) {
    const int g = I.lat_off + j;
    const int nxt = I.parity ^ 1;
    d.R(nxt)[g] = r1;
    d.M(nxt)[g] = m1;
    d.U(nxt)[g] = u1;
    if (!pos_finite_bits(r1) || !finite_bits(m1)) set_status(I, IMEXDS_ERR_NONPHYSICAL);
    sbits = dbits(fabs(u1) + c_fluid.ph[C.ph].a);
  }
  // the warp maximum of non-negative doubles is the maximum of their bit patterns: high words first, then
  // the low words of the lanes holding the maximal high word (integer reductions, off the FP64 pipe; taking
  // the maximum of |u| per phase and adding the sound speed once per tile was measured 10 % slower)
  const unsigned hi = (unsigned)(sbits >> 32);
  const unsigned mhi = __reduce_max_sync(0xffffffffu, hi);
  const unsigned mlo = __reduce_max_sync(0xffffffffu, hi == mhi ? (unsigned)sbits : 0u);
  const unsigned long long wmax = ((unsigned long long)mhi << 32) | mlo;
  if (lane == 0 && wmax != 0ull) atomicMax(&I.smax_bits, wmax);
}

// Per-step sweep kernel: one warp per tile of the tile table.
template <bool CREATION>
__global__ void __launch_bounds__(256) k_sweep(Dev d, int n_tiles) {
  const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (t >= n_tiles) return;
  const int2 tile = d.tiles[t];
  const Inst& I = d.inst[tile.x];
  if (!I.active || I.status) return;
  sweep_tile<CREATION>(d, tile.x, tile.y);
}

// ------------------------------------------------------------------------------------------ k_dts
// Algorithm 2 on the blocks of one zone: dual time stepping (Eq. dual time tau diff) with local
// pseudo steps dtau_i = theta_i dt, theta_i = min(theta_nb, h_i^n/h), fluxes at the implicit faces from
// the App. A solver and width iterates h_i^{n,l+1} = h_i^n + (w_{i+1/2} - w_{i-1/2}) dt (Sec. 3.4); stop
// test of Sec. 4; Part 2 re-flux with F_left/F_right from U^n. Zone cells outside every block take the
// explicit update.
struct BlockCtx {
  double r[ZB], m[ZB], w[ZB];
  int ph[ZB];
  int fpb[ZB + 1];  // face q between local cells q-1 and q
};

__device__ inline bool block_fluxes(const BlockCtx& B, int lo, int hi, const double* Wr, const double* Wm,
                                    double FL0, double FL1, double FR0, double FR1, double tau, double dt,
                                    double* F0, double* F1, double* wc, double* hl, double* gl, double* gr,
                                    long long& newton, long long& solves, bool& nonconv) {
  F0[lo] = FL0;
  F1[lo] = FL1;
  F0[hi + 1] = FR0;
  F1[hi + 1] = FR1;
  wc[lo] = 0.0;
  wc[hi + 1] = 0.0;
  for (int g = lo + 1; g <= hi; ++g) {
    if (B.fpb[g]) {
      PBOut R = pb_solve_warm(c_fluid, c_opts, tau, B.ph[g - 1], Wr[g - 1], Wm[g - 1], B.ph[g], Wr[g], Wm[g], gl[g],
                              gr[g]);
      newton += R.iters;
      solves++;
      if (!R.ok) {
        nonconv = true;
        return false;
      }
      F0[g] = R.F0;
      F1[g] = R.F1;
      wc[g] = R.w;
    } else {
      hll_fast(c_fluid.ph[B.ph[g]], Wr[g - 1], Wm[g - 1], Wr[g], Wm[g], F0[g], F1[g]);
      wc[g] = 0.0;
    }
  }
  for (int i = lo; i <= hi; ++i) hl[i] = __fma_rn(wc[i + 1] - wc[i], dt, B.w[i]);
  for (int i = lo; i <= hi; ++i)
    if (!pos_finite_bits(hl[i])) return false;
  return true;
}

// General Algorithm 2 on every block of a zone (any block shape), kept out of line.
__device__ __noinline__ bool dts_general(const Dev& d, Zone& Z, Inst& I, int e0, int nq, const BlockCtx& B,
                                        const double* Fx0, const double* Fx1, double* out_r, double* out_m,
                                        double* out_w, double* xpb_new, int* moved, long long& newton,
                                        long long& solves, long long& iters_sum, long long& iters_max,
                                        long long& maxiter) {
  const double dt = I.dt, h = I.h, tau = I.tau;
  for (int b = 0; b < Z.nblk; ++b) {
    const int lo = Z.blo[b] - e0, hi = Z.bhi[b] - e0;
    const double FL0 = Fx0[lo], FL1 = Fx1[lo], FR0 = Fx0[hi + 1], FR1 = Fx1[hi + 1];
    double Wr[ZB], Wm[ZB], Nr[ZB], Nm[ZB], theta[ZB], F0[ZB + 1], F1[ZB + 1], wc[ZB + 1], hl[ZB];
    for (int q = 0; q < nq; ++q) {
      Wr[q] = B.r[q];
      Wm[q] = B.m[q];
    }
    // the Sec. 4 test of a component, |W^{l+1} - W^l| (1 + theta) / (theta dt max(|W^l|, 1)) (x dt in the
    // res dt mode) below tol, as |W^{l+1} - W^l| < lim max(|W^l|, 1), lim = tol theta dt' / (1 + theta)
    const double dtr = (c_opts.res_mode == 1) ? 1.0 : dt;
    double ith[ZB], lim[ZB];
    for (int q = lo; q <= hi; ++q) {
      int e = q + e0;
      double hp = (e < 0 || e >= Z.nc) ? h : Z.hp[e];
      theta[q] = fmin(c_opts.theta_nb, hp / h);
      ith[q] = 1.0 / (1.0 + theta[q]);
      lim[q] = (((Z.tiny_mask >> (q + e0 + 1)) & 1u) ? c_opts.tol_k : c_opts.tol_nb) * theta[q] * dtr * ith[q];
    }
    bool stop = false, nonconv = false;
    double gl[ZB + 1], gr[ZB + 1];  // Newton starts per face: the zone's last solution, then the previous iterate
    for (int g = 0; g <= nq; ++g) {
      int e = g + e0;
      bool zf = (e >= 1 && e <= Z.nc - 1);
      gl[g] = zf ? Z.pwl[e] : 0.0;
      gr[g] = zf ? Z.pwr[e] : 0.0;
    }
    int l;
    for (l = 0; l < c_opts.l_max && !stop; ++l) {
      if (!block_fluxes(B, lo, hi, Wr, Wm, FL0, FL1, FR0, FR1, tau, dt, F0, F1, wc, hl, gl, gr, newton, solves,
                        nonconv)) {
        set_status(I, nonconv ? IMEXDS_ERR_PB_NOCONV : IMEXDS_ERR_VANISH);
        return false;
      }
      stop = true;
      for (int q = lo; q <= hi; ++q) {
        const double th = theta[q], ih = rcp_nr(hl[q]);
        const double tr = __fma_rn(-dt, F0[q + 1] - F0[q], B.w[q] * B.r[q]) * ih;
        const double tm = __fma_rn(-dt, F1[q + 1] - F1[q], B.w[q] * B.m[q]) * ih;
        Nr[q] = __fma_rn(th, tr, Wr[q]) * ith[q];
        Nm[q] = __fma_rn(th, tm, Wm[q]) * ith[q];
        stop = stop && below_tol(Nr[q] - Wr[q], Wr[q], lim[q]) && below_tol(Nm[q] - Wm[q], Wm[q], lim[q]);
      }
      for (int q = lo; q <= hi; ++q) {
        Wr[q] = Nr[q];
        Wm[q] = Nm[q];
      }
    }
    if (!stop) maxiter++;
    iters_sum += l;
    iters_max = max(iters_max, (long long)l);
    if (!block_fluxes(B, lo, hi, Wr, Wm, FL0, FL1, FR0, FR1, tau, dt, F0, F1, wc, hl, gl, gr, newton, solves,
                      nonconv)) {
      set_status(I, nonconv ? IMEXDS_ERR_PB_NOCONV : IMEXDS_ERR_VANISH);
      return false;
    }
    for (int g = lo + 1; g <= hi; ++g)
      if (B.fpb[g]) {
        Z.pwl[g + e0] = gl[g];
        Z.pwr[g + e0] = gr[g];
      }
    for (int q = lo; q <= hi; ++q) {
      out_r[q] = (B.w[q] * B.r[q] - dt * (F0[q + 1] - F0[q])) / hl[q];
      out_m[q] = (B.w[q] * B.m[q] - dt * (F1[q + 1] - F1[q])) / hl[q];
      out_w[q] = hl[q];
    }
    for (int g = lo + 1; g <= hi; ++g)
      if (B.fpb[g]) {
        int e = g + e0;
        moved[g] = 1;
        xpb_new[g] = Z.fx[e] + wc[g] * dt;
      }
  }
  return true;
}

// Newton on every block of a zone of any shape (the system of newton_simple, any block size): fluxes at the
// iterate with the boundary faces' Jacobians (kept per face), the stop test, then the block-tridiagonal
// Jacobian assembled into band storage (HLL faces' Jacobians evaluated here) and solve_band. Kept out of line.
__device__ __noinline__ bool newton_general(const Dev& d, Zone& Z, Inst& I, int e0, int nq, const BlockCtx& B,
                                           const double* Fx0, const double* Fx1, double* out_r, double* out_m,
                                           double* out_w, double* xpb_new, int* moved, long long& newton,
                                           long long& solves, long long& iters_sum, long long& iters_max,
                                           long long& maxiter) {
  const double dt = I.dt, tau = I.tau;
  const double dtr = (c_opts.res_mode == 1) ? 1.0 : dt;
  for (int b = 0; b < Z.nblk; ++b) {
    const int lo = Z.blo[b] - e0, hi = Z.bhi[b] - e0;
    double Wr[ZB], Wm[ZB], F0[ZB + 1], F1[ZB + 1], wc[ZB + 1], hl[ZB], Tr[ZB], Tm[ZB], ih[ZB], dr[ZB], dm[ZB];
    FaceJac fj[ZB + 1];
    for (int q = 0; q < nq; ++q) {
      Wr[q] = B.r[q];
      Wm[q] = B.m[q];
    }
    double gl[ZB + 1], gr[ZB + 1];
    for (int g = 0; g <= nq; ++g) {
      int e = g + e0;
      bool zf = (e >= 1 && e <= Z.nc - 1);
      gl[g] = zf ? Z.pwl[e] : 0.0;
      gr[g] = zf ? Z.pwr[e] : 0.0;
    }
    // fluxes, face speeds and widths at (Wr, Wm); boundary faces' Jacobians into fj. 0 ok, 1 a boundary
    // solve failed, 2 a width would vanish
    auto fluxes = [&]() -> int {
      F0[lo] = Fx0[lo];
      F1[lo] = Fx1[lo];
      F0[hi + 1] = Fx0[hi + 1];
      F1[hi + 1] = Fx1[hi + 1];
      wc[lo] = 0.0;
      wc[hi + 1] = 0.0;
      for (int g = lo + 1; g <= hi; ++g) {
        if (B.fpb[g]) {
          PBOut R = pb_solve_core<true>(c_fluid, c_opts, tau, B.ph[g - 1], Wr[g - 1], Wm[g - 1], B.ph[g], Wr[g],
                                        Wm[g], gl[g], gr[g], &fj[g]);
          newton += R.iters;
          solves++;
          if (!R.ok) return 1;
          F0[g] = R.F0;
          F1[g] = R.F1;
          wc[g] = R.w;
        } else {
          hll_fast(c_fluid.ph[B.ph[g]], Wr[g - 1], Wm[g - 1], Wr[g], Wm[g], F0[g], F1[g]);
          wc[g] = 0.0;
        }
      }
      for (int q = lo; q <= hi; ++q) hl[q] = __fma_rn(wc[q + 1] - wc[q], dt, B.w[q]);
      for (int q = lo; q <= hi; ++q)
        if (!pos_finite_bits(hl[q])) return 2;
      return 0;
    };
    bool stop = false;
    int l, fail = 0;
    double corr_prev = INFINITY;
    for (l = 0; l < c_opts.l_max; ++l) {
      fail = fluxes();
      if (fail) break;
      stop = true;
      for (int q = lo; q <= hi; ++q) {
        ih[q] = rcp_nr(hl[q]);
        Tr[q] = __fma_rn(-dt, F0[q + 1] - F0[q], B.w[q] * B.r[q]) * ih[q];
        Tm[q] = __fma_rn(-dt, F1[q + 1] - F1[q], B.w[q] * B.m[q]) * ih[q];
        const double lim = (((Z.tiny_mask >> (q + e0 + 1)) & 1u) ? c_opts.tol_k : c_opts.tol_nb) * dtr;
        stop = stop && below_tol(Tr[q] - Wr[q], Wr[q], lim) && below_tol(Tm[q] - Wm[q], Wm[q], lim);
      }
      if (stop) break;
      for (int g = lo + 1; g <= hi; ++g)
        if (!B.fpb[g]) hll_jac(c_fluid.ph[B.ph[g]], Wr[g - 1], Wm[g - 1], Wr[g], Wm[g], fj[g]);
      if (!newton_block_step(hi - lo + 1, dt, ih + lo, Tr + lo, Tm + lo, Wr + lo, Wm + lo, fj + lo, dr, dm)) {
        fail = 3;
        break;
      }
      const double corr = newton_corr(hi - lo + 1, Wr + lo, Wm + lo, dr, dm);
      const bool at_floor = newton_at_floor(corr, corr_prev);
      corr_prev = corr;
      for (int q = lo; q <= hi; ++q) {
        Wr[q] += dr[q - lo];
        Wm[q] += dm[q - lo];
      }
      if (at_floor) {
        ++l;
        break;
      }
    }
    if (!fail && !stop) fail = fluxes();
    if (fail) {
      set_status(I, fail == 2 ? IMEXDS_ERR_VANISH : IMEXDS_ERR_PB_NOCONV);
      return false;
    }
    if (!stop) maxiter++;
    iters_sum += l;
    iters_max = max(iters_max, (long long)l);
    for (int g = lo + 1; g <= hi; ++g)
      if (B.fpb[g]) {
        Z.pwl[g + e0] = gl[g];
        Z.pwr[g + e0] = gr[g];
      }
    for (int q = lo; q <= hi; ++q) {
      out_r[q] = (B.w[q] * B.r[q] - dt * (F0[q + 1] - F0[q])) / hl[q];
      out_m[q] = (B.w[q] * B.m[q] - dt * (F1[q + 1] - F1[q])) / hl[q];
      out_w[q] = hl[q];
    }
    for (int g = lo + 1; g <= hi; ++g)
      if (B.fpb[g]) {
        int e = g + e0;
        moved[g] = 1;
        xpb_new[g] = Z.fx[e] + wc[g] * dt;
      }
  }
  return true;
}

// Register-resident Algorithm 2 for the most common zone: two cells with one phase boundary between
// them and one pulled lattice cell on the tiny side, i.e. a block of three cells whose boundary is at
// face PBF (2 when the pulled cell is on the left, 1 when it is on the right). Everything lives in
// registers; the stop test is evaluated without divisions:
//   res < tol  <=>  (1 + theta)|dW| < tol theta dt' max(|W|, 1),  dt' = dt (printed residual) or 1 (res dt).
template <int PBF>
__device__ void dts_simple(const Dev& d, int zi) {
  Zone& Z = d.zones[zi];
  Inst& I = d.inst[Z.inst];
  const int cur = I.parity;
  const double* lr = d.R(cur) + I.lat_off;
  const double* lm = d.M(cur) + I.lat_off;
  const unsigned char* lph = d.phase + I.lat_off;
  const double dt = I.dt, h = I.h, tau = I.tau;
  const int N = I.N;
  const int jp = (PBF == 2) ? Z.A - 1 : Z.B;  // the pulled lattice cell
  // cells q = 0, 1, 2 and their extended indices e = q - 1 (pulled left) or q (pulled right)
  double Ur[3], Um[3], Uw[3], hp[3];
  int ph[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int e = (PBF == 2) ? q - 1 : q;
    if (e < 0 || e > 1) {
      Ur[q] = lr[jp];
      Um[q] = lm[jp];
      Uw[q] = h;
      hp[q] = h;
      ph[q] = lph[jp];
    } else {
      Ur[q] = Z.r[e];
      Um[q] = Z.m[e];
      Uw[q] = Z.w[e];
      hp[q] = Z.hp[e];
      ph[q] = Z.ph[e];
    }
  }
  // F_left / F_right from U^n (the same function as the sweep: identical bits)
  double FL0, FL1, FR0, FR1;
  if (Z.oA > 0)
    hll_fast(c_fluid.ph[ph[0]], lr[Z.oA - 1], lm[Z.oA - 1], Ur[0], Um[0], FL0, FL1);
  else
    phys_flux_fast(c_fluid.ph[ph[0]], Ur[0], Um[0], FL0, FL1);
  if (Z.oB < N)
    hll_fast(c_fluid.ph[ph[2]], Ur[2], Um[2], lr[Z.oB], lm[Z.oB], FR0, FR1);
  else
    phys_flux_fast(c_fluid.ph[ph[2]], Ur[2], Um[2], FR0, FR1);
  const double dtr = (c_opts.res_mode == 1) ? 1.0 : dt;
  double th[3], ith[3], lim[3], hU0[3], hU1[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int e = (PBF == 2) ? q - 1 : q;
    th[q] = fmin(c_opts.theta_nb, hp[q] / h);
    ith[q] = 1.0 / (1.0 + th[q]);
    const bool tiny = (Z.tiny_mask >> (e + 1)) & 1u;
    lim[q] = (tiny ? c_opts.tol_k : c_opts.tol_nb) * th[q] * dtr * ith[q];
    hU0[q] = Uw[q] * Ur[q];
    hU1[q] = Uw[q] * Um[q];
  }
  constexpr int a = PBF - 1;               // boundary between cells a and a+1
  constexpr int b = (PBF == 1) ? 2 : 1;    // fixed interior face between cells b-1 and b
  const double ih_fixed = rcp_nr(Uw[PBF == 1 ? 2 : 0]);  // the cell away from the boundary keeps its width
  double gl = Z.pwl[1], gr = Z.pwr[1];
  double W0[3] = {Ur[0], Ur[1], Ur[2]}, W1[3] = {Um[0], Um[1], Um[2]};
  long long newton = 0, solves = 0;
  double Fp0 = 0.0, Fp1 = 0.0, wpb = 0.0, Fh0 = 0.0, Fh1 = 0.0;
  bool fail = false;
  auto fluxes = [&]() -> bool {
    // the fixed face first: its divisions overlap the boundary solve that follows
    hll_fast(c_fluid.ph[ph[b]], W0[b - 1], W1[b - 1], W0[b], W1[b], Fh0, Fh1);
    PBOut R = pb_solve_warm(c_fluid, c_opts, tau, ph[a], W0[a], W1[a], ph[a + 1], W0[a + 1], W1[a + 1], gl, gr);
    newton += R.iters;
    solves++;
    if (!R.ok) return false;
    Fp0 = R.F0;
    Fp1 = R.F1;
    wpb = R.w;
    return true;
  };
  // fluxes at faces 0..3 in order
  auto face = [&](int g, double& f0, double& f1) {
    if (g == 0) {
      f0 = FL0;
      f1 = FL1;
    } else if (g == 3) {
      f0 = FR0;
      f1 = FR1;
    } else if (g == PBF) {
      f0 = Fp0;
      f1 = Fp1;
    } else {
      f0 = Fh0;
      f1 = Fh1;
    }
  };
  bool stop = false;
  int l;
  for (l = 0; l < c_opts.l_max && !stop; ++l) {
    if (!fluxes()) {
      fail = true;
      break;
    }
    const double ha = __fma_rn(wpb - 0.0, dt, Uw[a]), hb = __fma_rn(0.0 - wpb, dt, Uw[a + 1]);
    if (!pos_finite_bits(ha) || !pos_finite_bits(hb)) {
      set_status(I, IMEXDS_ERR_VANISH);
      return;
    }
    const double iha = rcp_nr(ha), ihb = rcp_nr(hb);
    stop = true;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      double f0l, f1l, f0r, f1r;
      face(q, f0l, f1l);
      face(q + 1, f0r, f1r);
      const double ih = (q == a) ? iha : ((q == a + 1) ? ihb : ih_fixed);
      const double n0 = __fma_rn(th[q], __fma_rn(-dt, f0r - f0l, hU0[q]) * ih, W0[q]) * ith[q];
      const double n1 = __fma_rn(th[q], __fma_rn(-dt, f1r - f1l, hU1[q]) * ih, W1[q]) * ith[q];
      stop = stop && below_tol(n0 - W0[q], W0[q], lim[q]) && below_tol(n1 - W1[q], W1[q], lim[q]);
      W0[q] = n0;
      W1[q] = n1;
    }
  }
  if (fail || !fluxes()) {  // Part 2 needs the fluxes at U^{n,*}
    set_status(I, IMEXDS_ERR_PB_NOCONV);
    return;
  }
  const double ha = __fma_rn(wpb - 0.0, dt, Uw[a]), hb = __fma_rn(0.0 - wpb, dt, Uw[a + 1]);
  if (!pos_finite_bits(ha) || !pos_finite_bits(hb)) {
    set_status(I, IMEXDS_ERR_VANISH);
    return;
  }
  double* nr = d.R(cur ^ 1) + I.lat_off;
  double* nm = d.M(cur ^ 1) + I.lat_off;
  double* nu = d.U(cur ^ 1) + I.lat_off;
  double smax = 0.0;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    double f0l, f1l, f0r, f1r;
    face(q, f0l, f1l);
    face(q + 1, f0r, f1r);
    const double hn1 = (q == a) ? ha : ((q == a + 1) ? hb : Uw[q]);
    const double r1 = (hU0[q] - dt * (f0r - f0l)) / hn1;
    const double m1 = (hU1[q] - dt * (f1r - f1l)) / hn1;
    if (!(r1 > 0.0) || !isfinite(r1) || !isfinite(m1)) set_status(I, IMEXDS_ERR_NONPHYSICAL);
    const double u1 = div_nr(m1, r1);
    smax = fmax(smax, fabs(u1) + c_fluid.ph[ph[q]].a);
    const int e = (PBF == 2) ? q - 1 : q;
    if (e < 0 || e > 1) {
      nr[jp] = r1;
      nm[jp] = m1;
      nu[jp] = u1;
    } else {
      Z.r[e] = r1;
      Z.m[e] = m1;
      Z.w[e] = hn1;
    }
  }
  Z.pwl[1] = gl;
  Z.pwr[1] = gr;
  Z.fx[1] = Z.fx[1] + wpb * dt;
  if (smax > 0.0) atomicMax(&I.smax_bits, dbits(smax));
  atomicAdd((unsigned long long*)&I.stats[1], (unsigned long long)l);
  atomicMax((unsigned long long*)&I.stats[2], (unsigned long long)l);
  atomicAdd((unsigned long long*)&I.stats[3], (unsigned long long)newton);
  if (!stop) atomicAdd((unsigned long long*)&I.stats[7], 1ull);
  atomicAdd((unsigned long long*)&I.stats[8], (unsigned long long)solves);
}

// Newton's method on the implicit system of a block instead of dual time stepping (the paper's outlook, Sec. 5;
// Sec. 3.3 notes that dual time is one way to solve that system). The system is R(W) = W - T(W) = 0, T the
// update of Algorithm 2 Part 1 (Eq. godunov_meth:nonunif) with fluxes and widths at W; its root is the
// dual-time limit. The Sec. 4 residual of an iterate W is |W - T(W)| / (dt max(|W|, 1)) component by
// component (a pseudo step moves W by theta (T(W) - W) / (1 + theta)), so the same test stops Newton:
//   stop  <=>  |T(W) - W| < tol dt' max(|W|, 1)  for every block cell (tol_k for tiny cells, tol_nb else),
// dt' = dt (printed residual) or 1 (res dt). Each iteration: fluxes at W (the boundary solve also gives the
// face Jacobian by the implicit function theorem, HLL faces theirs in closed form), T(W), the stop test, then
// dR/dW = I - dT/dW assembled from the face Jacobians,
//   dT_i/dW = -(dt / h_i) [(dF_{i+1/2} - dF_{i-1/2}) + T_i (dw_{i+1/2} - dw_{i-1/2})],
// and one linear solve with partial pivoting. The iteration count reported is the number of Newton steps.

// The common zone of dts_simple (three cells, the boundary at face PBF): a 6 x 6 system in registers.
template <int PBF>
__device__ __noinline__ void newton_simple(const Dev& d, int zi) {
  Zone& Z = d.zones[zi];
  Inst& I = d.inst[Z.inst];
  const int cur = I.parity;
  const double* lr = d.R(cur) + I.lat_off;
  const double* lm = d.M(cur) + I.lat_off;
  const unsigned char* lph = d.phase + I.lat_off;
  const double dt = I.dt, h = I.h, tau = I.tau;
  const int N = I.N;
  const int jp = (PBF == 2) ? Z.A - 1 : Z.B;  // the pulled lattice cell
  double Ur[3], Um[3], Uw[3];
  int ph[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int e = (PBF == 2) ? q - 1 : q;
    if (e < 0 || e > 1) {
      Ur[q] = lr[jp];
      Um[q] = lm[jp];
      Uw[q] = h;
      ph[q] = lph[jp];
    } else {
      Ur[q] = Z.r[e];
      Um[q] = Z.m[e];
      Uw[q] = Z.w[e];
      ph[q] = Z.ph[e];
    }
  }
  double FL0, FL1, FR0, FR1;
  if (Z.oA > 0)
    hll_fast(c_fluid.ph[ph[0]], lr[Z.oA - 1], lm[Z.oA - 1], Ur[0], Um[0], FL0, FL1);
  else
    phys_flux_fast(c_fluid.ph[ph[0]], Ur[0], Um[0], FL0, FL1);
  if (Z.oB < N)
    hll_fast(c_fluid.ph[ph[2]], Ur[2], Um[2], lr[Z.oB], lm[Z.oB], FR0, FR1);
  else
    phys_flux_fast(c_fluid.ph[ph[2]], Ur[2], Um[2], FR0, FR1);
  const double dtr = (c_opts.res_mode == 1) ? 1.0 : dt;
  double lim[3], hU0[3], hU1[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int e = (PBF == 2) ? q - 1 : q;
    const bool tiny = (Z.tiny_mask >> (e + 1)) & 1u;
    lim[q] = (tiny ? c_opts.tol_k : c_opts.tol_nb) * dtr;
    hU0[q] = Uw[q] * Ur[q];
    hU1[q] = Uw[q] * Um[q];
  }
  constexpr int a = PBF - 1;             // boundary between cells a and a+1
  constexpr int b = (PBF == 1) ? 2 : 1;  // fixed interior face between cells b-1 and b
  double gl = Z.pwl[1], gr = Z.pwr[1];
  double W0[3] = {Ur[0], Ur[1], Ur[2]}, W1[3] = {Um[0], Um[1], Um[2]};
  long long newton = 0, solves = 0;
  double Fp0 = 0.0, Fp1 = 0.0, wpb = 0.0, Fh0 = 0.0, Fh1 = 0.0;
  FaceJac Jp;
  auto face = [&](int g, double& f0, double& f1) {
    if (g == 0) {
      f0 = FL0;
      f1 = FL1;
    } else if (g == 3) {
      f0 = FR0;
      f1 = FR1;
    } else if (g == PBF) {
      f0 = Fp0;
      f1 = Fp1;
    } else {
      f0 = Fh0;
      f1 = Fh1;
    }
  };
  // fluxes at W and the boundary's face Jacobian; widths of the two boundary cells
  double ha = 0.0, hb = 0.0;
  auto fluxes = [&]() -> int {  // 0 ok, 1 boundary solve failed, 2 a width would vanish
    hll_fast(c_fluid.ph[ph[b]], W0[b - 1], W1[b - 1], W0[b], W1[b], Fh0, Fh1);
    PBOut R = pb_solve_core<true>(c_fluid, c_opts, tau, ph[a], W0[a], W1[a], ph[a + 1], W0[a + 1], W1[a + 1], gl,
                                  gr, &Jp);
    newton += R.iters;
    solves++;
    if (!R.ok) return 1;
    Fp0 = R.F0;
    Fp1 = R.F1;
    wpb = R.w;
    ha = __fma_rn(wpb - 0.0, dt, Uw[a]);
    hb = __fma_rn(0.0 - wpb, dt, Uw[a + 1]);
    if (!pos_finite_bits(ha) || !pos_finite_bits(hb)) return 2;
    return 0;
  };
  bool stop = false;
  int l, fail = 0;
  double T0[3], T1[3], ih[3];
  double corr_prev = INFINITY;
  for (l = 0; l < c_opts.l_max; ++l) {
    fail = fluxes();
    if (fail) break;
    ih[a] = rcp_nr(ha);
    ih[a + 1] = rcp_nr(hb);
    ih[(PBF == 1) ? 2 : 0] = rcp_nr(Uw[(PBF == 1) ? 2 : 0]);
    stop = true;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      double f0l, f1l, f0r, f1r;
      face(q, f0l, f1l);
      face(q + 1, f0r, f1r);
      T0[q] = __fma_rn(-dt, f0r - f0l, hU0[q]) * ih[q];
      T1[q] = __fma_rn(-dt, f1r - f1l, hU1[q]) * ih[q];
      stop = stop && below_tol(T0[q] - W0[q], W0[q], lim[q]) && below_tol(T1[q] - W1[q], W1[q], lim[q]);
    }
    if (stop) break;
    // Newton step: (I - dT/dW) d = T - W
    FaceJac fjs[3];
    fjs[PBF] = Jp;
    hll_jac(c_fluid.ph[ph[b]], W0[b - 1], W1[b - 1], W0[b], W1[b], fjs[b]);
    double d0[3], d1[3];
    if (!newton_block_step(3, dt, ih, T0, T1, W0, W1, fjs, d0, d1)) {
      fail = 3;
      break;
    }
    const double corr = newton_corr(3, W0, W1, d0, d1);
    const bool at_floor = newton_at_floor(corr, corr_prev);
    corr_prev = corr;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      W0[q] += d0[q];
      W1[q] += d1[q];
    }
    if (at_floor) {
      ++l;
      break;
    }
  }
  // Part 2 needs the fluxes at U^{n,*}: those of the last evaluation when the test stopped the iteration,
  // else evaluated at the last iterate
  if (!fail && !stop) fail = fluxes();
  if (fail) {
    set_status(I, fail == 2 ? IMEXDS_ERR_VANISH : IMEXDS_ERR_PB_NOCONV);
    return;
  }
  double* nr = d.R(cur ^ 1) + I.lat_off;
  double* nm = d.M(cur ^ 1) + I.lat_off;
  double* nu = d.U(cur ^ 1) + I.lat_off;
  double smax = 0.0;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    double f0l, f1l, f0r, f1r;
    face(q, f0l, f1l);
    face(q + 1, f0r, f1r);
    const double hn1 = (q == a) ? ha : ((q == a + 1) ? hb : Uw[q]);
    const double r1 = (hU0[q] - dt * (f0r - f0l)) / hn1;
    const double m1 = (hU1[q] - dt * (f1r - f1l)) / hn1;
    if (!(r1 > 0.0) || !isfinite(r1) || !isfinite(m1)) set_status(I, IMEXDS_ERR_NONPHYSICAL);
    const double u1 = div_nr(m1, r1);
    smax = fmax(smax, fabs(u1) + c_fluid.ph[ph[q]].a);
    const int e = (PBF == 2) ? q - 1 : q;
    if (e < 0 || e > 1) {
      nr[jp] = r1;
      nm[jp] = m1;
      nu[jp] = u1;
    } else {
      Z.r[e] = r1;
      Z.m[e] = m1;
      Z.w[e] = hn1;
    }
  }
  Z.pwl[1] = gl;
  Z.pwr[1] = gr;
  Z.fx[1] = Z.fx[1] + wpb * dt;
  if (smax > 0.0) atomicMax(&I.smax_bits, dbits(smax));
  atomicAdd((unsigned long long*)&I.stats[1], (unsigned long long)l);
  atomicMax((unsigned long long*)&I.stats[2], (unsigned long long)l);
  atomicAdd((unsigned long long*)&I.stats[3], (unsigned long long)newton);
  if (!stop) atomicAdd((unsigned long long*)&I.stats[7], 1ull);
  atomicAdd((unsigned long long*)&I.stats[8], (unsigned long long)solves);
}

template <bool NEWTON>
__device__ __noinline__ void dts_zone_general(const Dev& d, int zi);

// NEWTON: the kernel was launched for options.block_solver = 1 (Newton on each block); a template parameter so
// that the dual-time kernels carry none of the Newton code.
template <bool NEWTON>
__device__ void dts_zone(const Dev& d, int zi) {
  Zone& Z = d.zones[zi];
  if (!Z.alive) return;
  const Inst& I = d.inst[Z.inst];
  if (!I.active || I.status) return;
  if (Z.nc == 2 && Z.fpb[1] && Z.nblk == 1 && (Z.pullL + Z.pullR) == 1) {
    if (NEWTON) {
      if (Z.pullL)
        newton_simple<2>(d, zi);
      else
        newton_simple<1>(d, zi);
    } else {
      if (Z.pullL)
        dts_simple<2>(d, zi);
      else
        dts_simple<1>(d, zi);
    }
    return;
  }
  dts_zone_general<NEWTON>(d, zi);
}

// Algorithm 2 for any zone shape (blocks of any size, zone cells outside the blocks), kept out of line.
template <bool NEWTON>
__device__ __noinline__ void dts_zone_general(const Dev& d, int zi) {
  Zone& Z = d.zones[zi];
  Inst& I = d.inst[Z.inst];
  const int cur = I.parity;
  const double* lr = d.R(cur) + I.lat_off;
  const double* lm = d.M(cur) + I.lat_off;
  double* nr = d.R(cur ^ 1) + I.lat_off;
  double* nm = d.M(cur ^ 1) + I.lat_off;
  const unsigned char* lph = d.phase + I.lat_off;
  const double dt = I.dt, h = I.h;
  const int N = I.N;
  BlockCtx B;
  const int e0 = -Z.pullL;              // first extended index
  const int nq = Z.nc + Z.pullL + Z.pullR;
  // local cells q = e - e0
  for (int q = 0; q < nq; ++q) {
    int e = q + e0;
    if (e < 0) {
      B.r[q] = lr[Z.A - 1];
      B.m[q] = lm[Z.A - 1];
      B.w[q] = h;
      B.ph[q] = lph[Z.A - 1];
    } else if (e >= Z.nc) {
      B.r[q] = lr[Z.B];
      B.m[q] = lm[Z.B];
      B.w[q] = h;
      B.ph[q] = lph[Z.B];
    } else {
      B.r[q] = Z.r[e];
      B.m[q] = Z.m[e];
      B.w[q] = Z.w[e];
      B.ph[q] = Z.ph[e];
    }
  }
  for (int q = 0; q <= nq; ++q) {
    int e = q + e0;  // face between extended cells e-1 and e
    B.fpb[q] = (e >= 1 && e <= Z.nc - 1) ? Z.fpb[e] : 0;
  }
  // explicit fluxes at U^n on every face that is not a phase boundary (block outer faces and the faces
  // of zone cells outside the blocks)
  double Fx0[ZB + 1], Fx1[ZB + 1];
  for (int q = 0; q <= nq; ++q) {
    if (B.fpb[q]) {
      Fx0[q] = Fx1[q] = 0.0;
      continue;
    }
    if (q == 0) {
      if (Z.oA > 0)
        hll_fast(c_fluid.ph[B.ph[0]], lr[Z.oA - 1], lm[Z.oA - 1], B.r[0], B.m[0], Fx0[q], Fx1[q]);
      else
        phys_flux_fast(c_fluid.ph[B.ph[0]], B.r[0], B.m[0], Fx0[q], Fx1[q]);
    } else if (q == nq) {
      if (Z.oB < N)
        hll_fast(c_fluid.ph[B.ph[nq - 1]], B.r[nq - 1], B.m[nq - 1], lr[Z.oB], lm[Z.oB], Fx0[q], Fx1[q]);
      else
        phys_flux_fast(c_fluid.ph[B.ph[nq - 1]], B.r[nq - 1], B.m[nq - 1], Fx0[q], Fx1[q]);
    } else {
      hll_fast(c_fluid.ph[B.ph[q]], B.r[q - 1], B.m[q - 1], B.r[q], B.m[q], Fx0[q], Fx1[q]);
    }
  }
  int inblk[ZB];
  for (int q = 0; q < nq; ++q) inblk[q] = 0;
  for (int b = 0; b < Z.nblk; ++b)
    for (int q = Z.blo[b] - e0; q <= Z.bhi[b] - e0; ++q) inblk[q] = 1;
  long long newton = 0, solves = 0, iters_sum = 0, iters_max = 0, maxiter = 0;
  // Phase creation (App. B) at the zone's own faces between two explicit cells of one phase: the interior
  // faces of a zone joined from two boundary neighbourhoods (the lattice sweep examines the faces between
  // free lattice cells; a zone's first and last cells are boundary cells and lie in blocks). Detection by the
  // no-transition star pressure at U^n; a face whose left neighbour face is also detected is not used. The
  // cell left of a creation face sees the flux with the left boundary's mass flux and a face moving with w1,
  // the cell right of it the right boundary's and w2 (Eq. flux:cavitation / flux:nucleation); the created
  // cell is inserted into the zone after the step's update.
  bool cre[ZB + 1];
  double cF0L[ZB + 1], cF1L[ZB + 1], cF0R[ZB + 1], cF1R[ZB + 1], cW1[ZB + 1], cW2[ZB + 1], cRho[ZB + 1], cM[ZB + 1];
  int n_cre = 0;
  for (int q = 0; q <= nq; ++q) cre[q] = false;
  if (c_opts.creation) {
    bool det_prev = false;
    for (int q = 1; q < nq; ++q) {
      bool det = false;
      if (!B.fpb[q] && !inblk[q - 1] && !inblk[q])
        det = creation_detect(c_fluid, B.ph[q], B.r[q - 1], div_nr(B.m[q - 1], B.r[q - 1]), B.r[q],
                              div_nr(B.m[q], B.r[q]));
      if (det && !det_prev) {
        CreateOut Cr = creation_solve(c_fluid, c_opts, I.tau, B.ph[q], B.r[q - 1], B.m[q - 1], B.r[q], B.m[q]);
        newton += Cr.iters;
        if (!Cr.ok) {
          set_status(I, IMEXDS_ERR_PB_NOCONV);
          return;
        }
        cre[q] = true;
        cF0L[q] = -Cr.z1;
        cF1L[q] = -Cr.z1 * Cr.uC + Cr.pC;
        cF0R[q] = -Cr.z2;
        cF1R[q] = -Cr.z2 * Cr.uC + Cr.pC;
        cW1[q] = Cr.w1;
        cW2[q] = Cr.w2;
        cRho[q] = Cr.rhoC;
        cM[q] = Cr.rhoC * Cr.uC;
        n_cre++;
      }
      det_prev = det;
    }
  }
  double out_r[ZB], out_m[ZB], out_w[ZB];
  for (int q = 0; q < nq; ++q) {
    out_w[q] = B.w[q];
    if (inblk[q]) continue;
    // fluxes seen at the left / right face and the face speeds (non-zero at a creation face only)
    const double fl0 = cre[q] ? cF0R[q] : Fx0[q], fl1 = cre[q] ? cF1R[q] : Fx1[q];
    const double fr0 = cre[q + 1] ? cF0L[q + 1] : Fx0[q + 1], fr1 = cre[q + 1] ? cF1L[q + 1] : Fx1[q + 1];
    const double wl = cre[q] ? cW2[q] : 0.0, wr = cre[q + 1] ? cW1[q + 1] : 0.0;
    double hnp1 = B.w[q] + (wr - wl) * dt;
    out_r[q] = (B.w[q] * B.r[q] - dt * (fr0 - fl0)) / hnp1;
    out_m[q] = (B.w[q] * B.m[q] - dt * (fr1 - fl1)) / hnp1;
    out_w[q] = hnp1;
  }
  double xpb_new[ZB + 1];
  int moved[ZB + 1];
  for (int q = 0; q <= nq; ++q) moved[q] = 0;
  const bool ok = NEWTON
                      ? newton_general(d, Z, I, e0, nq, B, Fx0, Fx1, out_r, out_m, out_w, xpb_new, moved, newton,
                                       solves, iters_sum, iters_max, maxiter)
                      : dts_general(d, Z, I, e0, nq, B, Fx0, Fx1, out_r, out_m, out_w, xpb_new, moved, newton, solves,
                                    iters_sum, iters_max, maxiter);
  if (!ok) return;
  double smax = 0.0;
  double* nu = d.U(cur ^ 1) + I.lat_off;
  for (int q = 0; q < nq; ++q) {
    int e = q + e0;
    double r1 = out_r[q], m1 = out_m[q];
    if (!(r1 > 0.0) || !isfinite(r1) || !isfinite(m1) || !(out_w[q] > 0.0)) set_status(I, IMEXDS_ERR_NONPHYSICAL);
    const double u1 = div_nr(m1, r1);
    smax = fmax(smax, fabs(u1) + c_fluid.ph[B.ph[q]].a);
    if (e < 0) {
      nr[Z.A - 1] = r1;
      nm[Z.A - 1] = m1;
      nu[Z.A - 1] = u1;
    } else if (e >= Z.nc) {
      nr[Z.B] = r1;
      nm[Z.B] = m1;
      nu[Z.B] = u1;
    } else {
      Z.r[e] = r1;
      Z.m[e] = m1;
      Z.w[e] = out_w[q];
    }
  }
  for (int q = 1; q < nq; ++q)
    if (moved[q]) Z.fx[q + e0] = xpb_new[q];
  if (n_cre) {
    // insert the created cells, right to left so that the indices of the faces still to visit hold
    for (int q = nq - 1; q >= 1; --q) {
      if (!cre[q]) continue;
      const int e = q + e0;  // zone face between zone cells e-1 and e (both explicit, hence zone cells)
      const double xf = I.xL + (double)Z.fj[e] * h;
      if (!zone_insert_cell(Z, e)) {
        set_status(I, IMEXDS_ERR_CAPACITY);
        return;
      }
      Z.w[e] = (cW2[q] - cW1[q]) * dt;
      Z.r[e] = cRho[q];
      Z.m[e] = cM[q];
      Z.ph[e] = 1 - B.ph[q];
      Z.fpb[e] = 1;
      Z.fx[e] = xf + cW1[q] * dt;
      Z.fpb[e + 1] = 1;
      Z.fx[e + 1] = xf + cW2[q] * dt;
      Z.pwl[e] = Z.pwr[e] = Z.pwl[e + 1] = Z.pwr[e + 1] = 0.0;
      smax = fmax(smax, fabs(cM[q] / cRho[q]) + c_fluid.ph[1 - B.ph[q]].a);
    }
    Z.changed = 1;
    atomicAdd((unsigned long long*)&I.stats[6], (unsigned long long)n_cre);
  }
  if (smax > 0.0) atomicMax(&I.smax_bits, dbits(smax));
  atomicAdd((unsigned long long*)&I.stats[1], (unsigned long long)iters_sum);
  atomicMax((unsigned long long*)&I.stats[2], (unsigned long long)iters_max);
  atomicAdd((unsigned long long*)&I.stats[3], (unsigned long long)newton);
  atomicAdd((unsigned long long*)&I.stats[7], (unsigned long long)maxiter);
  atomicAdd((unsigned long long*)&I.stats[8], (unsigned long long)solves);
}

// ------------------------------------------------------------------------------------------ k_post
// Grid management after the step (Sec. 2.3, 3.4) and phase creation (App. B), one thread per instance:
// split boundary cells wider than split_ratio*h (keeping fixed faces on the lattice), return regular
// cells at the zone ends to the lattice, turn creation events into zones, join zones closer than
// ZONE_GAP, then advance t and set the next dt from the wave-speed maximum.

// Grid management after the step (Sec. 2.3, 3.4), the part of one zone: its owned lattice range is returned,
// boundary cells wider than split_ratio*h are split (fixed faces stay on the lattice), regular cells at its ends
// return to the lattice. A zone whose footprint changed in this step or that holds an interior run of ZONE_GAP
// regular lattice cells goes on its instance's work list for post_inst. Touches only this zone and the lattice
// cells it owns, so the zones of an instance can run in parallel (k_post_zones).
__device__ inline bool zone_interior_run(const Zone& Z, double h, int& a_out, int& b_out) {
  int a = -1, b = -1;
  for (int k = 1; k < Z.nc - 1 && b < 0; ++k) {
    bool reg = !Z.fpb[k] && !Z.fpb[k + 1] && Z.fj[k + 1] == Z.fj[k] + 1 && Z.w[k] == h;
    if (reg) {
      if (a < 0) a = k;
      if (k + 1 - a >= ZONE_GAP) {
        int e = k + 1;  // extend to the end of the run
        while (e < Z.nc - 1 && !Z.fpb[e] && !Z.fpb[e + 1] && Z.fj[e + 1] == Z.fj[e] + 1 && Z.w[e] == h) ++e;
        b = e;
      }
    } else {
      a = -1;
    }
  }
  a_out = a;
  b_out = b;
  return b >= 0;
}

__device__ __noinline__ void post_zone(const Dev& d, int zs) {
  Zone& Z = d.zones[zs];
  if (!Z.alive) return;
  Inst& I = d.inst[Z.inst];
  if (!I.active) return;
  int* own = d.own + I.lat_off;
  for (int j = Z.oA; j < Z.oB; ++j) own[j] = -1;
  Z.oA = Z.oB = 0;
  if (I.status) {
    if (Z.changed) d.work[I.zone_off + atomicAdd(&I.n_work, 1)] = zs;
    return;
  }
  const double h = I.h;
  const int nxt = I.parity ^ 1;
  double* nr = d.R(nxt) + I.lat_off;
  double* nm = d.M(nxt) + I.lat_off;
  double* nu = d.U(nxt) + I.lat_off;
  unsigned char* lph = d.phase + I.lat_off;
  long long splits = 0;
  // splits
  {
    for (int i = 0; i < Z.nc; ++i) {
      bool lpb = Z.fpb[i], rpb = Z.fpb[i + 1];
      if (!(lpb || rpb) || !(Z.w[i] > c_opts.split_ratio * h)) continue;
      double w1, w2;
      int jc;
      if (!lpb) {
        jc = Z.fj[i] + 1;
        w1 = h;
        w2 = Z.w[i] - h;
      } else if (!rpb) {
        jc = Z.fj[i + 1] - 1;
        w2 = h;
        w1 = Z.w[i] - h;
      } else {
        double xm = 0.5 * (Z.fx[i] + Z.fx[i + 1]);
        jc = (int)llround((xm - I.xL) / h);
        w1 = (I.xL + (double)jc * h) - Z.fx[i];
        w2 = Z.w[i] - w1;
        if (!(w1 > 0.0) || !(w2 > 0.0)) continue;
      }
      if (!zone_insert_cell(Z, i + 1)) {
        set_status(I, IMEXDS_ERR_CAPACITY);
        break;
      }
      // insert_cell shifted faces >= i+1 up; the new face i+1 is the split face
      Z.fpb[i + 1] = 0;
      Z.fj[i + 1] = jc;
      Z.fx[i + 1] = 0.0;
      Z.w[i] = w1;
      Z.w[i + 1] = w2;
      Z.r[i + 1] = Z.r[i];
      Z.m[i + 1] = Z.m[i];
      Z.ph[i + 1] = Z.ph[i];
      splits++;
      ++i;
    }
  }
  // release regular cells at the zone ends back to the lattice (a pure change of representation)
  {
    while (Z.nc > 1 && !Z.fpb[1] && Z.fj[1] == Z.A + 1 && Z.w[0] == h) {
      nr[Z.A] = Z.r[0];
      nm[Z.A] = Z.m[0];
      nu[Z.A] = div_nr(Z.m[0], Z.r[0]);
      lph[Z.A] = (unsigned char)Z.ph[0];
      zone_erase_cell(Z, 0);
      Z.A += 1;
      Z.fj[0] = Z.A;
      Z.fpb[0] = 0;
      Z.changed = 1;
    }
    while (Z.nc > 1 && !Z.fpb[Z.nc - 1] && Z.fj[Z.nc - 1] == Z.B - 1 && Z.w[Z.nc - 1] == h) {
      nr[Z.B - 1] = Z.r[Z.nc - 1];
      nm[Z.B - 1] = Z.m[Z.nc - 1];
      nu[Z.B - 1] = div_nr(Z.m[Z.nc - 1], Z.r[Z.nc - 1]);
      lph[Z.B - 1] = (unsigned char)Z.ph[Z.nc - 1];
      Z.nc--;
      Z.B -= 1;
      Z.fj[Z.nc] = Z.B;
      Z.fpb[Z.nc] = 0;
      Z.changed = 1;
    }
  }
  if (splits) atomicAdd((unsigned long long*)&I.stats[5], (unsigned long long)splits);
  int ra, rb;
  if (Z.changed || zone_interior_run(Z, h, ra, rb)) d.work[I.zone_off + atomicAdd(&I.n_work, 1)] = zs;
}

// Grid management after the step, the part of an instance (one thread), after post_zone has run for every
// zone of the instance: zones split at an interior run of ZONE_GAP regular lattice cells, creation events turned
// into zones, zones closer than ZONE_GAP lattice cells joined (only zones on the work list changed their
// footprint, so only they are checked against their neighbours), then t += dt and the next dt from the
// wave-speed maximum.
__device__ __noinline__ void post_inst(const Dev& d, int ii) {
  Inst& I = d.inst[ii];
  if (!I.active) return;
  const double h = I.h;
  const int nxt = I.parity ^ 1;
  double* nr = d.R(nxt) + I.lat_off;
  double* nm = d.M(nxt) + I.lat_off;
  double* nu = d.U(nxt) + I.lat_off;
  unsigned char* lph = d.phase + I.lat_off;
  Zone* zones = d.zones + I.zone_off;
  int* work = d.work + I.zone_off;  // global zone slots
  int nw = I.n_work;
  I.n_work = 0;
  if (I.status) {
    for (int w = 0; w < nw; ++w) d.zones[work[w]].changed = 0;
    I.active = 0;
    I.n_ev = 0;
    return;
  }
  // the work list in slot order (post_zone appends in any order)
  for (int w = 1; w < nw; ++w) {
    const int v = work[w];
    int x = w - 1;
    while (x >= 0 && work[x] > v) {
      work[x + 1] = work[x];
      --x;
    }
    work[x + 1] = v;
  }
  long long creations = 0;
  // split a zone at an interior run of at least ZONE_GAP regular lattice cells (returned to the lattice);
  // the part right of the run becomes a new zone (a pure change of representation)
  for (int w = 0; w < nw; ++w) {
    Zone& Z = d.zones[work[w]];
    if (!Z.alive) continue;
    int a, b;
    if (!zone_interior_run(Z, h, a, b)) continue;
    int slot = -1;
    for (int y = 0; y < I.zone_cap; ++y)
      if (!zones[y].alive) {
        slot = y;
        break;
      }
    if (slot < 0) {
      set_status(I, IMEXDS_ERR_CAPACITY);
      break;
    }
    Zone& Zn = zones[slot];
    Zn.alive = 1;
    Zn.inst = ii;
    Zn.merge_mask = 0;
    Zn.oA = Zn.oB = 0;
    Zn.nc = Z.nc - b;
    for (int i = 0; i < Zn.nc; ++i) {
      Zn.w[i] = Z.w[b + i];
      Zn.r[i] = Z.r[b + i];
      Zn.m[i] = Z.m[b + i];
      Zn.ph[i] = Z.ph[b + i];
    }
    for (int k = 0; k <= Zn.nc; ++k) {
      Zn.fpb[k] = Z.fpb[b + k];
      Zn.fj[k] = Z.fj[b + k];
      Zn.fx[k] = Z.fx[b + k];
      Zn.pwl[k] = Z.pwl[b + k];
      Zn.pwr[k] = Z.pwr[b + k];
    }
    Zn.A = Z.fj[b];
    Zn.B = Z.B;
    for (int k = a; k < b; ++k) {
      int j = Z.fj[k];
      nr[j] = Z.r[k];
      nm[j] = Z.m[k];
      nu[j] = div_nr(Z.m[k], Z.r[k]);
      lph[j] = (unsigned char)Z.ph[k];
    }
    Z.nc = a;
    Z.B = Z.fj[a];
    Z.changed = 1;
    Zn.changed = 1;
    work[nw++] = I.zone_off + slot;
  }
  double smax = __longlong_as_double((long long)I.smax_bits);
  // creation events -> new zones
  int nev = min(I.n_ev, EV_CAP);
  for (int k = 0; k < nev; ++k) {
    const Event& E = d.ev[ii * EV_CAP + k];
    int slot = -1;
    for (int z = 0; z < I.zone_cap; ++z)
      if (!zones[z].alive) {
        slot = z;
        break;
      }
    if (slot < 0) {
      set_status(I, IMEXDS_ERR_CAPACITY);
      break;
    }
    Zone& Z = zones[slot];
    int f = E.face;
    double xf = I.xL + (double)f * h;
    Z.alive = 1;
    Z.inst = ii;
    Z.A = f - 1;
    Z.B = f + 1;
    Z.nc = 3;
    Z.ph[0] = lph[f - 1];
    Z.ph[1] = E.phC;
    Z.ph[2] = lph[f];
    Z.w[0] = E.hl;
    Z.w[1] = (E.w2 - E.w1) * I.dt;
    Z.w[2] = E.hr;
    Z.r[0] = nr[f - 1];
    Z.m[0] = nm[f - 1];
    Z.r[1] = E.rhoC;
    Z.m[1] = E.mC;
    Z.r[2] = nr[f];
    Z.m[2] = nm[f];
    Z.fpb[0] = 0;
    Z.fj[0] = f - 1;
    Z.fpb[1] = 1;
    Z.fx[1] = xf + E.w1 * I.dt;
    Z.fpb[2] = 1;
    Z.fx[2] = xf + E.w2 * I.dt;
    Z.fpb[3] = 0;
    Z.fj[3] = f + 1;
    Z.oA = Z.oB = 0;
    Z.merge_mask = 0;
    for (int k = 0; k <= ZC; ++k) Z.pwl[k] = Z.pwr[k] = 0.0;
    Z.changed = 1;
    smax = fmax(smax, fabs(E.mC / E.rhoC) + c_fluid.ph[E.phC].a);
    work[nw++] = I.zone_off + slot;
    creations++;
  }
  I.n_ev = 0;
  // join zones closer than ZONE_GAP lattice cells; only zones whose footprint changed in this step are
  // checked against their neighbours (O(changed x zones))
  for (bool again = true; again;) {
    again = false;
    for (int w = 0; w < nw && !again; ++w) {
      const int a = work[w] - I.zone_off;
      if (!zones[a].alive || !zones[a].changed) continue;
      // nearest zone to the left (largest B <= A_a) and to the right (smallest A >= B_a)
      int left = -1, right = -1;
      for (int b = 0; b < I.zone_cap; ++b) {
        if (b == a || !zones[b].alive) continue;
        if (zones[b].A >= zones[a].B) {
          if (right < 0 || zones[b].A < zones[right].A) right = b;
        } else if (zones[b].B <= zones[a].A) {
          if (left < 0 || zones[b].B > zones[left].B) left = b;
        }
      }
      for (int pk = 0; pk < 2 && !again; ++pk) {
        const int ia = (pk == 0) ? left : a, ib = (pk == 0) ? a : right;  // the pairs (left, a) and (a, right)
        if (ia < 0 || ib < 0) continue;
        Zone& Za = zones[ia];
        Zone& Zb = zones[ib];
        int gap = Zb.A - Za.B;
        if (gap >= ZONE_GAP) continue;
        if (Za.nc + gap + Zb.nc > ZC) {
          set_status(I, IMEXDS_ERR_CAPACITY);
          break;
        }
        for (int j = Za.B; j < Zb.A; ++j) {  // absorb the regular lattice cells in between
          int i = Za.nc;
          Za.w[i] = h;
          Za.r[i] = nr[j];
          Za.m[i] = nm[j];
          Za.ph[i] = lph[j];
          Za.fpb[i] = 0;
          Za.fj[i] = j;
          Za.pwl[i] = Za.pwr[i] = 0.0;
          Za.nc++;
        }
        for (int i = 0; i < Zb.nc; ++i) {
          int k = Za.nc;
          Za.w[k] = Zb.w[i];
          Za.r[k] = Zb.r[i];
          Za.m[k] = Zb.m[i];
          Za.ph[k] = Zb.ph[i];
          Za.fpb[k] = Zb.fpb[i];
          Za.fj[k] = Zb.fj[i];
          Za.fx[k] = Zb.fx[i];
          Za.pwl[k] = Zb.pwl[i];
          Za.pwr[k] = Zb.pwr[i];
          Za.nc++;
        }
        Za.fpb[Za.nc] = 0;
        Za.fj[Za.nc] = Zb.B;
        Za.B = Zb.B;
        Zb.alive = 0;
        if (!Za.changed) work[nw++] = I.zone_off + ia;  // a zone that changes only now joins the list
        Za.changed = 1;
        again = true;
      }
    }
  }
  for (int w = 0; w < nw; ++w) d.zones[work[w]].changed = 0;
  if (creations) I.stats[6] += creations;
  // time and next step
  const Ctrl& C = *d.ctrl;
  I.t = I.clipped ? C.t_end : I.t + I.dt;
  I.stats[0] += 1;
  I.parity = nxt;
  I.smax_bits = 0ull;
  if (I.status) {
    I.active = 0;
    return;
  }
  double dtn = c_opts.cfl * h / smax;
  I.clipped = 0;
  if (C.clip) {
    if (!(I.t < C.t_end)) {
      I.active = 0;
      return;
    }
    if (C.t_end - I.t <= dtn) {
      dtn = C.t_end - I.t;
      I.clipped = 1;
    }
  }
  I.dt = dtn;
  I.lam = dtn / h;
}

// ---------------------------------------------------------------------------------- step kernels
__device__ inline bool zone_active(const Dev& d, int zi) {
  const Zone& Z = d.zones[zi];
  if (!Z.alive) return false;
  const Inst& I = d.inst[Z.inst];
  return I.active && !I.status;
}

__global__ void k_pre(Dev d, int n) {
  int zi = blockIdx.x * blockDim.x + threadIdx.x;
  if (zi < n) {
    d.zones[zi].merge_mask = 0;
    if (zone_active(d, zi)) pre_zone(d, zi);
  }
}
__global__ void k_plan(Dev d, int n) {
  int zi = blockIdx.x * blockDim.x + threadIdx.x;
  if (zi < n && zone_active(d, zi)) plan_zone(d, zi);
}
template <bool NEWTON>
__global__ void k_dts(Dev d, int n) {
  int zi = blockIdx.x * blockDim.x + threadIdx.x;
  if (zi < n && zone_active(d, zi)) dts_zone<NEWTON>(d, zi);
}
__global__ void k_post_zones(Dev d, int n) {
  int zi = blockIdx.x * blockDim.x + threadIdx.x;
  if (zi < n) post_zone(d, zi);
}
__global__ void k_post(Dev d, int n) {
  int ii = blockIdx.x * blockDim.x + threadIdx.x;
  if (ii < n && d.inst[ii].active) post_inst(d, ii);
}

// the whole grid management of one instance by one thread (the group kernels' warp 0)
__device__ inline void post_all(const Dev& d, int ii) {
  const Inst& I = d.inst[ii];
  for (int z = I.zone_off; z < I.zone_off + I.zone_cap; ++z) post_zone(d, z);
  post_inst(d, ii);
}

// Group-resident schedule: one CTA advances a group of instances (similar sizes) step after step
// without any grid-wide synchronisation. Warp 0 runs the per-instance work (lane i: instance i of the
// group: boundary solves, plan, dual time stepping, grid management); warps 1.. sweep the group's
// lattice cells while warp 0 runs the dual-time chains of the same step.
constexpr int GROUP_MAX = 32;
// NT: the CTA width the kernel is compiled for (128: two CTAs per SM, three sweep warps; 256: one CTA per SM,
// seven sweep warps); launched with at most NT threads.
template <bool CREATION, int NT, bool NEWTON>
__global__ void __launch_bounds__(NT, (NT <= 128 ? 2 : 1)) k_group(Dev d, const int* ginst, const int2* grange, int max_steps,
                                               long long* phase_cycles) {
  const int2 gr = grange[blockIdx.x];
  // SM clock cycles per phase (timing mode; the layout of imexds_get_group_phase_cycles): 0 boundary solves +
  // plan, 1 sweep (first sweep warp), 2 dual time (warp 0), 3 grid management, 4 the concurrent phase
  // (barrier to barrier: the longer of 1 and 2), 5 the whole launch. Phases 0, 3 and 4 are intervals between
  // the block's barriers read by thread 0, so 0 + 4 + 3 = 5 up to the loop's own instructions; 1 and 2 are
  // read after __syncwarp (every lane of the warp done) and lie within 4.
  long long cyc[6] = {0, 0, 0, 0, 0, 0};
  const long long c_start = clock64();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
  const int ii = (lane < gr.y) ? ginst[gr.x + lane] : -1;
  __shared__ int s_more;
  for (int step = 0; step < max_steps; ++step) {
    long long c0 = clock64();
    if (warp == 0 && ii >= 0) {
      Inst& I = d.inst[ii];
      if (I.active && !I.status) {
        for (int z = I.zone_off; z < I.zone_off + I.zone_cap; ++z) {
          d.zones[z].merge_mask = 0;
          if (d.zones[z].alive) pre_zone(d, z);
        }
        for (int z = I.zone_off; z < I.zone_off + I.zone_cap; ++z)
          if (d.zones[z].alive && !I.status) plan_zone(d, z);
      }
    }
    __syncthreads();
    long long c1 = clock64();
    if (warp == 0) {
      if (ii >= 0) {
        Inst& I = d.inst[ii];
        if (I.active && !I.status)
          for (int z = I.zone_off; z < I.zone_off + I.zone_cap; ++z)
            if (d.zones[z].alive && !I.status) dts_zone<NEWTON>(d, z);
      }
      __syncwarp();
      cyc[2] += clock64() - c1;
    } else {
      // the tiles of all active instances of the group, dealt to warps 1..nw-1
      int t = warp - 1, base = 0;
      for (int k = 0; k < gr.y; ++k) {
        const int ik = ginst[gr.x + k];
        const Inst& I = d.inst[ik];
        const int nt = (I.active && !I.status) ? (I.N + TILE - 1) / TILE : 0;
        for (; t < base + nt; t += nw - 1) sweep_tile<CREATION>(d, ik, (t - base) * TILE);
        base += nt;
      }
      __syncwarp();
      cyc[1] += clock64() - c1;
    }
    __syncthreads();
    long long c2 = clock64();
    cyc[0] += c1 - c0;
    cyc[4] += c2 - c1;
    if (warp == 0 && ii >= 0 && d.inst[ii].active) post_all(d, ii);
    if (threadIdx.x == 0) s_more = 0;
    __syncthreads();
    if (warp == 0 && ii >= 0 && d.inst[ii].active && !d.inst[ii].status) atomicOr(&s_more, 1);
    __syncthreads();
    cyc[3] += clock64() - c2;
    if (!s_more) break;
  }
  cyc[5] = clock64() - c_start;
  if (phase_cycles && lane == 0 && warp <= 1) {
    long long* pc = phase_cycles + 6 * blockIdx.x;
    if (warp == 0) {
      pc[0] += cyc[0];
      pc[2] += cyc[2];
      pc[3] += cyc[3];
      pc[4] += cyc[4];
      pc[5] += cyc[5];
    } else {
      pc[1] += cyc[1];
    }
  }
}

// Instance groups without a per-step barrier. Lane k of warp 0 runs instance k's serial work at its own
// pace; the other warps sweep the tiles of whichever instance has planned its step. Per instance,
// shared counters order the work of one step n:
//   lane k: boundary solves + merges + blocks (n) -> open the sweep of step n -> Algorithm 2 (n)
//           -> wait until every tile of step n is swept -> grid management (n) -> step n + 1
//   sweep warps: take a tile ticket of any open instance, sweep the tile, count it done.
// The tickets of step n + 1 are issued only after step n + 1 is planned (its counters are reset then), so a
// ticket taken late always belongs to a planned step. Every wait is bounded by the SM clock: an instance
// whose sweep does not complete within kWaitCycles stops with IMEXDS_ERR_TIMEOUT; an idle sweep warp leaves
// after kWaitCycles. The per-instance work and its order are those of k_group: the results are the same.
constexpr long long kWaitCycles = 40000000000LL;  // ~20 s at 2 GHz

template <bool CREATION, bool NEWTON>
__global__ void __launch_bounds__(128, 2) k_group_async(Dev d, const int* ginst, const int2* grange, int max_steps,
                                                     long long* phase_cycles) {
  const int2 gr = grange[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ int s_open[32], s_next[32], s_done[32], s_ntiles[32];
  __shared__ int s_alive;
  if (threadIdx.x < 32) {
    s_open[threadIdx.x] = 0;
    s_next[threadIdx.x] = 0;
    s_done[threadIdx.x] = 0;
    s_ntiles[threadIdx.x] = 0;
  }
  if (threadIdx.x == 0) s_alive = 0;
  __syncthreads();
  const int ii = (warp == 0 && lane < gr.y) ? ginst[gr.x + lane] : -1;
  bool live = false;
  if (ii >= 0) {
    const Inst& I = d.inst[ii];
    live = I.active && !I.status;
    if (live) atomicAdd(&s_alive, 1);
  }
  __syncthreads();
  volatile int* v_open = s_open;
  volatile int* v_done = s_done;
  volatile int* v_alive = &s_alive;
  if (warp == 0) {
    if (!live) return;
    Inst& I = d.inst[ii];
    const int nt = (I.N + TILE - 1) / TILE;
    long long cp = 0, cd = 0, cw = 0, cq = 0;
    for (int step = 0; step < max_steps; ++step) {
      long long c0 = clock64();
      for (int z = I.zone_off; z < I.zone_off + I.zone_cap; ++z) {
        d.zones[z].merge_mask = 0;
        if (d.zones[z].alive) pre_zone(d, z);
      }
      for (int z = I.zone_off; z < I.zone_off + I.zone_cap; ++z)
        if (d.zones[z].alive && !I.status) plan_zone(d, z);
      // open the sweep of this step: counters first, then the flag
      s_done[lane] = 0;
      __threadfence_block();
      s_next[lane] = 0;
      s_ntiles[lane] = (I.status) ? 0 : nt;
      __threadfence_block();
      v_open[lane] = 1;
      long long c1 = clock64();
      if (!I.status)
        for (int z = I.zone_off; z < I.zone_off + I.zone_cap; ++z)
          if (d.zones[z].alive && !I.status) dts_zone<NEWTON>(d, z);
      long long c2 = clock64();
      bool timeout = false;
      const int need = ((volatile int*)s_ntiles)[lane];  // every ticket issued for this step is swept first
      while (v_done[lane] < need) {
        __nanosleep(64);
        if (clock64() - c2 > kWaitCycles) {
          timeout = true;
          break;
        }
      }
      v_open[lane] = 0;
      __threadfence_block();
      long long c3 = clock64();
      if (timeout) {
        set_status(I, IMEXDS_ERR_TIMEOUT);
        break;
      }
      post_all(d, ii);
      long long c4 = clock64();
      cp += c1 - c0;
      cd += c2 - c1;
      cw += c3 - c2;
      cq += c4 - c3;
      if (!I.active || I.status) break;
    }
    v_open[lane] = 0;
    __threadfence_block();
    atomicSub(&s_alive, 1);
    if (phase_cycles) {
      // the slowest lane of the group: its boundary solves + plan, dual time, dual time plus the wait for the
      // sweep, grid management, and its whole run
      unsigned long long* pc = (unsigned long long*)(phase_cycles + 6 * blockIdx.x);
      atomicMax(&pc[0], (unsigned long long)cp);
      atomicMax(&pc[2], (unsigned long long)cd);
      atomicMax(&pc[3], (unsigned long long)cq);
      atomicMax(&pc[4], (unsigned long long)(cd + cw));
      atomicMax(&pc[5], (unsigned long long)(cp + cd + cw + cq));
    }
    return;
  }
  // sweep warps: lane 0 reads the shared state and takes the ticket, the warp follows its decision
  // (sweep_tile needs all 32 lanes)
  long long busy = 0, idle0 = clock64();
  int k = (gr.y > 0) ? (warp - 1) % gr.y : 0;
  for (;;) {
    int alive = 0, kk = -1, t = 0;
    if (lane == 0) {
      alive = *v_alive;
      for (int q = 0; alive > 0 && q < gr.y; ++q) {
        const int c = (k + q) % gr.y;
        if (!v_open[c]) continue;
        const int tt = atomicAdd(&s_next[c], 1);
        if (tt < ((volatile int*)s_ntiles)[c]) {
          kk = c;
          t = tt;
          break;
        }
      }
      __threadfence_block();  // the step's plan (written before its tickets were issued) is read after this
    }
    alive = __shfl_sync(0xffffffffu, alive, 0);
    kk = __shfl_sync(0xffffffffu, kk, 0);
    t = __shfl_sync(0xffffffffu, t, 0);
    __syncwarp();
    if (alive <= 0) break;
    if (kk >= 0) {
      long long b0 = clock64();
      sweep_tile<CREATION>(d, ginst[gr.x + kk], t * TILE);
      __threadfence_block();
      __syncwarp();
      if (lane == 0) atomicAdd(&s_done[kk], 1);
      busy += clock64() - b0;
      k = kk;
      idle0 = clock64();
    } else {
      __nanosleep(128);
      if (clock64() - idle0 > kWaitCycles) break;
    }
  }
  if (phase_cycles && lane == 0) atomicMax((unsigned long long*)&phase_cycles[6 * blockIdx.x + 1], (unsigned long long)busy);
}

// u = m / rho of every lattice cell, with the quotient the kernels use (set_states)
__global__ void k_init_u(const double* rho, const double* m, double* u, int n) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < n) u[g] = div_nr(m[g], rho[g]);
}

// Wave-speed maximum over all cells of every instance and the first dt (before the first step).
__global__ void k_init_dt(Dev d, int n_inst) {
  int ii = blockIdx.x;
  if (ii >= n_inst) return;
  Inst& I = d.inst[ii];
  if (I.status) {
    if (threadIdx.x == 0) I.active = 0;
    return;
  }
  const int cur = I.parity;
  const double* lr = d.R(cur) + I.lat_off;
  const double* lm = d.M(cur) + I.lat_off;
  const unsigned char* lph = d.phase + I.lat_off;
  const int* own = d.own + I.lat_off;
  double s = 0.0;
  for (int j = threadIdx.x; j < I.N; j += blockDim.x)
    if (own[j] < 0) s = fmax(s, fabs(lm[j] / lr[j]) + c_fluid.ph[lph[j]].a);
  for (int z = threadIdx.x; z < I.zone_cap; z += blockDim.x) {
    const Zone& Z = d.zones[I.zone_off + z];
    if (!Z.alive) continue;
    for (int i = 0; i < Z.nc; ++i) s = fmax(s, fabs(Z.m[i] / Z.r[i]) + c_fluid.ph[Z.ph[i]].a);
  }
  __shared__ double red[32];
  for (int off = 16; off > 0; off >>= 1) s = fmax(s, __shfl_down_sync(0xffffffffu, s, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double S = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) S = fmax(S, red[w]);
    const Ctrl& C = *d.ctrl;
    double dt = c_opts.cfl * I.h / S;
    I.clipped = 0;
    I.active = 1;
    if (C.clip) {
      if (!(I.t < C.t_end)) {
        I.active = 0;
      } else if (C.t_end - I.t <= dt) {
        dt = C.t_end - I.t;
        I.clipped = 1;
      }
    }
    I.dt = dt;
    I.lam = dt / I.h;
    I.smax_bits = 0ull;
  }
}

// ---------------------------------------------------------------------- cell lists on the device
// The current cell lists of every instance in the order of imexds_get_states (lattice cells outside zones
// and the zones' cells, left to right) written into device arrays, without staging through the host.

// Cells of every instance: its lattice cells plus, per alive zone, the zone's cells minus the lattice cells
// the zone covers.
__global__ void k_cell_counts(Dev d, int n_inst, int* counts) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_inst) return;
  const Inst& I = d.inst[i];
  int cnt = I.N;
  for (int z = 0; z < I.zone_cap; ++z) {
    const Zone& Z = d.zones[I.zone_off + z];
    if (Z.alive) cnt += Z.nc - (Z.B - Z.A);
  }
  counts[i] = cnt;
}

// One thread per zone slot: at the zone's first lattice cell, the number of cells it adds to the list
// (delta) and its slot + 1 (zstart); cov marks every lattice cell the zone covers. The three arrays are
// zero before the call.
__global__ void k_zone_marks(Dev d, int n_slots, int* delta, int* zstart, unsigned char* cov) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= n_slots) return;
  const Zone& Z = d.zones[z];
  if (!Z.alive) return;
  const int o = d.inst[Z.inst].lat_off;
  delta[o + Z.A] = Z.nc - (Z.B - Z.A);
  zstart[o + Z.A] = z + 1;
  for (int j = Z.A; j < Z.B; ++j) cov[o + j] = 1;
}

// One CTA (256 threads) per instance, its lattice in chunks of 256 cells: an exclusive block scan of delta
// gives the cells the zones add before each lattice cell; a cell outside every zone goes to
// off + j + extra(j), the cells of a zone starting at j to off + j + extra(j) + q.
__global__ void __launch_bounds__(256) k_gather_states(Dev d, const int* off, double* w, double* r, double* m,
                                                       unsigned char* ph, const int* delta, const int* zstart,
                                                       const unsigned char* cov) {
  const int i = blockIdx.x;
  const Inst& I = d.inst[i];
  const int lo = I.lat_off, N = I.N, p = I.parity, o0 = off[i];
  const double* R = d.R(p);
  const double* M = d.M(p);
  __shared__ int wsum[8];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int base = 0; base < N; base += 256) {
    const int j = base + threadIdx.x;
    const int v = (j < N) ? delta[lo + j] : 0;
    int x = v;  // inclusive warp scan
#pragma unroll
    for (int k = 1; k < 32; k <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, k);
      if (lane >= k) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    int before = carry;
    for (int k = 0; k < wid; ++k) before += wsum[k];
    const int extra = before + x - v;  // exclusive
    if (j < N) {
      const int g = lo + j;
      const int at = o0 + j + extra;
      if (!cov[g]) {
        w[at] = I.h;
        r[at] = R[g];
        m[at] = M[g];
        ph[at] = d.phase[g];
      } else if (zstart[g]) {
        const Zone& Z = d.zones[zstart[g] - 1];
        for (int q = 0; q < Z.nc; ++q) {
          w[at + q] = Z.w[q];
          r[at + q] = Z.r[q];
          m[at + q] = Z.m[q];
          ph[at + q] = (unsigned char)Z.ph[q];
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 255) carry = before + x;
    __syncthreads();
  }
}

// t and status of every instance, packed for one small copy.
__global__ void k_inst_ts(Dev d, int n_inst, double* t, int* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_inst) return;
  t[i] = d.inst[i].t;
  status[i] = d.inst[i].status;
}

__global__ void k_count_active(Dev d, int n_inst) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  int c = 0;
  for (int i = threadIdx.x; i < n_inst; i += blockDim.x) c += (d.inst[i].active && !d.inst[i].status) ? 1 : 0;
  atomicAdd(&cnt, c);
  __syncthreads();
  if (threadIdx.x == 0) d.ctrl->n_active = cnt;
}

}  // namespace
#include "noalloc.cuh"
#include "adjoint.cuh"
namespace {

// ---- the adjoint's seeds and gradients in device arrays (imexds_adjoint_device)
// Seeds in imexds_get_states order (offsets toff) into the adjoint's per-instance slots; one CTA per instance.
__global__ void k_scatter_seeds(const long long* offs, const int* toff, const double* sw, const double* sr,
                                const double* sm, double* lw, double* lr, double* lm) {
  const int i = blockIdx.x;
  const long long o = offs[i];
  const int a = toff[i], M = toff[i + 1] - a;
  for (int q = threadIdx.x; q < M; q += blockDim.x) {
    lw[o + q] = sw ? sw[a + q] : 0.0;
    lr[o + q] = sr[a + q];
    lm[o + q] = sm[a + q];
  }
}

// Largest deviation of the replayed final states (fin_*) from the forward run's (g*, imexds_get_states order):
// rho and m relative to max |rho|, widths relative to h; one CTA (128 threads) per instance.
__global__ void k_replay_err(const imexds::adj::AInst* I, const long long* offs, const int* toff, const double* fw,
                             const double* fr, const double* fm, const double* gw, const double* gr,
                             const double* gm, double* err) {
  const int i = blockIdx.x;
  const long long o = offs[i];
  const int a = toff[i], M = toff[i + 1] - a;
  double rmax = 0.0, dr = 0.0, dm = 0.0, dw = 0.0;
  for (int q = threadIdx.x; q < M; q += blockDim.x) {
    rmax = fmax(rmax, fabs(gr[a + q]));
    dr = fmax(dr, fabs(fr[o + q] - gr[a + q]));
    dm = fmax(dm, fabs(fm[o + q] - gm[a + q]));
    dw = fmax(dw, fabs(fw[o + q] - gw[a + q]));
  }
  __shared__ double red[4][4];
  for (int off = 16; off > 0; off >>= 1) {
    rmax = fmax(rmax, __shfl_down_sync(0xffffffffu, rmax, off));
    dr = fmax(dr, __shfl_down_sync(0xffffffffu, dr, off));
    dm = fmax(dm, __shfl_down_sync(0xffffffffu, dm, off));
    dw = fmax(dw, __shfl_down_sync(0xffffffffu, dw, off));
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[w][0] = rmax;
    red[w][1] = dr;
    red[w][2] = dm;
    red[w][3] = dw;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k)
      for (int c = 0; c < 4; ++c) red[0][c] = fmax(red[0][c], red[k][c]);
    const double R = red[0][0];
    err[i] = fmax(red[0][1] / R, fmax(red[0][2] / R, red[0][3] / I[i].h));
  }
}

// Gradients with respect to the initial lists into the caller's device arrays (imexds_set_states order,
// offsets u0off), one thread per instance: a boundary position is the last fixed face plus the widths after
// it, so its adjoint adds to the widths of those cells; cells with two fixed faces have the lattice width
// (gradient 0); an instance without gradient gets NaN.
__global__ void k_adj_grads(int n, const imexds::adj::AInst* I, const long long* offs, const int* u0off,
                            const unsigned char* fpb0, const double* lw, const double* lr, const double* lm,
                            const double* lx, double* gw0, double* gr0, double* gm0, double* gtau) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const imexds::adj::AInst& A = I[i];
  const int a = u0off[i], M0 = u0off[i + 1] - a;
  const long long o = offs[i];
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  gtau[i] = A.status ? nan : A.lam_tau;
  double acc = 0.0;  // adjoint of the boundary positions right of the cell, within its segment
  for (int q = M0 - 1; q >= 0; --q) {
    if (!fpb0[o + q + 1]) acc = 0.0;
    if (fpb0[o + q + 1]) acc += lx[o + q + 1];
    gr0[a + q] = A.status ? nan : lr[o + q];
    gm0[a + q] = A.status ? nan : lm[o + q];
    if (gw0) {
      const bool lattice = !fpb0[o + q] && !fpb0[o + q + 1];
      gw0[a + q] = A.status ? nan : (lattice ? 0.0 : lw[o + q] + acc);
    }
  }
}

// ---------------------------------------------------------------------------------------- host side
std::string g_last_error;

}  // namespace

struct imexds_ctx {
  int n_inst = 0;
  std::vector<int> N;
  std::vector<double> xL, xR, tau;
  Fluid fluid;
  Opts opts;
  int zone_cap_opt = 0;
  cudaStream_t stream = nullptr;
  Dev d{};
  int n_lat = 0, n_zone_slots = 0, n_tiles = 0;
  std::vector<int> lat_off, zone_off, zone_cap;
  bool loaded = false;
  int* h_active = nullptr;  // pinned
  long long launches = 0;
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  cudaStream_t side = nullptr;            // second stream of the step graph (k_dts beside k_sweep)
  int schedule = 0;                       // 1 per-step kernels, 2 instance groups (0 auto at set_states)
  int schedule_opt = 0, group_cells = 16384, use_groups = 0, group_threads = 128, async_groups = 0;
  bool group_cells_set = false;  // group_cells given by the caller (otherwise sized to fill the SMs)
  int n_groups = 0;
  long long* d_phase = nullptr;  // per-group phase cycles (timing mode)
  int* d_ginst = nullptr;
  int2* d_grange = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  // device copy of the state loaded by the last set_states (imexds_reset)
  Dev saved{};
  // optional per-kernel timing with events captured in the step graph
  int timing = 0;
  std::vector<cudaEvent_t> tev;  // 6 events per step of the graph
  double kt_ms[6] = {0, 0, 0, 0, 0, 0};
  long long kt_n[6] = {0, 0, 0, 0, 0, 0};
  cudaEvent_t gev[2] = {nullptr, nullptr};
  // the initial cell lists of the last imexds_set_states and the calls made since (the adjoint replays them)
  std::vector<int> u0_off;
  std::vector<double> u0_w, u0_r, u0_m;
  std::vector<uint8_t> u0_ph;
  double u0_t = 0.0;
  std::vector<int> prog_k;
  std::vector<double> prog_a;
  // adjoint buffers (kept between calls, grown on demand)
  int adj_k = 64;
  size_t adj_bytes = 0;
  void* adj_mem = nullptr;
  double adj_ms = 0.0, adj_replay_err = 0.0;
  std::vector<int32_t> adj_fin_off, adj_site;
  std::vector<double> adj_fin_w, adj_fin_r, adj_fin_m;
  long long adj_cell_steps = 0;
  // device scratch of the cell-list gather (imexds_cell_counts, imexds_get_states_device, imexds_adjoint_device)
  int *g_delta = nullptr, *g_zstart = nullptr, *g_counts = nullptr, *g_off = nullptr, *g_st = nullptr;
  unsigned char* g_cov = nullptr;
  double* g_t = nullptr;
  // device staging of the packed cell lists of imexds_get_states (w, rho, m then phase), grown on demand
  void* g_pack = nullptr;
  size_t g_pack_cells = 0;
};

namespace {

imexds_status cuda_fail(cudaError_t e) {
  g_last_error = cudaGetErrorString(e);
  return IMEXDS_ERR_CUDA;
}
#define CK(x)                                   \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_); \
  } while (0)

// Table of the table-driven logarithm: 128/j and ln(j/128) as a double plus remainder (long double).
LogTable make_log_table() {
  LogTable T;
  for (int t = 0; t < kLogJN; ++t) {
    int j = kLogJ0 + t;
    long double c = (long double)j / 128.0L;
    long double l = logl(c);
    T.c[t] = (double)j / 128.0;
    T.inv_c[t] = (double)(128.0L / (long double)j);
    T.lnc_hi[t] = (double)l;
    T.lnc_lo[t] = (double)(l - (long double)T.lnc_hi[t]);
  }
  return T;
}

__global__ void k_check_log(int n, const double* x, double* fast, double* ref) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    fast[i] = fast_log(x[i]);
    ref[i] = log(x[i]);
  }
}

Phase make_phase(const imexds_eos& e, double p_sat) {
  Phase P;
  P.kind = e.kind;
  P.a2 = e.a2;
  P.a = std::sqrt(e.a2);
  P.p0 = e.p0;
  P.rho0 = e.rho0;
  P.rho_sat = (e.kind == 0) ? p_sat / e.a2 : e.rho0 + (p_sat - e.p0) / e.a2;
  P.ia2 = 1.0 / e.a2;
  P.ia = 1.0 / P.a;
  P.ln_rho_sat = std::log(P.rho_sat);
  P.irho_sat = 1.0 / P.rho_sat;
  return P;
}

// The arrays that depend on the instance groups (rebuilt at every imexds_set_states), the timing counters and
// the step graph.
void free_groups(imexds_ctx* c) {
  cudaFree(c->d_ginst);
  cudaFree(c->d_grange);
  cudaFree(c->d_phase);
  c->d_ginst = nullptr;
  c->d_grange = nullptr;
  c->d_phase = nullptr;
  if (c->graph) cudaGraphExecDestroy(c->graph);
  c->graph = nullptr;
  for (auto e : c->tev) cudaEventDestroy(e);
  c->tev.clear();
}

void free_dev(imexds_ctx* c) {
  free_groups(c);
  Dev& d = c->d;
  for (int k = 0; k < 2; ++k) {
    cudaFree(d.rho[k]);
    cudaFree(d.m[k]);
    cudaFree(d.u[k]);
  }
  cudaFree(d.phase);
  cudaFree(d.own);
  cudaFree(d.zones);
  cudaFree(d.inst);
  cudaFree(d.ev);
  cudaFree(d.tiles);
  cudaFree(d.work);
  cudaFree(d.ctrl);
  cudaFree(c->g_delta);
  cudaFree(c->g_zstart);
  cudaFree(c->g_cov);
  cudaFree(c->g_counts);
  cudaFree(c->g_off);
  cudaFree(c->g_t);
  cudaFree(c->g_st);
  c->g_delta = c->g_zstart = c->g_counts = c->g_off = c->g_st = nullptr;
  c->g_cov = nullptr;
  c->g_t = nullptr;
  cudaFree(c->g_pack);
  c->g_pack = nullptr;
  c->g_pack_cells = 0;
  d = Dev{};
  Dev& sv = c->saved;
  for (int k = 0; k < 2; ++k) {
    cudaFree(sv.rho[k]);
    cudaFree(sv.m[k]);
    cudaFree(sv.u[k]);
  }
  cudaFree(sv.phase);
  cudaFree(sv.zones);
  cudaFree(sv.inst);
  sv = Dev{};
}

// one time step: five kernel launches on the context stream
// The step as a fork/join: k_sweep and k_dts only read U^n and write disjoint cells, so k_dts runs on a
// second stream beside k_sweep (used while capturing the step graph).
void launch_step_forked(imexds_ctx* c) {
  const int zt = 64;
  int zb = (c->n_zone_slots + zt - 1) / zt;
  int ib = (c->n_inst + zt - 1) / zt;
  k_pre<<<zb, zt, 0, c->stream>>>(c->d, c->n_zone_slots);
  k_plan<<<zb, zt, 0, c->stream>>>(c->d, c->n_zone_slots);
  cudaEventRecord(c->fork_ev, c->stream);
  cudaStreamWaitEvent(c->side, c->fork_ev, 0);
  if (c->opts.block_solver == 1)
    k_dts<true><<<zb, zt, 0, c->side>>>(c->d, c->n_zone_slots);
  else
    k_dts<false><<<zb, zt, 0, c->side>>>(c->d, c->n_zone_slots);
  cudaEventRecord(c->join_ev, c->side);
  const int sb = (c->n_tiles + 7) / 8;
  if (c->opts.creation)
    k_sweep<true><<<sb, 256, 0, c->stream>>>(c->d, c->n_tiles);
  else
    k_sweep<false><<<sb, 256, 0, c->stream>>>(c->d, c->n_tiles);
  cudaStreamWaitEvent(c->stream, c->join_ev, 0);
  k_post_zones<<<zb, zt, 0, c->stream>>>(c->d, c->n_zone_slots);
  k_post<<<ib, zt, 0, c->stream>>>(c->d, c->n_inst);
  c->launches += 6;
}

void launch_step(imexds_ctx* c, cudaEvent_t* ev = nullptr) {
  const int zt = 64;
  int zb = (c->n_zone_slots + zt - 1) / zt;
  int ib = (c->n_inst + zt - 1) / zt;
  if (ev) cudaEventRecord(ev[0], c->stream);
  k_pre<<<zb, zt, 0, c->stream>>>(c->d, c->n_zone_slots);
  if (ev) cudaEventRecord(ev[1], c->stream);
  k_plan<<<zb, zt, 0, c->stream>>>(c->d, c->n_zone_slots);
  if (ev) cudaEventRecord(ev[2], c->stream);
  const int sb = (c->n_tiles + 7) / 8;
  if (c->opts.creation)
    k_sweep<true><<<sb, 256, 0, c->stream>>>(c->d, c->n_tiles);
  else
    k_sweep<false><<<sb, 256, 0, c->stream>>>(c->d, c->n_tiles);
  if (ev) cudaEventRecord(ev[3], c->stream);
  if (c->opts.block_solver == 1)
    k_dts<true><<<zb, zt, 0, c->stream>>>(c->d, c->n_zone_slots);
  else
    k_dts<false><<<zb, zt, 0, c->stream>>>(c->d, c->n_zone_slots);
  if (ev) cudaEventRecord(ev[4], c->stream);
  k_post_zones<<<zb, zt, 0, c->stream>>>(c->d, c->n_zone_slots);
  k_post<<<ib, zt, 0, c->stream>>>(c->d, c->n_inst);
  if (ev) cudaEventRecord(ev[5], c->stream);
  c->launches += 6;
}

void accumulate_times(imexds_ctx* c, int steps) {
  for (int s = 0; s < steps; ++s)
    for (int k = 0; k < 5; ++k) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, c->tev[6 * s + k], c->tev[6 * s + k + 1]) == cudaSuccess) {
        c->kt_ms[k] += ms;
        c->kt_n[k] += 1;
      }
    }
}

imexds_status set_ctrl(imexds_ctx* c, double t_end, int clip) {
  // the fluid and options live in module constants shared by every context: load this context's
  CK(cudaMemcpyToSymbolAsync(c_fluid, &c->fluid, sizeof(Fluid), 0, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyToSymbolAsync(c_opts, &c->opts, sizeof(Opts), 0, cudaMemcpyHostToDevice, c->stream));
  Ctrl C{t_end, clip, 0};
  CK(cudaMemcpyAsync(c->d.ctrl, &C, sizeof(Ctrl), cudaMemcpyHostToDevice, c->stream));
  return IMEXDS_OK;
}

// The group-resident kernel for the context's schedule, creation option and block solver.
template <bool CREATION, bool NEWTON>
void launch_group_t(imexds_ctx* c, int n, long long* pc) {
  if (c->async_groups && c->group_threads <= 128)
    k_group_async<CREATION, NEWTON><<<c->n_groups, c->group_threads, 0, c->stream>>>(c->d, c->d_ginst, c->d_grange, n,
                                                                                      pc);
  else if (c->group_threads > 128)
    k_group<CREATION, 256, NEWTON><<<c->n_groups, c->group_threads, 0, c->stream>>>(c->d, c->d_ginst, c->d_grange, n,
                                                                                     pc);
  else
    k_group<CREATION, 128, NEWTON><<<c->n_groups, c->group_threads, 0, c->stream>>>(c->d, c->d_ginst, c->d_grange, n,
                                                                                     pc);
}

void launch_group(imexds_ctx* c, int n, long long* pc) {
  const bool cr = c->opts.creation != 0, nw = c->opts.block_solver == 1;
  if (cr && nw)
    launch_group_t<true, true>(c, n, pc);
  else if (cr)
    launch_group_t<true, false>(c, n, pc);
  else if (nw)
    launch_group_t<false, true>(c, n, pc);
  else
    launch_group_t<false, false>(c, n, pc);
}

imexds_status run_groups(imexds_ctx* c, long long max_steps, bool until_done) {
  // one launch advances every group until its instances are done (or max_steps steps)
  long long done = 0;
  if (c->timing && !c->gev[0]) {
    CK(cudaEventCreate(&c->gev[0]));
    CK(cudaEventCreate(&c->gev[1]));
  }
  if (c->timing && !c->d_phase) {
    CK(cudaMalloc(&c->d_phase, sizeof(long long) * 6 * c->n_groups));
    CK(cudaMemsetAsync(c->d_phase, 0, sizeof(long long) * 6 * c->n_groups, c->stream));
  }
  long long* pc = c->timing ? c->d_phase : nullptr;
  while (done < max_steps) {
    int n = (int)std::min<long long>(max_steps - done, 1 << 30);
    if (c->timing) cudaEventRecord(c->gev[0], c->stream);
    launch_group(c, n, pc);
    if (c->timing) cudaEventRecord(c->gev[1], c->stream);
    k_count_active<<<1, 256, 0, c->stream>>>(c->d, c->n_inst);
    c->launches += 2;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(c->h_active, &c->d.ctrl->n_active, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (c->timing) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, c->gev[0], c->gev[1]) == cudaSuccess) {
        c->kt_ms[5] += ms;
        c->kt_n[5] += 1;
      }
    }
    done += n;
    if (!until_done || *c->h_active == 0) break;
  }
  return IMEXDS_OK;
}

imexds_status run_steps(imexds_ctx* c, long long max_steps, bool until_done) {
  if (c->use_groups) return run_groups(c, max_steps, until_done);
  // Steps are replayed from a CUDA graph of S steps; the host checks the number of active instances
  // after each replay.
  const int S = 8;
  if (c->timing && (int)c->tev.size() < 6 * S) {
    for (int k = (int)c->tev.size(); k < 6 * S; ++k) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      c->tev.push_back(e);
    }
  }
  if (!c->graph || c->graph_steps != S) {
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
    cudaStream_t cs;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    if (!c->side) CK(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
    if (!c->fork_ev) CK(cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming));
    if (!c->join_ev) CK(cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming));
    cudaStream_t saved = c->stream;
    c->stream = cs;
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    long long l0 = c->launches;
    for (int s = 0; s < S; ++s) launch_step_forked(c);
    k_count_active<<<1, 256, 0, cs>>>(c->d, c->n_inst);
    cudaGraph_t g;
    CK(cudaStreamEndCapture(cs, &g));
    c->launches = l0;
    CK(cudaGraphInstantiate(&c->graph, g, 0));
    cudaGraphDestroy(g);
    c->stream = saved;
    cudaStreamDestroy(cs);
    c->graph_steps = S;
  }
  long long done = 0;
  if (c->timing) {
    // measurement mode: eager launches with an event between the kernels of every step
    while (done < max_steps) {
      int n = (int)std::min<long long>(S, max_steps - done);
      for (int s = 0; s < n; ++s) launch_step(c, &c->tev[6 * s]);
      k_count_active<<<1, 256, 0, c->stream>>>(c->d, c->n_inst);
      c->launches += 1;
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(c->h_active, &c->d.ctrl->n_active, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
      CK(cudaStreamSynchronize(c->stream));
      accumulate_times(c, n);
      done += n;
      if (until_done && *c->h_active == 0) break;
    }
    return IMEXDS_OK;
  }
  while (done < max_steps) {
    if (!until_done && max_steps - done < S) {
      for (long long s = done; s < max_steps; ++s) launch_step(c);
      k_count_active<<<1, 256, 0, c->stream>>>(c->d, c->n_inst);
      c->launches += 1;
      CK(cudaGetLastError());
      done = max_steps;
      break;
    }
    CK(cudaGraphLaunch(c->graph, c->stream));
    c->launches += 5 * S + 1;
    done += S;
    if (until_done) {
      CK(cudaMemcpyAsync(c->h_active, &c->d.ctrl->n_active, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
      CK(cudaStreamSynchronize(c->stream));
      if (*c->h_active == 0) break;
    }
  }
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaGetLastError());
  return IMEXDS_OK;
}

}  // namespace

extern "C" {

const char* imexds_status_string(imexds_status s) {
  switch (s) {
    case IMEXDS_OK: return "ok";
    case IMEXDS_ERR_ARG: return "invalid argument";
    case IMEXDS_ERR_CUDA: return "CUDA error";
    case IMEXDS_ERR_NONPHYSICAL: return "non-physical state";
    case IMEXDS_ERR_PB_NOCONV: return "phase-boundary Newton iteration did not converge";
    case IMEXDS_WARN_DTS_MAXITER: return "dual time stepping reached l_max";
    case IMEXDS_ERR_VANISH: return "a phase would vanish";
    case IMEXDS_ERR_TIMEOUT: return "device wait timed out";
    case IMEXDS_ERR_STATE: return "call order";
    case IMEXDS_ERR_CAPACITY: return "zone capacity exceeded";
  }
  return "unknown status";
}

const char* imexds_last_error_string(void) { return g_last_error.c_str(); }

imexds_status imexds_create(const imexds_problem* prob, const imexds_options* opts, void* stream,
                            imexds_ctx** out) {
  if (!out) return IMEXDS_ERR_ARG;
  *out = nullptr;
  if (!prob || prob->n_inst <= 0 || !prob->n_lattice || !prob->x_left || !prob->x_right || !prob->tau)
    return IMEXDS_ERR_ARG;
  imexds_ctx* c = new imexds_ctx();
  c->n_inst = prob->n_inst;
  for (int i = 0; i < prob->n_inst; ++i) {
    if (prob->n_lattice[i] < 2 || !(prob->x_right[i] > prob->x_left[i]) || !(prob->tau[i] >= 0.0)) {
      delete c;
      return IMEXDS_ERR_ARG;
    }
    c->N.push_back(prob->n_lattice[i]);
    c->xL.push_back(prob->x_left[i]);
    c->xR.push_back(prob->x_right[i]);
    c->tau.push_back(prob->tau[i]);
  }
  const imexds_fluid& f = prob->fluid;
  c->fluid.ph[VAP] = make_phase(f.vapour, f.p_sat);
  c->fluid.ph[LIQ] = make_phase(f.liquid, f.p_sat);
  c->fluid.p_sat = f.p_sat;
  c->fluid.p_min = f.p_min;
  c->fluid.p_tilde = f.p_tilde;
  imexds_options o;
  if (opts) {
    o = *opts;
  } else {
    o.cfl = 0.5;
    o.theta_nb = 0.9;
    o.tol_nb = 1e-3;
    o.tol_k = 1e-1;
    o.res_mode = 0;
    o.l_max = 10000;
    o.newton_tol = 1e-12;
    o.newton_itmax = 50;
    o.alpha_min = 1e-8;
    o.split_ratio = 2.0;
    o.creation = 0;
    o.zone_capacity = 0;
    o.schedule = 0;
    o.group_cells = 0;
    o.group_threads = 0;
    o.block_solver = 0;
  }
  if (!(o.cfl > 0.0) || o.l_max < 1 || o.newton_itmax < 1 || !(o.split_ratio > 1.0) || o.block_solver < 0 ||
      o.block_solver > 1) {
    delete c;
    return IMEXDS_ERR_ARG;
  }
  c->opts = Opts{o.cfl, o.theta_nb, o.tol_nb, o.tol_k, o.res_mode, o.l_max, o.newton_tol, o.newton_itmax,
                 o.alpha_min, o.split_ratio, o.creation, o.block_solver};
  c->zone_cap_opt = o.zone_capacity;
  if (o.schedule < 0 || o.schedule > 3) {
    delete c;
    return IMEXDS_ERR_ARG;
  }
  c->schedule_opt = o.schedule;
  if (o.group_cells > 0) {
    c->group_cells = o.group_cells;
    c->group_cells_set = true;
  }
  if (o.group_threads != 0) {
    if (o.group_threads < 64 || o.group_threads > 256 || o.group_threads % 32) {
      delete c;
      return IMEXDS_ERR_ARG;
    }
    c->group_threads = o.group_threads;
  }
  c->stream = (cudaStream_t)stream;
  cudaError_t e = cudaMallocHost(&c->h_active, sizeof(int));
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e);
  }
  *out = c;
  return IMEXDS_OK;
}

void imexds_destroy(imexds_ctx* c) {
  if (!c) return;
  free_dev(c);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->fork_ev) cudaEventDestroy(c->fork_ev);
  if (c->join_ev) cudaEventDestroy(c->join_ev);
  if (c->h_active) cudaFreeHost(c->h_active);
  if (c->adj_mem) cudaFree(c->adj_mem);
  delete c;
}

imexds_status imexds_set_states(imexds_ctx* c, const int32_t* off, const double* widths, const double* rho,
                                const double* m, const uint8_t* phase, double t0) {
  if (!c || !off || !widths || !rho || !m || !phase) return IMEXDS_ERR_ARG;
  const int n = c->n_inst;
  if (off[0] != 0) return IMEXDS_ERR_ARG;
  // host-side parse into lattice + zones
  std::vector<int> lat_off(n + 1, 0);
  for (int i = 0; i < n; ++i) lat_off[i + 1] = lat_off[i] + c->N[i];
  const int n_lat = lat_off[n];
  std::vector<double> hr(n_lat, 1.0), hm(n_lat, 0.0);
  std::vector<unsigned char> hph(n_lat, 1);
  std::vector<std::vector<Zone>> inst_zones(n);
  std::vector<int> status(n, 0);
  // instances are parsed independently (each writes its own lattice range and zone list), on the host's cores
  auto parse = [&](int i) -> imexds_status {
    const int a = off[i], b = off[i + 1], M = b - a, N = c->N[i];
    const double xL = c->xL[i], h = (c->xR[i] - c->xL[i]) / (double)N;
    if (M < 1) return IMEXDS_ERR_ARG;
    // faces: positions accumulate the widths from the last fixed face
    std::vector<int> fpb(M + 1, 0), fj(M + 1, 0);
    std::vector<double> fx(M + 1, 0.0);
    long jfix = 0;
    double part = 0.0;
    bool bad = false;
    for (int k = 0; k < M; ++k) {
      part += widths[a + k];
      if (k + 1 < M && phase[a + k + 1] != phase[a + k]) {
        fpb[k + 1] = 1;
        fx[k + 1] = xL + (double)jfix * h + part;
      } else {
        double units = part / h;
        long j = jfix + std::lround(units);
        if (std::fabs(units - std::round(units)) > 1e-9 || j <= jfix || j > N) bad = true;
        fj[k + 1] = (int)j;
        jfix = j;
        part = 0.0;
      }
    }
    if (fpb[M] || fj[M] != N) bad = true;
    if (bad) return IMEXDS_ERR_ARG;
    for (int k = 0; k < M; ++k)
      if (phase[a + k] > 1 || !(rho[a + k] > 0.0) || !std::isfinite(rho[a + k]) || !std::isfinite(m[a + k]) ||
          !(widths[a + k] > 0.0))
        return IMEXDS_ERR_ARG;
    // cells with two fixed faces spanning one lattice cell are lattice cells; every other cell is part of
    // a zone (runs of such cells, joined when closer than ZONE_GAP)
    std::vector<int> special(M, 0);
    for (int k = 0; k < M; ++k) {
      bool lat = !fpb[k] && !fpb[k + 1] && fj[k + 1] == fj[k] + 1;
      special[k] = !lat;
      if (!fpb[k] && !fpb[k + 1] && !lat) return IMEXDS_ERR_ARG;  // a regular cell spanning several lattice cells
    }
    // group special cells into runs with their lattice footprints
    std::vector<std::pair<int, int>> runs;  // [k0, k1) in cell indices
    for (int k = 0; k < M;) {
      if (!special[k]) {
        ++k;
        continue;
      }
      int k1 = k;
      while (k1 < M && special[k1]) ++k1;
      runs.push_back({k, k1});
      k = k1;
    }
    // join runs whose footprints are closer than ZONE_GAP lattice cells
    std::vector<std::pair<int, int>> joined;
    for (auto& r : runs) {
      if (!joined.empty() && fj[r.first] - fj[joined.back().second] < ZONE_GAP)
        joined.back().second = r.second;
      else
        joined.push_back(r);
    }
    for (auto& r : joined) {
      Zone Z;
      std::memset(&Z, 0, sizeof(Z));
      Z.alive = 1;
      Z.inst = i;
      Z.nc = r.second - r.first;
      if (Z.nc > ZC) return IMEXDS_ERR_CAPACITY;
      Z.A = fj[r.first];
      Z.B = fj[r.second];
      for (int q = 0; q < Z.nc; ++q) {
        int k = r.first + q;
        bool lat = !special[k];
        Z.w[q] = lat ? h : widths[a + k];
        Z.r[q] = rho[a + k];
        Z.m[q] = m[a + k];
        Z.ph[q] = phase[a + k];
      }
      for (int q = 0; q <= Z.nc; ++q) {
        int k = r.first + q;
        Z.fpb[q] = fpb[k];
        Z.fj[q] = fj[k];
        Z.fx[q] = fx[k];
      }
      inst_zones[i].push_back(Z);
    }
    for (int k = 0; k < M; ++k) {
      if (special[k]) continue;
      int j = fj[k];
      hr[lat_off[i] + j] = rho[a + k];
      hm[lat_off[i] + j] = m[a + k];
      hph[lat_off[i] + j] = phase[a + k];
    }
    // lattice phase under zones: the phase of the zone cell covering it (kept for released cells)
    for (auto& Z : inst_zones[i])
      for (int j = Z.A; j < Z.B; ++j) hph[lat_off[i] + j] = (unsigned char)Z.ph[0];
    return IMEXDS_OK;
  };
  {
    for (int i = 0; i < n; ++i)
      if (off[i + 1] - off[i] < 1) return IMEXDS_ERR_ARG;
    std::vector<imexds_status> perr(n, IMEXDS_OK);
    const int nth = std::max(1, std::min({(int)std::thread::hardware_concurrency(), 16, n}));
    auto work = [&](int t) {
      for (int i = t; i < n; i += nth) perr[i] = parse(i);
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < nth; ++t) pool.emplace_back(work, t);
    work(0);
    for (auto& th : pool) th.join();
    for (int i = 0; i < n; ++i)  // the first failing instance decides, as a sequential parse would
      if (perr[i] != IMEXDS_OK) return perr[i];
  }
  std::vector<int> zone_off(n + 1, 0), zone_cap(n, 0);
  for (int i = 0; i < n; ++i) {
    int npb = 0;
    for (auto& Z : inst_zones[i])
      for (int q = 1; q < Z.nc; ++q) npb += Z.fpb[q];
    int cap = c->zone_cap_opt > 0 ? c->zone_cap_opt : 4 + 2 * npb;
    cap = std::max<int>(cap, (int)inst_zones[i].size());
    zone_cap[i] = cap;
    zone_off[i + 1] = zone_off[i] + cap;
  }
  const int n_zone = zone_off[n];
  std::vector<Zone> hz(n_zone);
  std::memset(hz.data(), 0, sizeof(Zone) * hz.size());
  for (int i = 0; i < n; ++i)
    for (size_t q = 0; q < inst_zones[i].size(); ++q) hz[zone_off[i] + q] = inst_zones[i][q];
  std::vector<Inst> hi(n);
  std::memset(hi.data(), 0, sizeof(Inst) * n);
  for (int i = 0; i < n; ++i) {
    Inst& I = hi[i];
    I.N = c->N[i];
    I.lat_off = lat_off[i];
    I.zone_off = zone_off[i];
    I.zone_cap = zone_cap[i];
    I.xL = c->xL[i];
    I.h = (c->xR[i] - c->xL[i]) / (double)c->N[i];
    I.tau = c->tau[i];
    I.t = t0;
    I.status = status[i];
    I.active = 1;
  }
  std::vector<int2> tiles;
  for (int i = 0; i < n; ++i)
    for (int j0 = 0; j0 < c->N[i]; j0 += TILE) tiles.push_back(make_int2(i, j0));
  // the lattice is fixed by the context (n_lat), the zone slots by the boundaries per instance: a call with the
  // layout of the loaded states keeps every device buffer and only uploads the states
  const bool reuse = c->loaded && c->n_lat == n_lat && c->n_zone_slots == n_zone && c->n_tiles == (int)tiles.size();
  if (reuse)
    free_groups(c);
  else
    free_dev(c);
  Dev& d = c->d;
  Dev& sv = c->saved;
  if (!reuse) {
    for (int k = 0; k < 2; ++k) {
      CK(cudaMalloc(&d.rho[k], sizeof(double) * n_lat));
      CK(cudaMalloc(&d.m[k], sizeof(double) * n_lat));
      CK(cudaMalloc(&d.u[k], sizeof(double) * n_lat));
      CK(cudaMalloc(&sv.rho[k], sizeof(double) * n_lat));
      CK(cudaMalloc(&sv.m[k], sizeof(double) * n_lat));
      CK(cudaMalloc(&sv.u[k], sizeof(double) * n_lat));
    }
    CK(cudaMalloc(&d.phase, n_lat));
    CK(cudaMalloc(&d.own, sizeof(int) * n_lat));
    CK(cudaMalloc(&d.zones, sizeof(Zone) * std::max(1, n_zone)));
    CK(cudaMalloc(&d.inst, sizeof(Inst) * n));
    CK(cudaMalloc(&d.ev, sizeof(Event) * EV_CAP * n));
    CK(cudaMalloc(&d.work, sizeof(int) * std::max(1, n_zone)));
    CK(cudaMalloc(&d.tiles, sizeof(int2) * tiles.size()));
    CK(cudaMalloc(&d.ctrl, sizeof(Ctrl)));
    CK(cudaMalloc(&sv.phase, n_lat));
    CK(cudaMalloc(&sv.zones, sizeof(Zone) * std::max(1, n_zone)));
    CK(cudaMalloc(&sv.inst, sizeof(Inst) * n));
    CK(cudaMemcpyAsync(d.tiles, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice, c->stream));
  }
  // both parity buffers start from the same states: one upload, the second buffer filled on the device
  CK(cudaMemcpyAsync(d.rho[0], hr.data(), sizeof(double) * n_lat, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(d.m[0], hm.data(), sizeof(double) * n_lat, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(d.rho[1], d.rho[0], sizeof(double) * n_lat, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMemcpyAsync(d.m[1], d.m[0], sizeof(double) * n_lat, cudaMemcpyDeviceToDevice, c->stream));
  for (int k = 0; k < 2; ++k) k_init_u<<<(n_lat + 255) / 256, 256, 0, c->stream>>>(d.rho[k], d.m[k], d.u[k], n_lat);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(d.phase, hph.data(), n_lat, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemsetAsync(d.own, 0xff, sizeof(int) * n_lat, c->stream));
  CK(cudaMemcpyAsync(d.zones, hz.data(), sizeof(Zone) * n_zone, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(d.inst, hi.data(), sizeof(Inst) * n, cudaMemcpyHostToDevice, c->stream));
  {
    static LogTable host_tab = make_log_table();
    CK(cudaMemcpyToSymbolAsync(g_logtab, &host_tab, sizeof(LogTable), 0, cudaMemcpyHostToDevice, c->stream));
  }
  CK(cudaMemcpyToSymbolAsync(c_fluid, &c->fluid, sizeof(Fluid), 0, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyToSymbolAsync(c_opts, &c->opts, sizeof(Opts), 0, cudaMemcpyHostToDevice, c->stream));
  for (int k = 0; k < 2; ++k) {
    CK(cudaMemcpyAsync(sv.rho[k], d.rho[k], sizeof(double) * n_lat, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(sv.m[k], d.m[k], sizeof(double) * n_lat, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(sv.u[k], d.u[k], sizeof(double) * n_lat, cudaMemcpyDeviceToDevice, c->stream));
  }
  CK(cudaMemcpyAsync(sv.phase, d.phase, n_lat, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMemcpyAsync(sv.zones, d.zones, sizeof(Zone) * n_zone, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMemcpyAsync(sv.inst, d.inst, sizeof(Inst) * n, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  {
    // instance groups: instances sorted by size (largest first), at most GROUP_MAX per group and
    // group_cells lattice cells (at least one instance). (Capping each group's work, sum of N^2, at the
    // balanced share was measured slower: more groups per SM lengthen every group's dual-time chain.)
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return c->N[a] > c->N[b]; });
    // a batch too small to give every SM a group of group_cells cells gets smaller groups (unless the
    // caller fixed group_cells): about total cells / SMs each, at least one instance
    int gcells = c->group_cells;
    if (!c->group_cells_set) {
      int dev = 0, n_sm = 1;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
      long long tot = 0;
      for (int i = 0; i < n; ++i) tot += c->N[i];
      if (tot < (long long)gcells * n_sm) gcells = (int)std::max<long long>(1, (tot + n_sm - 1) / n_sm);
    }
    std::vector<int> ginst;
    std::vector<int2> grange;
    int k = 0;
    while (k < n) {
      int start = k, cells = 0;
      while (k < n && k - start < GROUP_MAX && (k == start || cells + c->N[order[k]] <= gcells)) {
        cells += c->N[order[k]];
        ginst.push_back(order[k]);
        ++k;
      }
      grange.push_back(make_int2(start, k - start));
    }
    CK(cudaMalloc(&c->d_ginst, sizeof(int) * ginst.size()));
    CK(cudaMemcpyAsync(c->d_ginst, ginst.data(), sizeof(int) * ginst.size(), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMalloc(&c->d_grange, sizeof(int2) * grange.size()));
    CK(cudaMemcpyAsync(c->d_grange, grange.data(), sizeof(int2) * grange.size(), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->n_groups = (int)grange.size();
    int maxcap = 0;
    for (int i = 0; i < n; ++i) maxcap = std::max(maxcap, zone_cap[i]);
    // automatic schedule: groups for batches of instances with few boundaries each
    c->use_groups = (c->schedule_opt == 2 || c->schedule_opt == 3) || (c->schedule_opt == 0 && n >= 2 && maxcap <= 16);
    c->async_groups = (c->schedule_opt == 3);
  }
  c->n_lat = n_lat;
  c->n_zone_slots = n_zone;
  c->n_tiles = (int)tiles.size();
  c->lat_off = lat_off;
  c->zone_off = zone_off;
  c->zone_cap = zone_cap;
  c->loaded = true;
  const int ncell = off[n];
  c->u0_off.assign(off, off + n + 1);
  c->u0_w.assign(widths, widths + ncell);
  c->u0_r.assign(rho, rho + ncell);
  c->u0_m.assign(m, m + ncell);
  c->u0_ph.assign(phase, phase + ncell);
  c->u0_t = t0;
  c->prog_k.clear();
  c->prog_a.clear();
  return IMEXDS_OK;
}

imexds_status imexds_set_states_device(imexds_ctx* c, const int32_t* off, const double* w_d, const double* r_d,
                                       const double* m_d, const uint8_t* ph_d, double t0) {
  if (!c || !off || !w_d || !r_d || !m_d || !ph_d) return IMEXDS_ERR_ARG;
  if (off[0] != 0) return IMEXDS_ERR_ARG;
  for (int i = 0; i < c->n_inst; ++i)
    if (off[i + 1] <= off[i]) return IMEXDS_ERR_ARG;  // every instance holds at least one cell
  int n = off[c->n_inst];
  std::vector<double> w(n), r(n), m(n);
  std::vector<uint8_t> ph(n);
  CK(cudaMemcpyAsync(w.data(), w_d, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(r.data(), r_d, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(m.data(), m_d, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(ph.data(), ph_d, n, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return imexds_set_states(c, off, w.data(), r.data(), m.data(), ph.data(), t0);
}

imexds_status imexds_step(imexds_ctx* c, int32_t n_steps) {
  if (!c || n_steps < 0) return IMEXDS_ERR_ARG;
  if (!c->loaded) return IMEXDS_ERR_STATE;
  c->launches = 0;
  imexds_status s = set_ctrl(c, 0.0, 0);
  if (s) return s;
  int gb = c->n_inst;
  k_init_dt<<<gb, 256, 0, c->stream>>>(c->d, c->n_inst);
  c->launches += 1;
  imexds_status st = run_steps(c, n_steps, false);
  if (st == IMEXDS_OK && n_steps > 0) {
    c->prog_k.push_back(0);
    c->prog_a.push_back((double)n_steps);
  }
  return st;
}

imexds_status imexds_run_to(imexds_ctx* c, double t_end) {
  if (!c) return IMEXDS_ERR_ARG;
  if (!c->loaded) return IMEXDS_ERR_STATE;
  c->launches = 0;
  imexds_status s = set_ctrl(c, t_end, 1);
  if (s) return s;
  k_init_dt<<<c->n_inst, 256, 0, c->stream>>>(c->d, c->n_inst);
  c->launches += 1;
  imexds_status st = run_steps(c, kRunToMaxSteps, true);
  if (st == IMEXDS_OK && *c->h_active != 0) return IMEXDS_ERR_TIMEOUT;
  if (st == IMEXDS_OK) {
    c->prog_k.push_back(1);
    c->prog_a.push_back(t_end);
  }
  return st;
}

// device scratch of the gather, allocated with the context's lattice (freed by free_dev)
static imexds_status ensure_gather(imexds_ctx* c) {
  if (c->g_delta) return IMEXDS_OK;
  CK(cudaMalloc(&c->g_delta, sizeof(int) * std::max(1, c->n_lat)));
  CK(cudaMalloc(&c->g_zstart, sizeof(int) * std::max(1, c->n_lat)));
  CK(cudaMalloc(&c->g_cov, std::max(1, c->n_lat)));
  CK(cudaMalloc(&c->g_counts, sizeof(int) * c->n_inst));
  CK(cudaMalloc(&c->g_off, sizeof(int) * (c->n_inst + 1)));
  CK(cudaMalloc(&c->g_t, sizeof(double) * c->n_inst));
  CK(cudaMalloc(&c->g_st, sizeof(int) * c->n_inst));
  return IMEXDS_OK;
}

imexds_status imexds_cell_counts(imexds_ctx* c, int32_t* counts) {
  if (!c || !counts) return IMEXDS_ERR_ARG;
  if (!c->loaded) return IMEXDS_ERR_STATE;
  imexds_status st = ensure_gather(c);
  if (st) return st;
  k_cell_counts<<<(c->n_inst + 127) / 128, 128, 0, c->stream>>>(c->d, c->n_inst, c->g_counts);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(counts, c->g_counts, sizeof(int) * c->n_inst, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return IMEXDS_OK;
}

// The cell lists into device arrays (offsets off_host, already computed from the counts, are copied to the
// device here); no synchronisation.
static imexds_status gather_states(imexds_ctx* c, const int32_t* off_host, double* w_d, double* r_d, double* m_d,
                            uint8_t* ph_d) {
  imexds_status st = ensure_gather(c);
  if (st) return st;
  cudaStream_t sm = c->stream;
  CK(cudaMemcpyAsync(c->g_off, off_host, sizeof(int) * (c->n_inst + 1), cudaMemcpyHostToDevice, sm));
  CK(cudaMemsetAsync(c->g_delta, 0, sizeof(int) * c->n_lat, sm));
  CK(cudaMemsetAsync(c->g_zstart, 0, sizeof(int) * c->n_lat, sm));
  CK(cudaMemsetAsync(c->g_cov, 0, c->n_lat, sm));
  if (c->n_zone_slots > 0)
    k_zone_marks<<<(c->n_zone_slots + 127) / 128, 128, 0, sm>>>(c->d, c->n_zone_slots, c->g_delta, c->g_zstart,
                                                               c->g_cov);
  k_gather_states<<<c->n_inst, 256, 0, sm>>>(c->d, c->g_off, w_d, r_d, m_d, ph_d, c->g_delta, c->g_zstart,
                                             c->g_cov);
  CK(cudaGetLastError());
  return IMEXDS_OK;
}

imexds_status imexds_get_states_device(imexds_ctx* c, int32_t* off, double* w_d, double* r_d, double* m_d,
                                       uint8_t* ph_d, double* t, int32_t* inst_status) {
  if (!c || !off || !w_d || !r_d || !m_d || !ph_d || !t || !inst_status) return IMEXDS_ERR_ARG;
  if (!c->loaded) return IMEXDS_ERR_STATE;
  const int n = c->n_inst;
  std::vector<int32_t> counts(n);
  imexds_status st = imexds_cell_counts(c, counts.data());
  if (st) return st;
  off[0] = 0;
  for (int i = 0; i < n; ++i) off[i + 1] = off[i] + counts[i];
  st = gather_states(c, off, w_d, r_d, m_d, ph_d);
  if (st) return st;
  k_inst_ts<<<(n + 127) / 128, 128, 0, c->stream>>>(c->d, n, c->g_t, c->g_st);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(t, c->g_t, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(inst_status, c->g_st, sizeof(int) * n, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return IMEXDS_OK;
}

// The cell lists gathered on the device (the kernels of imexds_get_states_device) into a packed staging buffer the
// context keeps, then one copy per array into the caller's host memory: only the cells themselves cross the bus.
imexds_status imexds_get_states(imexds_ctx* c, int32_t* off, double* widths, double* rho, double* m,
                                uint8_t* phase, double* t, int32_t* inst_status) {
  if (!c || !off || !widths || !rho || !m || !phase || !t || !inst_status) return IMEXDS_ERR_ARG;
  if (!c->loaded) return IMEXDS_ERR_STATE;
  const int n = c->n_inst;
  std::vector<int32_t> counts(n);
  imexds_status st = imexds_cell_counts(c, counts.data());
  if (st) return st;
  off[0] = 0;
  for (int i = 0; i < n; ++i) off[i + 1] = off[i] + counts[i];
  const size_t tot = (size_t)off[n];
  if (tot > c->g_pack_cells) {
    cudaFree(c->g_pack);
    c->g_pack = nullptr;
    c->g_pack_cells = 0;
    CK(cudaMalloc(&c->g_pack, tot * (3 * sizeof(double) + 1)));
    c->g_pack_cells = tot;
  }
  double* gw = (double*)c->g_pack;
  double* gr = gw + tot;
  double* gm = gr + tot;
  uint8_t* gph = (uint8_t*)(gm + tot);
  st = gather_states(c, off, gw, gr, gm, gph);
  if (st) return st;
  k_inst_ts<<<(n + 127) / 128, 128, 0, c->stream>>>(c->d, n, c->g_t, c->g_st);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(widths, gw, sizeof(double) * tot, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(rho, gr, sizeof(double) * tot, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(m, gm, sizeof(double) * tot, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(phase, gph, tot, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(t, c->g_t, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(inst_status, c->g_st, sizeof(int) * n, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return IMEXDS_OK;
}

imexds_status imexds_reset(imexds_ctx* c) {
  if (!c) return IMEXDS_ERR_ARG;
  if (!c->loaded) return IMEXDS_ERR_STATE;
  Dev& d = c->d;
  Dev& sv = c->saved;
  for (int k = 0; k < 2; ++k) {
    CK(cudaMemcpyAsync(d.rho[k], sv.rho[k], sizeof(double) * c->n_lat, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(d.m[k], sv.m[k], sizeof(double) * c->n_lat, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(d.u[k], sv.u[k], sizeof(double) * c->n_lat, cudaMemcpyDeviceToDevice, c->stream));
  }
  CK(cudaMemcpyAsync(d.phase, sv.phase, c->n_lat, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMemsetAsync(d.own, 0xff, sizeof(int) * c->n_lat, c->stream));
  CK(cudaMemcpyAsync(d.zones, sv.zones, sizeof(Zone) * c->n_zone_slots, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMemcpyAsync(d.inst, sv.inst, sizeof(Inst) * c->n_inst, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->prog_k.clear();
  c->prog_a.clear();
  return IMEXDS_OK;
}

imexds_status imexds_set_kernel_timing(imexds_ctx* c, int32_t on) {
  if (!c) return IMEXDS_ERR_ARG;
  if ((on != 0) != (c->timing != 0)) {
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  c->timing = on ? 1 : 0;
  for (int k = 0; k < 6; ++k) {
    c->kt_ms[k] = 0.0;
    c->kt_n[k] = 0;
  }
  if (c->d_phase) CK(cudaMemsetAsync(c->d_phase, 0, sizeof(long long) * 6 * c->n_groups, c->stream));
  return IMEXDS_OK;
}

__global__ void k_check_div(const double* a, const double* b, double* fast, double* ref, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    fast[i] = div_nr(a[i], b[i]);
    ref[i] = a[i] / b[i];
  }
}

imexds_status imexds_check_div(int32_t n, const double* a, const double* b, double* fast, double* ref) {
  if (n <= 0 || !a || !b || !fast || !ref) return IMEXDS_ERR_ARG;
  double* d = nullptr;
  CK(cudaMalloc(&d, sizeof(double) * 4 * (size_t)n));
  CK(cudaMemcpy(d, a, sizeof(double) * n, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d + n, b, sizeof(double) * n, cudaMemcpyHostToDevice));
  k_check_div<<<(n + 255) / 256, 256>>>(d, d + n, d + 2 * (size_t)n, d + 3 * (size_t)n, n);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpy(fast, d + 2 * (size_t)n, sizeof(double) * n, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(ref, d + 3 * (size_t)n, sizeof(double) * n, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e);
  return IMEXDS_OK;
}

__global__ void k_check_tol(const double* d, const double* w, const double* lim, uint8_t* fast, uint8_t* ref,
                            int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    fast[i] = below_tol(d[i], w[i], lim[i]) ? 1 : 0;
    ref[i] = (fabs(d[i]) < lim[i] * fmax(fabs(w[i]), 1.0)) ? 1 : 0;
  }
}

imexds_status imexds_check_tol(int32_t n, const double* d, const double* w, const double* lim, uint8_t* fast,
                               uint8_t* ref) {
  if (n <= 0 || !d || !w || !lim || !fast || !ref) return IMEXDS_ERR_ARG;
  double* g = nullptr;
  CK(cudaMalloc(&g, sizeof(double) * 3 * (size_t)n + 2 * (size_t)n));
  uint8_t* gb = (uint8_t*)(g + 3 * (size_t)n);
  cudaError_t e = cudaMemcpy(g, d, sizeof(double) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(g + n, w, sizeof(double) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(g + 2 * (size_t)n, lim, sizeof(double) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_check_tol<<<(n + 255) / 256, 256>>>(g, g + n, g + 2 * (size_t)n, gb, gb + n, n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(fast, gb, n, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(ref, gb + n, n, cudaMemcpyDeviceToHost);
  cudaFree(g);
  if (e != cudaSuccess) return cuda_fail(e);
  return IMEXDS_OK;
}

imexds_status imexds_check_log(int32_t n, const double* x, double* fast, double* ref) {
  if (n <= 0 || !x || !fast || !ref) return IMEXDS_ERR_ARG;
  static LogTable host_tab = make_log_table();
  CK(cudaMemcpyToSymbol(g_logtab, &host_tab, sizeof(LogTable)));
  double *dx = nullptr, *df = nullptr, *dr = nullptr;
  CK(cudaMalloc(&dx, sizeof(double) * n));
  CK(cudaMalloc(&df, sizeof(double) * n));
  CK(cudaMalloc(&dr, sizeof(double) * n));
  CK(cudaMemcpy(dx, x, sizeof(double) * n, cudaMemcpyHostToDevice));
  k_check_log<<<(n + 255) / 256, 256>>>(n, dx, df, dr);
  CK(cudaGetLastError());
  CK(cudaMemcpy(fast, df, sizeof(double) * n, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(ref, dr, sizeof(double) * n, cudaMemcpyDeviceToHost));
  cudaFree(dx);
  cudaFree(df);
  cudaFree(dr);
  return IMEXDS_OK;
}

imexds_status imexds_step_uniform_noalloc(const imexds_fluid* fluid, double cfl, int32_t n_inst,
                                          const int32_t* n_lattice, const double* x_left, const double* x_right,
                                          const double* rho_in, const double* m_in, const uint8_t* phase,
                                          double* rho_out, double* m_out, double* dt_out, void* stream) {
  namespace na = imexds_noalloc;
  auto arg_error = [](const char* why) {
    g_last_error = std::string("imexds_step_uniform_noalloc: ") + why;
    return IMEXDS_ERR_ARG;
  };
  if (!fluid || !n_lattice || !x_left || !x_right || !rho_in || !m_in || !phase || !rho_out || !m_out || !dt_out)
    return arg_error("a pointer argument is NULL");
  if (!(cfl > 0.0)) return arg_error("cfl must be positive");
  if (n_inst <= 0) return arg_error("n_inst must be positive");
  if (n_inst > na::kMaxInst) {
    g_last_error = "imexds_step_uniform_noalloc: n_inst exceeds the fixed scratch size (16384 instances)";
    return IMEXDS_ERR_CAPACITY;
  }
  long long cells = 0, tiles = 0;
  for (int i = 0; i < n_inst; ++i) {
    if (n_lattice[i] < 2) return arg_error("an instance has fewer than 2 cells");
    if (!(x_right[i] > x_left[i])) return arg_error("an instance has x_right <= x_left");
    cells += n_lattice[i];
    tiles += (n_lattice[i] + 31) / 32;
  }
  if (cells > 0x7fffffffLL) return arg_error("more than 2^31 - 1 cells in total");
  // set-up once per device, with that device current: the device address of the scratch array
  static void* scratch_ptr[64] = {nullptr};
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return arg_error("device ordinal above 63");
  if (!scratch_ptr[dev]) CK(cudaGetSymbolAddress(&scratch_ptr[dev], na::g_scratch));
  na::Scratch* scr = (na::Scratch*)scratch_ptr[dev];
  cudaStream_t st = (cudaStream_t)stream;
  Fluid F;
  F.ph[VAP] = make_phase(fluid->vapour, fluid->p_sat);
  F.ph[LIQ] = make_phase(fluid->liquid, fluid->p_sat);
  F.p_sat = fluid->p_sat;
  F.p_min = fluid->p_min;
  F.p_tilde = fluid->p_tilde;
  CK(cudaMemcpyAsync(scr->n_lattice, n_lattice, sizeof(int) * n_inst, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(scr->x_left, x_left, sizeof(double) * n_inst, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(scr->x_right, x_right, sizeof(double) * n_inst, cudaMemcpyHostToDevice, st));
  na::k_setup<<<1, 32, 0, st>>>(scr, n_inst);
  na::k_dt<<<n_inst, 256, 0, st>>>(scr, F, cfl, rho_in, m_in, phase, dt_out);
  na::k_sweep<<<(int)((tiles + 7) / 8), 256, 0, st>>>(scr, F, n_inst, (int)tiles, rho_in, m_in, phase, rho_out,
                                                      m_out);
  CK(cudaGetLastError());
  int err = 0;
  CK(cudaMemcpyAsync(&err, &scr->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (err & na::kErrState)
    return arg_error("a cell has a phase byte above 1, a density that is not positive and finite, or a non-finite "
                     "momentum (rho_out and m_out were not written)");
  if (err & na::kErrMixed)
    return arg_error("an instance holds cells of both phases (rho_out and m_out were not written)");
  return IMEXDS_OK;
}

imexds_status imexds_get_group_phase_cycles(imexds_ctx* c, int64_t* slowest6, int64_t* sum6) {
  if (!c || !slowest6 || !sum6) return IMEXDS_ERR_ARG;
  for (int k = 0; k < 6; ++k) slowest6[k] = sum6[k] = 0;
  if (!c->d_phase) return IMEXDS_OK;
  std::vector<long long> h(6 * c->n_groups);
  CK(cudaMemcpy(h.data(), c->d_phase, sizeof(long long) * h.size(), cudaMemcpyDeviceToHost));
  int worst = 0;
  for (int g = 0; g < c->n_groups; ++g) {
    if (h[6 * g + 5] > h[6 * worst + 5]) worst = g;
    for (int k = 0; k < 6; ++k) sum6[k] += h[6 * g + k];
  }
  for (int k = 0; k < 6; ++k) slowest6[k] = h[6 * worst + k];
  return IMEXDS_OK;
}

imexds_status imexds_set_schedule(imexds_ctx* c, int32_t schedule) {
  if (!c || schedule < 0 || schedule > 3) return IMEXDS_ERR_ARG;
  if (!c->loaded) return IMEXDS_ERR_STATE;
  c->schedule_opt = schedule;
  int maxcap = 0;
  for (int i = 0; i < c->n_inst; ++i) maxcap = std::max(maxcap, c->zone_cap[i]);
  c->use_groups = (schedule == 2 || schedule == 3) || (schedule == 0 && c->n_inst >= 2 && maxcap <= 16);
  c->async_groups = (schedule == 3);
  return IMEXDS_OK;
}

imexds_status imexds_get_kernel_times(imexds_ctx* c, double* total_ms, int64_t* launches) {
  if (!c || !total_ms || !launches) return IMEXDS_ERR_ARG;
  for (int k = 0; k < 6; ++k) {
    total_ms[k] = c->kt_ms[k];
    launches[k] = c->kt_n[k];
  }
  return IMEXDS_OK;
}

imexds_status imexds_get_stats(imexds_ctx* c, int64_t* stats) {
  if (!c || !stats) return IMEXDS_ERR_ARG;
  if (!c->loaded) return IMEXDS_ERR_STATE;
  std::vector<Inst> hi(c->n_inst);
  CK(cudaMemcpyAsync(hi.data(), c->d.inst, sizeof(Inst) * c->n_inst, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (int i = 0; i < c->n_inst; ++i) {
    for (int k = 0; k < N_STATS; ++k) stats[10 * i + k] = hi[i].stats[k];
    stats[10 * i + 9] = c->launches;
  }
  return IMEXDS_OK;
}

imexds_status imexds_set_adjoint_checkpoint(imexds_ctx* c, int32_t every) {
  if (!c || every < 1) return IMEXDS_ERR_ARG;
  c->adj_k = every;
  return IMEXDS_OK;
}

namespace {
// One imexds_adjoint / imexds_adjoint_device call: the layout of the per-instance slots and what the host keeps.
struct AdjRun {
  int n = 0, oT = 0;
  long long stride = 0;
  std::vector<int32_t> MT;   // final cell counts of the forward run
  std::vector<int64_t> stats;
  std::vector<long long> offs;
  std::vector<unsigned char> hfpb;  // initial face kinds, slot layout
  std::vector<imexds::adj::AInst> hI;
  imexds::adj::ADev A{};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  // device copies for the device variant
  long long* d_offs = nullptr;
  int *d_toff = nullptr, *d_u0off = nullptr;
  unsigned char *d_fpb0 = nullptr, *chk_ph = nullptr;
  double *chk_w = nullptr, *chk_r = nullptr, *chk_m = nullptr, *d_err = nullptr;
};
}  // namespace

// The steps both adjoint entry points share: the slot layout, one device allocation kept by the context, the
// initial lists of the last imexds_set_states (the library's own copies), the seeds (host arrays copied in, or
// device arrays scattered by k_scatter_seeds) and the k_adjoint launch between two events. No synchronisation.
static imexds_status adjoint_launch(imexds_ctx* c, AdjRun& R, const double* dJ_dw_T, const double* dJ_drho_T,
                                    const double* dJ_dm_T, bool dev_seeds) {
  using namespace imexds::adj;
  const int n = c->n_inst;
  R.n = n;
  // the last forward: final cell counts and steps per instance
  R.MT.assign(n, 0);
  imexds_status st = imexds_cell_counts(c, R.MT.data());
  if (st) return st;
  R.stats.assign((size_t)n * 10, 0);
  st = imexds_get_stats(c, R.stats.data());
  if (st) return st;
  long long max_steps = 0;
  for (int i = 0; i < n; ++i) max_steps = std::max<long long>(max_steps, R.stats[10 * i]);
  const int k = c->adj_k;
  const int n_ck = (int)(max_steps / k) + 1;
  // layout: instance i owns slots [off_i, off_i + cap_i + 1) of every per-cell / per-face array
  R.offs.assign(n, 0);
  std::vector<int> caps(n);
  long long stride = 0;
  R.oT = 0;
  for (int i = 0; i < n; ++i) {
    const int M0 = c->u0_off[i + 1] - c->u0_off[i];
    caps[i] = std::max(M0, (int)R.MT[i]) + ACAP_PAD;
    R.offs[i] = stride;
    stride += caps[i] + 1;
    R.oT += R.MT[i];
  }
  R.stride = stride;
  const int n_prog = (int)c->prog_k.size();
  // one device allocation carved into the arrays
  const size_t nd_cell = 28, nb_cell = 6, ni_cell = 1;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  size_t bytes = 0;
  bytes += al(sizeof(AInst) * n) + al(sizeof(int) * (n_prog + 1)) + al(sizeof(double) * (n_prog + 1));
  bytes += nd_cell * al(sizeof(double) * stride) + nb_cell * al(stride) + ni_cell * al(sizeof(int) * stride);
  bytes += 6 * al(sizeof(double) * stride * n_ck) + 2 * al(stride * n_ck) + al(sizeof(int) * stride * n_ck);
  bytes += al(sizeof(ACk) * (size_t)n * n_ck) + al(sizeof(int) * n);
  bytes += 3 * al(sizeof(double) * stride * k) + 2 * al(stride * k) + al(sizeof(int) * (size_t)n * k);
  bytes += al(sizeof(StepRec) * (size_t)n * k);
  // device variant: slot offsets, final and initial offsets, initial face kinds, the forward run's final
  // lists for the replay check, per-instance deviations
  bytes += al(sizeof(long long) * n) + 2 * al(sizeof(int) * (n + 1)) + 2 * al(stride) + 3 * al(sizeof(double) * stride);
  bytes += al(sizeof(double) * n);
  if (bytes > c->adj_bytes) {
    if (c->adj_mem) cudaFree(c->adj_mem);
    c->adj_mem = nullptr;
    c->adj_bytes = 0;
    CK(cudaMalloc(&c->adj_mem, bytes));
    c->adj_bytes = bytes;
  }
  char* p = (char*)c->adj_mem;
  auto take = [&](size_t b) {
    char* q = p;
    p += al(b);
    return (void*)q;
  };
  ADev& A = R.A;
  A = ADev{};
  A.n_inst = n;
  A.k = k;
  A.n_ck = n_ck;
  A.n_prog = n_prog;
  A.stride = stride;
  A.I = (AInst*)take(sizeof(AInst) * n);
  int* d_pk = (int*)take(sizeof(int) * (n_prog + 1));
  double* d_pa = (double*)take(sizeof(double) * (n_prog + 1));
  A.pk = d_pk;
  A.pa = d_pa;
  double** dcell[28] = {&A.w,  &A.r,  &A.m,  &A.fx, &A.F0, &A.F1, &A.LF0, &A.LF1, &A.CL0, &A.CL1,
                        &A.CR0, &A.CR1, &A.pw, &A.pr, &A.pm, &A.lw, &A.lr,  &A.lm,  &A.lx,  &A.nw,
                        &A.nr,  &A.nm,  &A.nx, &A.fin_w, &A.fin_r, &A.fin_m, &A.pwl, &A.pwr};
  for (auto q : dcell) *q = (double*)take(sizeof(double) * stride);
  unsigned char** bcell[6] = {&A.ph, &A.fpb, &A.pph, &A.pfpb, &A.fin_ph, &A.cdet};
  for (auto q : bcell) *q = (unsigned char*)take(stride);
  A.fj = (int*)take(sizeof(int) * stride);
  A.ck_w = (double*)take(sizeof(double) * stride * n_ck);
  A.ck_r = (double*)take(sizeof(double) * stride * n_ck);
  A.ck_m = (double*)take(sizeof(double) * stride * n_ck);
  A.ck_fx = (double*)take(sizeof(double) * stride * n_ck);
  A.ck_pwl = (double*)take(sizeof(double) * stride * n_ck);
  A.ck_pwr = (double*)take(sizeof(double) * stride * n_ck);
  A.ck_ph = (unsigned char*)take(stride * n_ck);
  A.ck_fpb = (unsigned char*)take(stride * n_ck);
  A.ck_fj = (int*)take(sizeof(int) * stride * n_ck);
  A.ck_h = (ACk*)take(sizeof(ACk) * (size_t)n * n_ck);
  A.fin_M = (int*)take(sizeof(int) * n);
  A.tp_w = (double*)take(sizeof(double) * stride * k);
  A.tp_r = (double*)take(sizeof(double) * stride * k);
  A.tp_m = (double*)take(sizeof(double) * stride * k);
  A.tp_ph = (unsigned char*)take(stride * k);
  A.tp_fpb = (unsigned char*)take(stride * k);
  A.tp_M = (int*)take(sizeof(int) * (size_t)n * k);
  A.rec = (StepRec*)take(sizeof(StepRec) * (size_t)n * k);
  R.d_offs = (long long*)take(sizeof(long long) * n);
  R.d_toff = (int*)take(sizeof(int) * (n + 1));
  R.d_u0off = (int*)take(sizeof(int) * (n + 1));
  R.d_fpb0 = (unsigned char*)take(stride);
  R.chk_ph = (unsigned char*)take(stride);
  R.chk_w = (double*)take(sizeof(double) * stride);
  R.chk_r = (double*)take(sizeof(double) * stride);
  R.chk_m = (double*)take(sizeof(double) * stride);
  R.d_err = (double*)take(sizeof(double) * n);
  // initial lists (faces as in imexds_set_states: positions accumulate from the last fixed face)
  std::vector<double> hw(stride, 0.0), hr(stride, 0.0), hm(stride, 0.0), hfx(stride, 0.0);
  std::vector<unsigned char> hph(stride, 0);
  R.hfpb.assign(stride, 0);
  std::vector<unsigned char>& hfpb = R.hfpb;
  std::vector<int> hfj(stride, 0);
  R.hI.assign(n, AInst{});
  for (int i = 0; i < n; ++i) {
    const int a = c->u0_off[i], M0 = c->u0_off[i + 1] - a;
    const long long o = R.offs[i];
    const double h = (c->xR[i] - c->xL[i]) / c->N[i];
    long jfix = 0;
    double part = 0.0;
    hfpb[o] = 0;
    hfj[o] = 0;
    for (int q = 0; q < M0; ++q) {
      hw[o + q] = c->u0_w[a + q];
      hr[o + q] = c->u0_r[a + q];
      hm[o + q] = c->u0_m[a + q];
      hph[o + q] = c->u0_ph[a + q];
      part += c->u0_w[a + q];
      if (q + 1 < M0 && c->u0_ph[a + q + 1] != c->u0_ph[a + q]) {
        hfpb[o + q + 1] = 1;
        hfx[o + q + 1] = c->xL[i] + (double)jfix * h + part;
      } else {
        long j = jfix + std::lround(part / h);
        hfj[o + q + 1] = (int)j;
        jfix = j;
        part = 0.0;
      }
    }
    for (int q = 0; q < M0; ++q)  // a cell with two fixed faces is a whole number of lattice cells
      if (!hfpb[o + q] && !hfpb[o + q + 1]) hw[o + q] = (double)(hfj[o + q + 1] - hfj[o + q]) * h;
    AInst& I = R.hI[i];
    I.off = o;
    I.cap = caps[i];
    I.M = M0;
    I.M_seed = R.MT[i];
    I.nexp = (int)R.stats[10 * i];
    I.h = h;
    I.xL = c->xL[i];
    I.tau = c->tau[i];
    I.t = c->u0_t;
  }
  cudaStream_t sm = c->stream;
  st = set_ctrl(c, 0.0, 0);
  if (st) return st;
  CK(cudaMemcpyAsync(A.I, R.hI.data(), sizeof(AInst) * n, cudaMemcpyHostToDevice, sm));
  if (n_prog) {
    CK(cudaMemcpyAsync(d_pk, c->prog_k.data(), sizeof(int) * n_prog, cudaMemcpyHostToDevice, sm));
    CK(cudaMemcpyAsync(d_pa, c->prog_a.data(), sizeof(double) * n_prog, cudaMemcpyHostToDevice, sm));
  }
  CK(cudaMemcpyAsync(A.w, hw.data(), sizeof(double) * stride, cudaMemcpyHostToDevice, sm));
  CK(cudaMemcpyAsync(A.r, hr.data(), sizeof(double) * stride, cudaMemcpyHostToDevice, sm));
  CK(cudaMemcpyAsync(A.m, hm.data(), sizeof(double) * stride, cudaMemcpyHostToDevice, sm));
  CK(cudaMemcpyAsync(A.fx, hfx.data(), sizeof(double) * stride, cudaMemcpyHostToDevice, sm));
  CK(cudaMemcpyAsync(A.ph, hph.data(), stride, cudaMemcpyHostToDevice, sm));
  CK(cudaMemcpyAsync(A.fpb, hfpb.data(), stride, cudaMemcpyHostToDevice, sm));
  CK(cudaMemcpyAsync(A.fj, hfj.data(), sizeof(int) * stride, cudaMemcpyHostToDevice, sm));
  // seeds in the slots of the final lists
  if (dev_seeds) {
    std::vector<int> toff(n + 1, 0);
    for (int i = 0; i < n; ++i) toff[i + 1] = toff[i] + R.MT[i];
    CK(cudaMemcpyAsync(R.d_offs, R.offs.data(), sizeof(long long) * n, cudaMemcpyHostToDevice, sm));
    CK(cudaMemcpyAsync(R.d_toff, toff.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, sm));
    CK(cudaMemcpyAsync(R.d_u0off, c->u0_off.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, sm));
    CK(cudaMemcpyAsync(R.d_fpb0, hfpb.data(), stride, cudaMemcpyHostToDevice, sm));
    CK(cudaMemsetAsync(A.lw, 0, sizeof(double) * stride, sm));
    CK(cudaMemsetAsync(A.lr, 0, sizeof(double) * stride, sm));
    CK(cudaMemsetAsync(A.lm, 0, sizeof(double) * stride, sm));
    k_scatter_seeds<<<n, 128, 0, sm>>>(R.d_offs, R.d_toff, dJ_dw_T, dJ_drho_T, dJ_dm_T, A.lw, A.lr, A.lm);
    CK(cudaGetLastError());
  } else {
    std::vector<double> lw(stride, 0.0), lr(stride, 0.0), lm(stride, 0.0);
    int oT = 0;
    for (int i = 0; i < n; ++i)
      for (int q = 0; q < R.MT[i]; ++q, ++oT) {
        lw[R.offs[i] + q] = dJ_dw_T ? dJ_dw_T[oT] : 0.0;
        lr[R.offs[i] + q] = dJ_drho_T[oT];
        lm[R.offs[i] + q] = dJ_dm_T[oT];
      }
    CK(cudaMemcpyAsync(A.lw, lw.data(), sizeof(double) * stride, cudaMemcpyHostToDevice, sm));
    CK(cudaMemcpyAsync(A.lr, lr.data(), sizeof(double) * stride, cudaMemcpyHostToDevice, sm));
    CK(cudaMemcpyAsync(A.lm, lm.data(), sizeof(double) * stride, cudaMemcpyHostToDevice, sm));
    CK(cudaStreamSynchronize(sm));  // the staging vectors leave scope
  }
  CK(cudaMemsetAsync(A.lx, 0, sizeof(double) * stride, sm));
  CK(cudaMemsetAsync(A.pwl, 0, sizeof(double) * stride, sm));
  CK(cudaMemsetAsync(A.pwr, 0, sizeof(double) * stride, sm));
  CK(cudaEventCreate(&R.e0));
  CK(cudaEventCreate(&R.e1));
  CK(cudaEventRecord(R.e0, sm));
  // instances per CTA (one warp each): as many as give about two CTAs per SM, at most AWARPS
  int dev = 0, n_sm = 1;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  const int G = std::max(1, std::min(AWARPS, (n + 2 * n_sm - 1) / (2 * n_sm)));
  k_adjoint<<<(n + G - 1) / G, 32 * G, 0, sm>>>(A);
  CK(cudaGetLastError());
  CK(cudaEventRecord(R.e1, sm));
  // the host staging of the initial lists must outlive the copies
  CK(cudaStreamSynchronize(sm));
  return IMEXDS_OK;
}

// The kernel time of the last launch and the replay check shared by both entry points: an instance whose
// replay took another step count or ended with another cell count than the forward run reports
// IMEXDS_ERR_STATE; err[i] is the instance's largest deviation of its replayed final states.
static void adjoint_finish(imexds_ctx* c, AdjRun& R, const std::vector<int>& fM, const std::vector<double>& err) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, R.e0, R.e1);
  cudaEventDestroy(R.e0);
  cudaEventDestroy(R.e1);
  c->adj_ms = ms;
  double worst = 0.0;
  long long cell_steps = 0;
  for (int i = 0; i < R.n; ++i) {
    imexds::adj::AInst& I = R.hI[i];
    if (I.status == 0 && (I.nsteps != R.stats[10 * i] || fM[i] != R.MT[i])) {
      I.status = IMEXDS_ERR_STATE;
      I.site = (I.nsteps != R.stats[10 * i]) ? 6 : 7;
    }
    if (I.status) continue;
    worst = std::max(worst, err[i]);
    cell_steps += (long long)I.nsteps * (c->u0_off[i + 1] - c->u0_off[i]);
  }
  c->adj_replay_err = worst;
  c->adj_cell_steps = cell_steps;
}

imexds_status imexds_adjoint(imexds_ctx* c, const double* dJ_dw_T, const double* dJ_drho_T, const double* dJ_dm_T,
                             double* dJ_dw0, double* dJ_drho0, double* dJ_dm0, double* dJ_dtau,
                             int32_t* inst_status) {
  if (!c || !dJ_drho_T || !dJ_dm_T || !dJ_drho0 || !dJ_dm0 || !dJ_dtau) return IMEXDS_ERR_ARG;
  if (!c->loaded || c->u0_off.empty()) return IMEXDS_ERR_STATE;
  AdjRun R;
  imexds_status st = adjoint_launch(c, R, dJ_dw_T, dJ_drho_T, dJ_dm_T, false);
  if (st) return st;
  const int n = R.n;
  const long long stride = R.stride;
  const imexds::adj::ADev& A = R.A;
  cudaStream_t sm = c->stream;
  // results
  CK(cudaMemcpyAsync(R.hI.data(), A.I, sizeof(imexds::adj::AInst) * n, cudaMemcpyDeviceToHost, sm));
  std::vector<double> lw(stride), lr(stride), lm(stride), lx(stride), fw(stride), fr(stride), fm(stride);
  std::vector<int> fM(n);
  CK(cudaMemcpyAsync(lw.data(), A.lw, sizeof(double) * stride, cudaMemcpyDeviceToHost, sm));
  CK(cudaMemcpyAsync(lr.data(), A.lr, sizeof(double) * stride, cudaMemcpyDeviceToHost, sm));
  CK(cudaMemcpyAsync(lm.data(), A.lm, sizeof(double) * stride, cudaMemcpyDeviceToHost, sm));
  CK(cudaMemcpyAsync(lx.data(), A.lx, sizeof(double) * stride, cudaMemcpyDeviceToHost, sm));
  CK(cudaMemcpyAsync(fw.data(), A.fin_w, sizeof(double) * stride, cudaMemcpyDeviceToHost, sm));
  CK(cudaMemcpyAsync(fr.data(), A.fin_r, sizeof(double) * stride, cudaMemcpyDeviceToHost, sm));
  CK(cudaMemcpyAsync(fm.data(), A.fin_m, sizeof(double) * stride, cudaMemcpyDeviceToHost, sm));
  CK(cudaMemcpyAsync(fM.data(), A.fin_M, sizeof(int) * n, cudaMemcpyDeviceToHost, sm));
  CK(cudaStreamSynchronize(sm));
  // the replay must reproduce the last forward: same steps, same cells, states to round-off
  std::vector<int32_t> toff(n + 1);
  std::vector<double> gw(R.oT), gr(R.oT), gm(R.oT), gt(n);
  std::vector<uint8_t> gph(R.oT);
  std::vector<int32_t> gst(n);
  st = imexds_get_states(c, toff.data(), gw.data(), gr.data(), gm.data(), gph.data(), gt.data(), gst.data());
  if (st) return st;
  std::vector<double> err(n, 0.0);
  for (int i = 0; i < n; ++i) {
    if (fM[i] != R.MT[i]) continue;
    double rmax = 0.0, dr = 0.0, dm = 0.0, dw = 0.0;
    for (int q = 0; q < R.MT[i]; ++q) rmax = std::max(rmax, std::fabs(gr[toff[i] + q]));
    for (int q = 0; q < R.MT[i]; ++q) {
      const long long o = R.offs[i] + q;
      dr = std::max(dr, std::fabs(fr[o] - gr[toff[i] + q]));
      dm = std::max(dm, std::fabs(fm[o] - gm[toff[i] + q]));
      dw = std::max(dw, std::fabs(fw[o] - gw[toff[i] + q]) / ((c->xR[i] - c->xL[i]) / c->N[i]));
    }
    err[i] = std::max(dr / rmax, std::max(dm / rmax, dw));
  }
  adjoint_finish(c, R, fM, err);
  c->adj_fin_off.assign(n + 1, 0);
  c->adj_fin_w.clear();
  c->adj_fin_r.clear();
  c->adj_fin_m.clear();
  c->adj_site.assign(n, 0);
  for (int i = 0; i < n; ++i) {
    const long long o = R.offs[i];
    for (int q = 0; q < fM[i]; ++q) {
      c->adj_fin_w.push_back(fw[o + q]);
      c->adj_fin_r.push_back(fr[o + q]);
      c->adj_fin_m.push_back(fm[o + q]);
    }
    c->adj_fin_off[i + 1] = c->adj_fin_off[i] + fM[i];
    c->adj_site[i] = R.hI[i].site;
  }
  // gradients with respect to the initial lists; a boundary position is the last fixed face plus the
  // widths after it, so its adjoint adds to the widths of those cells; lattice cells have fixed widths
  const double nan = std::nan("");
  for (int i = 0; i < n; ++i) {
    const imexds::adj::AInst& I = R.hI[i];
    const int a = c->u0_off[i], M0 = c->u0_off[i + 1] - a;
    const long long o = R.offs[i];
    if (inst_status) inst_status[i] = I.status;
    dJ_dtau[i] = I.status ? nan : I.lam_tau;
    double acc = 0.0;  // adjoint of the boundary positions to the right of the current cell, within its segment
    std::vector<double> wtot(M0, 0.0);
    for (int q = M0 - 1; q >= 0; --q) {
      if (!R.hfpb[o + q + 1]) acc = 0.0;
      if (R.hfpb[o + q + 1]) acc += lx[o + q + 1];
      wtot[q] = lw[o + q] + acc;
    }
    for (int q = 0; q < M0; ++q) {
      dJ_drho0[a + q] = I.status ? nan : lr[o + q];
      dJ_dm0[a + q] = I.status ? nan : lm[o + q];
      if (dJ_dw0) {
        const bool lattice = !R.hfpb[o + q] && !R.hfpb[o + q + 1];
        dJ_dw0[a + q] = I.status ? nan : (lattice ? 0.0 : wtot[q]);
      }
    }
  }
  return IMEXDS_OK;
}

imexds_status imexds_adjoint_device(imexds_ctx* c, const double* dJ_dw_T, const double* dJ_drho_T,
                                    const double* dJ_dm_T, double* dJ_dw0, double* dJ_drho0, double* dJ_dm0,
                                    double* dJ_dtau, int32_t* inst_status) {
  if (!c || !dJ_drho_T || !dJ_dm_T || !dJ_drho0 || !dJ_dm0 || !dJ_dtau) return IMEXDS_ERR_ARG;
  if (!c->loaded || c->u0_off.empty()) return IMEXDS_ERR_STATE;
  AdjRun R;
  imexds_status st = adjoint_launch(c, R, dJ_dw_T, dJ_drho_T, dJ_dm_T, true);
  if (st) return st;
  const int n = R.n;
  const imexds::adj::ADev& A = R.A;
  cudaStream_t sm = c->stream;
  // the replay check on the device: the forward run's final lists gathered beside the replayed ones
  std::vector<int32_t> toff(n + 1, 0);
  for (int i = 0; i < n; ++i) toff[i + 1] = toff[i] + R.MT[i];
  st = gather_states(c, toff.data(), R.chk_w, R.chk_r, R.chk_m, R.chk_ph);
  if (st) return st;
  k_replay_err<<<n, 128, 0, sm>>>(A.I, R.d_offs, R.d_toff, A.fin_w, A.fin_r, A.fin_m, R.chk_w, R.chk_r, R.chk_m,
                                  R.d_err);
  CK(cudaGetLastError());
  std::vector<int> fM(n);
  std::vector<double> err(n);
  CK(cudaMemcpyAsync(R.hI.data(), A.I, sizeof(imexds::adj::AInst) * n, cudaMemcpyDeviceToHost, sm));
  CK(cudaMemcpyAsync(fM.data(), A.fin_M, sizeof(int) * n, cudaMemcpyDeviceToHost, sm));
  CK(cudaMemcpyAsync(err.data(), R.d_err, sizeof(double) * n, cudaMemcpyDeviceToHost, sm));
  CK(cudaStreamSynchronize(sm));
  adjoint_finish(c, R, fM, err);
  // the replay's final lists stay on the device: imexds_adjoint_replay reports the sites only
  c->adj_fin_off.assign(n + 1, 0);
  c->adj_fin_w.clear();
  c->adj_fin_r.clear();
  c->adj_fin_m.clear();
  c->adj_site.assign(n, 0);
  for (int i = 0; i < n; ++i) c->adj_site[i] = R.hI[i].site;
  // gradients into the caller's arrays, with the statuses of the check
  CK(cudaMemcpyAsync(A.I, R.hI.data(), sizeof(imexds::adj::AInst) * n, cudaMemcpyHostToDevice, sm));
  k_adj_grads<<<(n + 127) / 128, 128, 0, sm>>>(n, A.I, R.d_offs, R.d_u0off, R.d_fpb0, A.lw, A.lr, A.lm, A.lx,
                                              dJ_dw0, dJ_drho0, dJ_dm0, dJ_dtau);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(sm));
  if (inst_status)
    for (int i = 0; i < n; ++i) inst_status[i] = R.hI[i].status;
  return IMEXDS_OK;
}

imexds_status imexds_adjoint_replay(imexds_ctx* c, int32_t* cell_offsets, double* widths, double* rho, double* m,
                                    int32_t* stop_site) {
  if (!c || !cell_offsets) return IMEXDS_ERR_ARG;
  if (c->adj_fin_off.empty()) return IMEXDS_ERR_STATE;
  const int n = c->n_inst;
  for (int i = 0; i <= n; ++i) cell_offsets[i] = c->adj_fin_off[i];
  const size_t tot = c->adj_fin_w.size();
  if (widths) std::copy(c->adj_fin_w.begin(), c->adj_fin_w.end(), widths);
  if (rho) std::copy(c->adj_fin_r.begin(), c->adj_fin_r.end(), rho);
  if (m) std::copy(c->adj_fin_m.begin(), c->adj_fin_m.end(), m);
  (void)tot;
  if (stop_site)
    for (int i = 0; i < n; ++i) stop_site[i] = c->adj_site[i];
  return IMEXDS_OK;
}

imexds_status imexds_adjoint_info(imexds_ctx* c, double* kernel_ms, double* replay_err, int64_t* cell_steps) {
  if (!c) return IMEXDS_ERR_ARG;
  if (kernel_ms) *kernel_ms = c->adj_ms;
  if (replay_err) *replay_err = c->adj_replay_err;
  if (cell_steps) *cell_steps = c->adj_cell_steps;
  return IMEXDS_OK;
}

}  // extern "C"
