// Oracle: plain FP64 CPU implementation of the explicit-implicit domain-splitting scheme of
// May & Thein (arXiv 2211.00705) for the 1-D isothermal Euler equations with a sharp
// liquid-vapour interface and kinetic-relation mass transfer.
//
// TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU baseline of the
// benchmark; the product library never links, includes or calls it. It is written to be read
// against the paper: a moving-grid cell list (one std::vector entry per cell, insert/erase on
// topology events), every formula in the paper's order and notation, no blocking or fusion.
// Build with -O2 -ffp-contract=off (no fused multiply-add, no fast-math).
//
// Readings of points the paper leaves open are marked "Reading:" and are listed in the design
// notes of the repository.
#include "oracle.h"

#include "counted.h"
#include "dual.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <thread>
#include <type_traits>
#include <vector>

namespace {

const int VAP = 0;
const int LIQ = 1;

// ---------------------------------------------------------------- thermodynamics (Sec. 2.1, Sec. 4)

struct Phase {
  int kind;
  double a2, a, p0, rho0;
  double rho_sat;  // density at the saturation pressure: zero of the Gibbs energy
};

struct Fluid {
  Phase ph[2];
  double p_sat, p_min, p_tilde;
};

Fluid make_fluid(const orc_fluid* f) {
  Fluid F;
  for (int k = 0; k < 2; ++k) {
    F.ph[k].kind = f->ph[k].kind;
    F.ph[k].a2 = f->ph[k].a2;
    F.ph[k].a = std::sqrt(f->ph[k].a2);
    F.ph[k].p0 = f->ph[k].p0;
    F.ph[k].rho0 = f->ph[k].rho0;
  }
  F.p_sat = f->p_sat;
  F.p_min = f->p_min;
  F.p_tilde = f->p_tilde;
  for (int k = 0; k < 2; ++k) {
    const Phase& e = F.ph[k];
    F.ph[k].rho_sat = (e.kind == 0) ? F.p_sat / e.a2 : e.rho0 + (F.p_sat - e.p0) / e.a2;
  }
  return F;
}

// Every function below is a template on the scalar type T: T = double is the oracle itself; T = a
// forward-mode dual number (dual.h) gives the derivative of the same computation (the oracle's
// tangent-linear mode). Branches, maxima and stop tests act on values only.
using orcdual::tmax;
using orcdual::tmin;
using orcdual::val;
template <class T>
T tsqrt(const T& x) {
  using orcdual::sqrt;
  using std::sqrt;
  return sqrt(x);
}
template <class T>
T tlog(const T& x) {
  using orcdual::log;
  using std::log;
  return log(x);
}
template <class T>
T texp(const T& x) {
  using orcdual::exp;
  using std::exp;
  return exp(x);
}
template <class T>
T tfabs(const T& x) {
  using orcdual::fabs;
  using std::fabs;
  return fabs(x);
}

// Vapour: ideal gas p = (kT0/m) rho (Eq. eos:isoT_idgas). Liquid: linear Tait p = p0 + K0(rho/rho0 - 1)
// (Eq. eos:isoT_lintait; Reading: the printed "- p0" inside the bracket is read as "- 1", a2 = K0/rho0).
template <class T>
T pressure(const Phase& e, const T& rho) {
  return e.kind == 0 ? T(e.a2 * rho) : T(e.p0 + e.a2 * (rho - e.rho0));
}
template <class T>
T density(const Phase& e, const T& p) {
  return e.kind == 0 ? T(p / e.a2) : T(e.rho0 + (p - e.p0) / e.a2);
}
// Admissible pressure range of a phase: the density it maps to must be positive.
template <class T>
bool valid_pressure(const Phase& e, const T& p) {
  return std::isfinite(val(p)) && val(density(e, p)) > 0.0;
}
// Gibbs energy g = f + p/rho with dg = v dp at fixed T (Sec. 2.1). For both EOS, dp = a2 drho, so
// g = a2 ln(rho/rho_sat). Reading: both phases share the zero at the saturation pressure, where
// the Maxwell construction makes the Gibbs energies equal.
template <class T>
T gibbs(const Phase& e, const T& rho) {
  return e.a2 * tlog(T(rho / e.rho_sat));
}

// Physical flux F(U) = (rho u, rho u^2 + p) of the isothermal Euler system (Eq. eeq:isoT both).
template <class T>
void phys_flux(const Phase& e, const T& r, const T& m, T F[2]) {
  T u = m / r;
  F[0] = m;
  F[1] = m * u + pressure(e, r);
}

// HLL approximate Riemann solver (Toro) at a face between two cells of the same phase, used at all
// regular faces (Sec. 4). Reading: Davis wave-speed estimates S_L = min(u_l - a, u_r - a),
// S_R = max(u_l + a, u_r + a).
template <class T>
void hll(const Phase& e, const T& rl, const T& ml, const T& rr, const T& mr, T F[2]) {
  T ul = ml / rl, ur = mr / rr;
  T Fl[2], Fr[2];
  phys_flux(e, rl, ml, Fl);
  phys_flux(e, rr, mr, Fr);
  T SL = tmin(T(ul - e.a), T(ur - e.a));
  T SR = tmax(T(ul + e.a), T(ur + e.a));
  if (val(SL) >= 0.0) {
    F[0] = Fl[0];
    F[1] = Fl[1];
  } else if (val(SR) <= 0.0) {
    F[0] = Fr[0];
    F[1] = Fr[1];
  } else {
    T Ul[2] = {rl, ml}, Ur[2] = {rr, mr};
    for (int c = 0; c < 2; ++c) F[c] = (SR * Fl[c] - SL * Fr[c] + SL * SR * (Ur[c] - Ul[c])) / (SR - SL);
  }
}

// Wave function of a classical outer wave (App. A): f_K(p*) = sqrt(-[[p]][[v]]) for a shock
// (p* > p_K), and the integral of v/a from p_K to p* for a rarefaction. For an isothermal linear EOS
// (dp = a2 drho) that integral is a ln(rho*/rho_K). df/dp* is returned in *dfdp.
template <class T>
T wave_f(const Phase& e, const T& pstar, const T& rhoK, T* dfdp) {
  T pK = pressure(e, rhoK);
  T rs = density(e, pstar);
  T vs = 1.0 / rs;
  if (val(pstar) > val(pK)) {
    T dv = 1.0 / rhoK - vs;  // v_K - v* >= 0
    T q = (pstar - pK) * dv;
    T f = tsqrt(q);
    T dq = dv + (pstar - pK) * vs * vs / e.a2;  // d/dp* of (p* - p_K)(v_K - v*)
    *dfdp = (val(f) > 0.0) ? T(0.5 * dq / f) : T(vs / e.a);
    if constexpr (orcdual::is_dual<T>::value) {
      // Tangent mode only. For the linear isothermal EOS (dp = a2 drho on either branch)
      // (p* - p_K)(v_K - v*) = (p* - p_K)^2 / (a2 rho_K rho*), so f = (p* - p_K) / (a sqrt(rho_K rho*)) and
      // df/dp* = (1 - (p* - p_K) v* / (2 a2)) / (a sqrt(rho_K rho*)). The derivative parts come from these
      // forms: near p* = p_K the product rounds to zero and the square root's derivative is 0 * inf, theirs
      // stay finite. The values remain those of the definition above.
      T den = e.a * tsqrt(T(rhoK * rs));
      f = orcdual::with_value(val(f), T((pstar - pK) / den));
      *dfdp = orcdual::with_value(val(*dfdp), T((1.0 - (pstar - pK) * vs / (2.0 * e.a2)) / den));
    }
    return f;
  }
  *dfdp = vs / e.a;
  return e.a * tlog(T(rs / rhoK));
}

// One side of a phase boundary: star pressure, phase, density, volume, Gibbs energy and dv/dp.
template <class T>
struct Side {
  T p, rho, v, g, dv;
};

template <class T>
Side<T> side_at(const Phase& e, const T& p) {
  Side<T> s;
  s.p = p;
  s.rho = density(e, p);
  s.v = 1.0 / s.rho;
  s.g = gibbs(e, s.rho);
  s.dv = -s.v * s.v / e.a2;  // dv/dp = -v^2/a^2
  return s;
}

// Kinetic relation z = tau p_V [[g + e_kin]] (Eq. isoT:kin_rel1) at a phase boundary with left star
// side L and right star side R. Reading: e_kin = (u - w)^2 / 2 is taken relative to the moving
// boundary, so [[e_kin]] = z^2 [[v^2]] / 2, and z^2 = -[[p]]/[[v]] (Eq. isoT:pb_mom_balance) turns it
// into [[e_kin]] = -[[p]] (v_L + v_R) / 2. dz/dp of both sides in *dzl, *dzr.
template <class T>
T kinetic_z(const T& tau, bool left_is_vapour, const Side<T>& L, const Side<T>& R, T* dzl, T* dzr) {
  T pV = left_is_vapour ? L.p : R.p;
  T jp = R.p - L.p;
  T Q = (R.g - L.g) - 0.5 * jp * (L.v + R.v);
  // dQ/dp_L = -v_L + (v_L+v_R)/2 - jp dv_L/2 ; dQ/dp_R = v_R - (v_L+v_R)/2 - jp dv_R/2 (dg/dp = v)
  T dQl = -L.v + 0.5 * (L.v + R.v) - 0.5 * jp * L.dv;
  T dQr = R.v - 0.5 * (L.v + R.v) - 0.5 * jp * R.dv;
  *dzl = tau * ((left_is_vapour ? Q : T(0.0)) + pV * dQl);
  *dzr = tau * ((left_is_vapour ? T(0.0) : Q) + pV * dQr);
  return tau * pV * Q;
}

// The 2x2 system G(p_l*, p_r*) of Eq. 2p_RP:ex_sys, oriented left/right:
//   G1 = [[p]] + z^2 [[v]],  G2 = f_l + f_r + z [[v]] + (u_r - u_l)
// and its Jacobian (Eq. jacobian:ex_sys).
template <class T>
struct PBSys {
  T G[2], J[2][2], z;
  Side<T> L, R;
  T fl, fr;
};

template <class T>
bool pb_eval(const Fluid& F, const T& tau, int phl, const T& rl, const T& ul, int phr, const T& rr, const T& ur,
             const T& pls, const T& prs, PBSys<T>* S) {
  const Phase& El = F.ph[phl];
  const Phase& Er = F.ph[phr];
  if (!valid_pressure(El, pls) || !valid_pressure(Er, prs)) return false;
  S->L = side_at(El, pls);
  S->R = side_at(Er, prs);
  T dzl, dzr;
  T z = kinetic_z(tau, phl == VAP, S->L, S->R, &dzl, &dzr);
  T dfl, dfr;
  S->fl = wave_f(El, pls, rl, &dfl);
  S->fr = wave_f(Er, prs, rr, &dfr);
  T jp = prs - pls, jv = S->R.v - S->L.v;
  S->z = z;
  S->G[0] = jp + z * z * jv;
  S->G[1] = S->fl + S->fr + z * jv + (ur - ul);
  // d[[v]]/dp_l = -dv_l, d[[v]]/dp_r = dv_r
  S->J[0][0] = -1.0 + 2.0 * z * dzl * jv - z * z * S->L.dv;
  S->J[0][1] = 1.0 + 2.0 * z * dzr * jv + z * z * S->R.dv;
  S->J[1][0] = dfl + dzl * jv - z * S->L.dv;
  S->J[1][1] = dfr + dzr * jv + z * S->R.dv;
  return std::isfinite(val(S->G[0])) && std::isfinite(val(S->G[1]));
}

template <class T>
struct PBResult {
  T pl, pr, rl, rr, ul, ur, z, w, F[2];
  int iters;
  int ok;
};

// Initial guess (App. A, Eq. HLLC:2p_nopt): HLLC wave-speed estimates give the boundary speed w and
// the liquid star density; the liquid EOS gives a star pressure used for both unknowns.
// Reading: if that pressure is not positive, the vapour side starts at max(p_vapour, 1e-3 p_sat) and
// the liquid side at its own pressure. (Computed on values: the converged Newton solution does not
// depend on where it started.)
void pb_initial_guess(const Fluid& F, int phl, double rl, double ul, int phr, double rr, double ur,
                      double* pl0, double* pr0) {
  const Phase& El = F.ph[phl];
  const Phase& Er = F.ph[phr];
  double pl = pressure(El, rl), pr = pressure(Er, rr);
  double Sl = ul - El.a, Sr = ur + Er.a;
  double w = (pr - pl + rl * ul * (Sl - ul) - rr * ur * (Sr - ur)) / (rl * (Sl - ul) - rr * (Sr - ur));
  double rls;
  if (phl == LIQ)
    rls = rl * (Sl - ul) / (Sl - w);
  else
    rls = rr * (Sr - ur) / (Sr - w);
  double p = pressure(F.ph[LIQ], rls);
  if (std::isfinite(p) && p > 0.0) {
    *pl0 = p;
    *pr0 = p;
    return;
  }
  double pv = (phl == VAP) ? pl : pr;
  double pliq = (phl == LIQ) ? pl : pr;
  double pvg = std::max(pv, 1e-3 * F.p_sat);
  *pl0 = (phl == VAP) ? pvg : pliq;
  *pr0 = (phr == VAP) ? pvg : pliq;
}

// Newton's method with the Armijo rule (Kelley 1995): direction d = -DG^{-1} G, step halving until
// ||G(x + lam d)|| <= (1 - 1e-4 lam) ||G(x)||. Reading: the merit norm is the Euclidean norm of
// (G1 / (rho_l a_l + rho_r a_r), G2), both in m/s; at most 20 halvings; convergence when the
// accepted step is below newton_tol relative to max(|p|, p_sat).
template <class T>
PBResult<T> pb_solve(const Fluid& F, const orc_opts& o, const T& tau, int phl, const T& rl, const T& ml, int phr,
                     const T& rr, const T& mr) {
  PBResult<T> R;
  R.ok = 0;
  R.iters = 0;
  T ul = ml / rl, ur = mr / rr;
  double imp = val(rl) * F.ph[phl].a + val(rr) * F.ph[phr].a;
  double x0, x1;
  pb_initial_guess(F, phl, val(rl), val(ul), phr, val(rr), val(ur), &x0, &x1);
  T x[2] = {x0, x1};
  PBSys<T> S;
  if (!pb_eval(F, tau, phl, rl, ul, phr, rr, ur, x[0], x[1], &S)) return R;
  double nrm = std::hypot(val(S.G[0]) / imp, val(S.G[1]));
  bool conv = (nrm == 0.0);
  int it = 0;
  while (!conv && it < o.newton_itmax) {
    ++it;
    T det = S.J[0][0] * S.J[1][1] - S.J[0][1] * S.J[1][0];
    if (!(std::isfinite(val(det))) || val(det) == 0.0) break;
    T d0 = -(S.J[1][1] * S.G[0] - S.J[0][1] * S.G[1]) / det;
    T d1 = -(-S.J[1][0] * S.G[0] + S.J[0][0] * S.G[1]) / det;
    double lam = 1.0;
    bool acc = false;
    PBSys<T> Tr;
    for (int ls = 0; ls <= 20; ++ls) {
      if (pb_eval(F, tau, phl, rl, ul, phr, rr, ur, T(x[0] + lam * d0), T(x[1] + lam * d1), &Tr)) {
        double nt = std::hypot(val(Tr.G[0]) / imp, val(Tr.G[1]));
        if (nt <= (1.0 - 1e-4 * lam) * nrm) {
          acc = true;
          nrm = nt;
          break;
        }
      }
      lam *= 0.5;
    }
    double s0 = std::fabs(val(d0)) / std::max(std::fabs(val(x[0])), F.p_sat);
    double s1 = std::fabs(val(d1)) / std::max(std::fabs(val(x[1])), F.p_sat);
    if (!acc) {
      // No decrease possible: accept only if the full Newton step is already at round-off level.
      if (std::max(s0, s1) <= 1e-9) conv = true;
      break;
    }
    x[0] = x[0] + lam * d0;
    x[1] = x[1] + lam * d1;
    S = Tr;
    if (lam * std::max(s0, s1) <= o.newton_tol || nrm == 0.0) conv = true;
  }
  R.iters = it;
  if (!conv) return R;
  // Recovery (App. A): densities from the EOS, velocities from the outer-wave relations,
  // boundary speed from z = -rho (u - w), flux F_PB = (-z, -z u* + p*) (Eq. pb_flux:pt).
  // Reading: the vapour-side star state enters the momentum flux and w.
  R.pl = x[0];
  R.pr = x[1];
  R.rl = S.L.rho;
  R.rr = S.R.rho;
  R.ul = ul - S.fl;
  R.ur = ur + S.fr;
  R.z = S.z;
  T uV = (phl == VAP) ? R.ul : R.ur;
  T vV = (phl == VAP) ? S.L.v : S.R.v;
  T pV = (phl == VAP) ? R.pl : R.pr;
  R.w = uV + R.z * vV;
  R.F[0] = -R.z;
  R.F[1] = -R.z * uV + pV;
  R.ok = 1;
  return R;
}

// Star pressure of the same-phase Riemann problem without phase transition, the root of
// phi(p) = f(p; W_l) + f(p; W_r) + (u_r - u_l). Two rarefactions give the closed form
// rho* = sqrt(rho_l rho_r) exp((u_l - u_r) / (2a)), exact when p* <= min(p_l, p_r). Otherwise the
// root lies in [min(p_l, p_r), p_TR] (a shock curve lies above the rarefaction curve) and is found by
// bisection to round-off. (Used for the creation decision only: values.)
double nopt_star(const Phase& e, double rl, double ul, double rr, double ur) {
  double pl = pressure(e, rl), pr = pressure(e, rr);
  double pm = std::min(pl, pr);
  double rs = std::sqrt(rl * rr) * std::exp((ul - ur) / (2.0 * e.a));
  double ptr = pressure(e, rs);
  if (ptr <= pm) return ptr;
  double lo = pm, hi = ptr, d;
  for (int i = 0; i < 200; ++i) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    double phi = wave_f(e, mid, rl, &d) + wave_f(e, mid, rr, &d) + (ur - ul);
    if (phi > 0.0)
      hi = mid;
    else
      lo = mid;
  }
  return 0.5 * (lo + hi);
}

// Single-phase Riemann problem with phase creation (App. B; the system itself is in the cited work
// and not printed). Reading: unknowns (p_P-, p_C, p_P+) for parent phase P and created phase C; the
// two boundaries each satisfy the momentum jump [[p]] + z^2 [[v]] = 0 with their own z from the
// kinetic relation, and the velocity chains through both boundaries:
//   f_P(p_P-; W_l) + f_P(p_P+; W_r) + z1 [[v]]_1 + z2 [[v]]_2 + (u_r - u_l) = 0.
template <class T>
struct CreateResult {
  T pPl, pC, pPr, rhoC, uC, z1, z2, w1, w2, uPl, uPr;
  int iters;
  int ok;
};

template <class T>
struct CrSys {
  T E[3], J[3][3];
  Side<T> Pl, C, Pr;
  T z1, z2, fl, fr;
};

template <class T>
bool cr_eval(const Fluid& F, const T& tau, int P, const T& rl, const T& ul, const T& rr, const T& ur, const T x[3],
             CrSys<T>* S) {
  int Cph = 1 - P;
  const Phase& EP = F.ph[P];
  const Phase& EC = F.ph[Cph];
  if (!valid_pressure(EP, x[0]) || !valid_pressure(EC, x[1]) || !valid_pressure(EP, x[2])) return false;
  S->Pl = side_at(EP, x[0]);
  S->C = side_at(EC, x[1]);
  S->Pr = side_at(EP, x[2]);
  T dz1a, dz1b, dz2a, dz2b;
  // left boundary: parent (left) | created (right); right boundary: created (left) | parent (right)
  S->z1 = kinetic_z(tau, P == VAP, S->Pl, S->C, &dz1a, &dz1b);
  S->z2 = kinetic_z(tau, Cph == VAP, S->C, S->Pr, &dz2a, &dz2b);
  T dfl, dfr;
  S->fl = wave_f(EP, x[0], rl, &dfl);
  S->fr = wave_f(EP, x[2], rr, &dfr);
  T jv1 = S->C.v - S->Pl.v, jv2 = S->Pr.v - S->C.v;
  T z1 = S->z1, z2 = S->z2;
  S->E[0] = (x[1] - x[0]) + z1 * z1 * jv1;
  S->E[1] = (x[2] - x[1]) + z2 * z2 * jv2;
  S->E[2] = S->fl + S->fr + z1 * jv1 + z2 * jv2 + (ur - ul);
  // derivatives with respect to x0 = p_P-, x1 = p_C, x2 = p_P+
  S->J[0][0] = -1.0 + 2.0 * z1 * dz1a * jv1 - z1 * z1 * S->Pl.dv;
  S->J[0][1] = 1.0 + 2.0 * z1 * dz1b * jv1 + z1 * z1 * S->C.dv;
  S->J[0][2] = 0.0;
  S->J[1][0] = 0.0;
  S->J[1][1] = -1.0 + 2.0 * z2 * dz2a * jv2 - z2 * z2 * S->C.dv;
  S->J[1][2] = 1.0 + 2.0 * z2 * dz2b * jv2 + z2 * z2 * S->Pr.dv;
  S->J[2][0] = dfl + dz1a * jv1 - z1 * S->Pl.dv;
  S->J[2][1] = dz1b * jv1 + z1 * S->C.dv + dz2a * jv2 - z2 * S->C.dv;
  S->J[2][2] = dfr + dz2b * jv2 + z2 * S->Pr.dv;
  return std::isfinite(val(S->E[0])) && std::isfinite(val(S->E[1])) && std::isfinite(val(S->E[2]));
}

// Solve a 3x3 linear system by Gaussian elimination with partial pivoting.
template <class T>
bool solve3(T A[3][3], T b[3], T x[3]) {
  T M[3][4];
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) M[i][j] = A[i][j];
    M[i][3] = b[i];
  }
  for (int c = 0; c < 3; ++c) {
    int p = c;
    for (int r = c + 1; r < 3; ++r)
      if (std::fabs(val(M[r][c])) > std::fabs(val(M[p][c]))) p = r;
    if (val(M[p][c]) == 0.0 || !std::isfinite(val(M[p][c]))) return false;
    if (p != c)
      for (int j = 0; j < 4; ++j) std::swap(M[p][j], M[c][j]);
    for (int r = c + 1; r < 3; ++r) {
      T f = M[r][c] / M[c][c];
      for (int j = c; j < 4; ++j) M[r][j] = M[r][j] - f * M[c][j];
    }
  }
  for (int i = 2; i >= 0; --i) {
    T s = M[i][3];
    for (int j = i + 1; j < 3; ++j) s = s - M[i][j] * x[j];
    x[i] = s / M[i][i];
  }
  return true;
}

// Newton-Armijo for the creation system, as for the two-phase boundary. Reading: all three
// pressures start at the saturation pressure; the merit norm scales the two momentum jumps by the
// parent impedance rho a.
template <class T>
CreateResult<T> creation_solve(const Fluid& F, const orc_opts& o, const T& tau, int P, const T& rl, const T& ml,
                               const T& rr, const T& mr) {
  CreateResult<T> R;
  R.ok = 0;
  R.iters = 0;
  T ul = ml / rl, ur = mr / rr;
  double imp = (val(rl) + val(rr)) * F.ph[P].a;
  T x[3] = {F.p_sat, F.p_sat, F.p_sat};
  CrSys<T> S;
  if (!cr_eval(F, tau, P, rl, ul, rr, ur, x, &S)) return R;
  auto norm = [&](const CrSys<T>& s) {
    double e0 = val(s.E[0]), e1 = val(s.E[1]), e2 = val(s.E[2]);
    return std::sqrt((e0 / imp) * (e0 / imp) + (e1 / imp) * (e1 / imp) + e2 * e2);
  };
  double nrm = norm(S);
  bool conv = (nrm == 0.0);
  int it = 0;
  while (!conv && it < o.newton_itmax) {
    ++it;
    T b[3] = {-S.E[0], -S.E[1], -S.E[2]}, d[3];
    if (!solve3(S.J, b, d)) break;
    double lam = 1.0;
    bool acc = false;
    CrSys<T> Tr;
    for (int ls = 0; ls <= 20; ++ls) {
      T xt[3] = {x[0] + lam * d[0], x[1] + lam * d[1], x[2] + lam * d[2]};
      if (cr_eval(F, tau, P, rl, ul, rr, ur, xt, &Tr)) {
        double nt = norm(Tr);
        if (nt <= (1.0 - 1e-4 * lam) * nrm) {
          acc = true;
          nrm = nt;
          break;
        }
      }
      lam *= 0.5;
    }
    double s = 0.0;
    for (int i = 0; i < 3; ++i) s = std::max(s, std::fabs(val(d[i])) / std::max(std::fabs(val(x[i])), F.p_sat));
    if (!acc) {
      if (s <= 1e-9) conv = true;
      break;
    }
    for (int i = 0; i < 3; ++i) x[i] = x[i] + lam * d[i];
    S = Tr;
    if (lam * s <= o.newton_tol || nrm == 0.0) conv = true;
  }
  R.iters = it;
  if (!conv) return R;
  R.pPl = x[0];
  R.pC = x[1];
  R.pPr = x[2];
  R.rhoC = S.C.rho;
  R.z1 = S.z1;
  R.z2 = S.z2;
  R.uPl = ul - S.fl;
  R.uPr = ur + S.fr;
  R.uC = R.uPl - S.z1 * (S.C.v - S.Pl.v);  // velocity jump across the left boundary: [[u]] = -z [[v]]
  R.w1 = R.uC + S.z1 * S.C.v;              // z = -rho (u - w) on the created side
  R.w2 = R.uC + S.z2 * S.C.v;
  R.ok = (val(R.w2) > val(R.w1)) ? 1 : 0;
  return R;
}

// ---------------------------------------------------------------- moving grid (Sec. 2.3, Sec. 3.4)

template <class T>
struct Face {
  int pb;     // 1: phase boundary (moves with w); 0: fixed face on the background lattice
  long j;     // lattice index of a fixed face (position x_left + j h)
  T x;        // position of a phase boundary
};

template <class T>
struct Inst {
  long N = 0;
  double xL = 0, xR = 0, h = 0;
  T tau = 0.0;
  std::vector<Face<T>> f;               // M + 1 faces
  std::vector<T> w, r, m;               // M cells: width, rho, rho u
  std::vector<int> ph;                  // M cells: phase label
  T t = 0.0;
  int status = 0;
  long long steps = 0, dts_iters = 0, dts_max = 0, newton = 0, merges = 0, splits = 0, creations = 0,
            maxiter = 0, pb_solves = 0;
  double last_implicit_res = 0;
  int M() const { return (int)r.size(); }
  T face_x(int i) const { return f[i].pb ? f[i].x : T(xL + (double)f[i].j * h); }
};

struct Ctx;

double sound(const Fluid& F, int ph) { return F.ph[ph].a; }

template <class T>
bool finite_state(const Inst<T>& I) {
  for (int i = 0; i < I.M(); ++i)
    if (!(val(I.r[i]) > 0.0) || !std::isfinite(val(I.r[i])) || !std::isfinite(val(I.m[i])) || !(val(I.w[i]) > 0.0))
      return false;
  return true;
}

// Merge cell i with its neighbour nb (same phase, shared fixed face): conservative average.
template <class T>
void merge_cells(Inst<T>& I, int i, int nb) {
  int a = std::min(i, nb), b = std::max(i, nb);
  T wm = I.w[a] + I.w[b];
  T rm = (I.w[a] * I.r[a] + I.w[b] * I.r[b]) / wm;
  T mm = (I.w[a] * I.m[a] + I.w[b] * I.m[b]) / wm;
  I.w[a] = wm;
  I.r[a] = rm;
  I.m[a] = mm;
  I.w.erase(I.w.begin() + b);
  I.r.erase(I.r.begin() + b);
  I.m.erase(I.m.begin() + b);
  I.ph.erase(I.ph.begin() + b);
  I.f.erase(I.f.begin() + b);  // face between a and b
  I.merges++;
}

// Solve the phase-boundary problem at face g between cells g-1 and g of the given states.
template <class T>
PBResult<T> solve_face(const Fluid& F, const orc_opts& o, Inst<T>& I, int phl, const T& rl, const T& ml, int phr,
                       const T& rr, const T& mr) {
  PBResult<T> R = pb_solve(F, o, I.tau, phl, rl, ml, phr, rr, mr);
  I.pb_solves++;
  I.newton += R.iters;
  return R;
}

// Flux of the dual-time loop / Part 2 at an interior face g of a block, given the block states
// W (indexed by cell). Returns the face speed (0 for a fixed face).
template <class T>
bool block_face_flux(const Fluid& Fl, const orc_opts& o, Inst<T>& I, int g, const std::vector<T>& Wr,
                     const std::vector<T>& Wm, T F[2], T* wface) {
  if (I.f[g].pb) {
    PBResult<T> R = solve_face(Fl, o, I, I.ph[g - 1], Wr[g - 1], Wm[g - 1], I.ph[g], Wr[g], Wm[g]);
    if (!R.ok) return false;
    F[0] = R.F[0];
    F[1] = R.F[1];
    *wface = R.w;
  } else {
    hll(Fl.ph[I.ph[g]], Wr[g - 1], Wm[g - 1], Wr[g], Wm[g], F);
    *wface = 0.0;
  }
  return true;
}

// The update T of Algorithm 2 Part 1 for the cells lo..hi of a block (Eq. godunov_meth:nonunif with fluxes
// and widths at the iterate W): T_i = (h^n_i U^n_i - dt (F_{i+1/2}(W) - F_{i-1/2}(W))) / h_i(W),
// h_i(W) = h^n_i + (w_{i+1/2}(W) - w_{i-1/2}(W)) dt, the outer fluxes FL, FR fixed at U^n. Written for any
// scalar type S of the iterate (everything else as plain values), so that dual numbers give dT/dW.
template <class S>
bool block_update(const Fluid& Fl, const orc_opts& o, double tau, const std::vector<int>& ph,
                  const std::vector<Face<double>>& f, int lo, int hi, const std::vector<double>& wn,
                  const std::vector<double>& rn, const std::vector<double>& mn, const double FL[2],
                  const double FR[2], double dt, const std::vector<S>& Wr, const std::vector<S>& Wm,
                  std::vector<S>& out) {
  const int n = hi - lo + 1;
  std::vector<S> F0(n + 1), F1(n + 1), wc(n + 1, S(0.0));
  F0[0] = FL[0];
  F1[0] = FL[1];
  F0[n] = FR[0];
  F1[n] = FR[1];
  for (int g = lo + 1; g <= hi; ++g) {
    const int q = g - lo;
    S Fx[2];
    if (f[g].pb) {
      PBResult<S> R = pb_solve(Fl, o, S(tau), ph[g - 1], Wr[g - 1], Wm[g - 1], ph[g], Wr[g], Wm[g]);
      if (!R.ok) return false;
      Fx[0] = R.F[0];
      Fx[1] = R.F[1];
      wc[q] = R.w;
    } else {
      hll(Fl.ph[ph[g]], Wr[g - 1], Wm[g - 1], Wr[g], Wm[g], Fx);
    }
    F0[q] = Fx[0];
    F1[q] = Fx[1];
  }
  for (int i = lo; i <= hi; ++i) {
    const int q = i - lo;
    S hl = wn[i] + (wc[q + 1] - wc[q]) * dt;
    if (!(val(hl) > 0.0)) return false;
    out[2 * q] = wn[i] / hl * rn[i] - dt / hl * (F0[q + 1] - F0[q]);
    out[2 * q + 1] = wn[i] / hl * mn[i] - dt / hl * (F1[q + 1] - F1[q]);
  }
  return true;
}

// dT/dW of block_update at the values Wr, Wm of the iterate (row 2q + c: component c of cell lo + q; column
// likewise), by forward-mode dual numbers, eight unknowns at a time: exact up to rounding (the boundary solve's
// Newton iteration, carried on dual numbers, gives its converged root's derivative).
bool block_jacobian(const Fluid& Fl, const orc_opts& o, double tau, const std::vector<int>& ph,
                    const std::vector<Face<double>>& f, int lo, int hi, const std::vector<double>& wn,
                    const std::vector<double>& rn, const std::vector<double>& mn, const double FL[2],
                    const double FR[2], double dt, const std::vector<double>& Wr, const std::vector<double>& Wm,
                    std::vector<std::vector<double>>& dT) {
  typedef orcdual::Dual<8> DJ;
  const int n2 = 2 * (hi - lo + 1);
  std::vector<DJ> Dr(Wr.size()), Dm(Wm.size()), out(n2);
  for (int c0 = 0; c0 < n2; c0 += 8) {
    for (size_t i = 0; i < Wr.size(); ++i) {
      Dr[i] = DJ(Wr[i]);
      Dm[i] = DJ(Wm[i]);
    }
    for (int j = c0; j < std::min(n2, c0 + 8); ++j) {
      const int i = lo + j / 2;
      if (j % 2 == 0)
        Dr[i].d[j - c0] = 1.0;
      else
        Dm[i].d[j - c0] = 1.0;
    }
    if (!block_update(Fl, o, tau, ph, f, lo, hi, wn, rn, mn, FL, FR, dt, Dr, Dm, out)) return false;
    for (int r = 0; r < n2; ++r)
      for (int j = c0; j < std::min(n2, c0 + 8); ++j) dT[r][j] = out[r].d[j - c0];
  }
  return true;
}

// One time step of Algorithm 1 with the dual-time stepping of Algorithm 2 on every block,
// including the moving-grid width updates (Eq. godunov_meth:nonunif) and grid management.
// t_end > 0 clips the step to land on t_end.
// Solve A x = b for the augmented n x (n+1) matrix [A | b] in place by Gaussian elimination with partial
// pivoting (pivots chosen on values); the solution replaces column n. False if a pivot is zero.
template <class T>
bool gauss_solve(std::vector<std::vector<T>>& A, int n) {
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(val(A[r][c])) > std::fabs(val(A[p][c]))) p = r;
    if (!(std::fabs(val(A[p][c])) > 0.0)) return false;
    std::swap(A[c], A[p]);
    for (int r = c + 1; r < n; ++r) {
      T f = A[r][c] / A[c][c];
      for (int k = c; k <= n; ++k) A[r][k] = A[r][k] - f * A[c][k];
    }
  }
  for (int c = n - 1; c >= 0; --c) {
    T sum = A[c][n];
    for (int k = c + 1; k < n; ++k) sum = sum - A[c][k] * A[k][n];
    A[c][n] = sum / A[c][c];
  }
  return true;
}

template <class T>
void step_instance(const Fluid& F, const orc_opts& o, Inst<T>& I, double t_end) {
  if (I.status != ORC_OK) return;
  // (1) time step from the CFL condition, Eq. cfl_cond:unif, with the regular width h.
  //     Reading: S_max is taken over all cells, the width is always the background h.
  T S = 0.0;
  for (int i = 0; i < I.M(); ++i) S = tmax(S, T(tfabs(T(I.m[i] / I.r[i])) + sound(F, I.ph[i])));
  T dt = o.cfl * I.h / S;
  bool clipped = false;
  if (t_end > 0.0 && val(t_end - I.t) <= val(dt)) {
    dt = t_end - I.t;
    clipped = true;
  }
  // (2) Grid management before the step (Sec. 2.3, Sec. 3.4): phase-boundary speeds at U^n predict
  //     the widths; a cell next to a phase boundary that would fall below max(alpha_min h, h_i/2)
  //     is merged with its neighbour across its fixed face (possible only within one phase).
  std::vector<T> hpred;  // predicted widths at t^{n+1} after the merges (Sec. 3.1: the model mesh is the mesh at t^{n+1})
  {
    int M = I.M();
    std::vector<T> wf(M + 1, T(0.0));
    for (int g = 1; g < M; ++g) {
      if (!I.f[g].pb) continue;
      PBResult<T> R = solve_face(F, o, I, I.ph[g - 1], I.r[g - 1], I.m[g - 1], I.ph[g], I.r[g], I.m[g]);
      if (!R.ok) {
        I.status = ORC_ERR_PB_NOCONV;
        return;
      }
      wf[g] = R.w;
    }
    std::vector<int> mark(M, 0);
    for (int i = 0; i < M; ++i) {
      if (!(I.f[i].pb || I.f[i + 1].pb)) continue;
      T hp = I.w[i] + (wf[i + 1] - wf[i]) * dt;
      if (val(hp) < std::max(o.alpha_min * I.h, 0.5 * val(I.w[i]))) mark[i] = 1;
    }
    for (int i = 0; i < I.M(); ++i) {
      if (!mark[i]) continue;
      bool left_fixed = (i > 0) && !I.f[i].pb;
      bool right_fixed = (i + 1 < I.M()) && !I.f[i + 1].pb;
      if (left_fixed) {
        merge_cells(I, i, i - 1);
        mark.erase(mark.begin() + i);
        mark[i - 1] = 0;
        --i;
      } else if (right_fixed) {
        merge_cells(I, i, i + 1);
        mark.erase(mark.begin() + i + 1);
        mark[i] = 0;
      } else {
        I.status = ORC_ERR_VANISH;  // a cell bounded by two phase boundaries would vanish
        return;
      }
    }
  }
  const int M = I.M();
  {
    // predicted widths on the merged grid: boundary speeds from U^n of the (possibly merged) cells
    hpred.assign(I.w.begin(), I.w.end());
    std::vector<T> wf(M + 1, T(0.0));
    for (int g = 1; g < M; ++g) {
      if (!I.f[g].pb) continue;
      PBResult<T> R = solve_face(F, o, I, I.ph[g - 1], I.r[g - 1], I.m[g - 1], I.ph[g], I.r[g], I.m[g]);
      if (!R.ok) {
        I.status = ORC_ERR_PB_NOCONV;
        return;
      }
      wf[g] = R.w;
    }
    for (int i = 0; i < M; ++i) hpred[i] = I.w[i] + (wf[i + 1] - wf[i]) * dt;
  }
  // (3) Implicit neighbourhoods (Sec. 3.2): at every phase boundary the smaller adjacent cell is the
  //     tiny cell k; {k-1, k, k+1} is treated implicitly. Overlapping neighbourhoods are joined.
  std::vector<int> blk(M, -1), tiny(M, 0);
  std::vector<std::pair<int, int>> blocks;
  for (int g = 1; g < M; ++g) {
    if (!I.f[g].pb) continue;
    int k = (val(I.w[g - 1]) < val(I.w[g])) ? g - 1 : g;
    tiny[k] = 1;
    int lo = std::max(k - 1, 0), hi = std::min(k + 1, M - 1);
    if (!blocks.empty() && lo <= blocks.back().second)
      blocks.back().second = std::max(blocks.back().second, hi);
    else
      blocks.push_back({lo, hi});
  }
  for (size_t b = 0; b < blocks.size(); ++b)
    for (int i = blocks[b].first; i <= blocks[b].second; ++i) blk[i] = (int)b;
  // (4) Phase creation (App. B) at same-phase faces between two explicit cells.
  std::vector<int> create(M + 1, 0);
  std::vector<CreateResult<T>> cres(M + 1);
  if (o.creation) {
    std::vector<int> det(M + 1, 0);
    for (int g = 1; g < M; ++g) {
      if (I.f[g].pb || blk[g - 1] >= 0 || blk[g] >= 0) continue;
      int P = I.ph[g];
      double ps = nopt_star(F.ph[P], val(I.r[g - 1]), val(I.m[g - 1] / I.r[g - 1]), val(I.r[g]),
                            val(I.m[g] / I.r[g]));
      det[g] = (P == LIQ) ? (ps < F.p_min) : (ps > F.p_tilde);
    }
    for (int g = 1; g < M; ++g) {
      if (!det[g] || det[g - 1]) continue;
      CreateResult<T> R = creation_solve(F, o, I.tau, I.ph[g], I.r[g - 1], I.m[g - 1], I.r[g], I.m[g]);
      I.newton += R.iters;
      if (!R.ok) {
        I.status = ORC_ERR_PB_NOCONV;
        return;
      }
      create[g] = 1;
      cres[g] = R;
    }
  }
  // (5) Algorithm 1, Step 1: fluxes from U^n at every face that is not inside a block, and the
  //     explicit update of every cell outside the blocks. Fl[g]/Fr[g] are the fluxes seen by the cell
  //     left/right of face g (they differ only at a creation face, Eq. flux:cavitation/nucleation).
  std::vector<T> Fl0(M + 1, T(0.0)), Fl1(M + 1, T(0.0)), Fr0(M + 1, T(0.0)), Fr1(M + 1, T(0.0));
  std::vector<T> wl(M + 1, T(0.0)), wr(M + 1, T(0.0));  // speed of face g seen from left/right cell
  for (int g = 0; g <= M; ++g) {
    T Fx[2];
    if (g == 0) {
      phys_flux(F.ph[I.ph[0]], I.r[0], I.m[0], Fx);  // transmissive boundary (Reading: ghost = cell)
    } else if (g == M) {
      phys_flux(F.ph[I.ph[M - 1]], I.r[M - 1], I.m[M - 1], Fx);
    } else if (blk[g - 1] >= 0 && blk[g - 1] == blk[g]) {
      continue;  // interior face of a block: computed in Algorithm 2
    } else if (create[g]) {
      const CreateResult<T>& R = cres[g];
      // Eq. flux:cavitation / flux:nucleation with each boundary's own mass flux
      Fl0[g] = -R.z1;
      Fl1[g] = -R.z1 * R.uC + R.pC;
      Fr0[g] = -R.z2;
      Fr1[g] = -R.z2 * R.uC + R.pC;
      wl[g] = R.w1;
      wr[g] = R.w2;
      continue;
    } else {
      hll(F.ph[I.ph[g]], I.r[g - 1], I.m[g - 1], I.r[g], I.m[g], Fx);
    }
    Fl0[g] = Fr0[g] = Fx[0];
    Fl1[g] = Fr1[g] = Fx[1];
  }
  std::vector<T> rn = I.r, mn = I.m, wn = I.w;  // U^n and h^n
  for (int i = 0; i < M; ++i) {
    if (blk[i] >= 0) continue;
    T hnp1 = wn[i] + (wl[i + 1] - wr[i]) * dt;
    I.r[i] = (wn[i] * rn[i] - dt * (Fl0[i + 1] - Fr0[i])) / hnp1;
    I.m[i] = (wn[i] * mn[i] - dt * (Fl1[i + 1] - Fr1[i])) / hnp1;
    I.w[i] = hnp1;
  }
  // (6) Algorithm 1, Step 2 = Algorithm 2 on each block, with the local pseudo time steps of
  //     Eq. dual time tau diff and the width iterates of Sec. 3.4.
  std::vector<T> xpb_new(M + 1, T(0.0));
  std::vector<int> pb_moved(M + 1, 0);
  double worst_defect = 0.0;
  for (size_t b = 0; b < blocks.size(); ++b) {
    int lo = blocks[b].first, hi = blocks[b].second;
    T FL[2] = {Fr0[lo], Fr1[lo]};        // F_left  = flux at face lo from U^n
    T FR[2] = {Fl0[hi + 1], Fl1[hi + 1]}; // F_right = flux at face hi+1 from U^n
    std::vector<T> Wr = rn, Wm = mn;      // dual-time iterate, indexed like the cells
    std::vector<T> theta(M, T(0.0));
    // Delta tau_i = theta_i dt with theta_i <= h_i/h for stability (Sec. 3.3). Reading: the widths are
    // those of the mesh at t^{n+1} (Sec. 3.1 treats the model mesh as the mesh at t^{n+1}), predicted
    // with the boundary speeds at U^n.
    for (int i = lo; i <= hi; ++i) theta[i] = tmin(T(o.theta_nb), T(hpred[i] / I.h));
    std::vector<T> Fc0(M + 1), Fc1(M + 1), wc(M + 1, T(0.0)), hl(M);
    auto fluxes = [&](const std::vector<T>& Ar, const std::vector<T>& Am) -> bool {
      Fc0[lo] = FL[0];
      Fc1[lo] = FL[1];
      Fc0[hi + 1] = FR[0];
      Fc1[hi + 1] = FR[1];
      wc[lo] = 0.0;
      wc[hi + 1] = 0.0;
      for (int g = lo + 1; g <= hi; ++g) {
        T Fx[2], wx;
        if (!block_face_flux(F, o, I, g, Ar, Am, Fx, &wx)) return false;
        Fc0[g] = Fx[0];
        Fc1[g] = Fx[1];
        wc[g] = wx;
      }
      for (int i = lo; i <= hi; ++i) hl[i] = wn[i] + (wc[i + 1] - wc[i]) * dt;
      for (int i = lo; i <= hi; ++i)
        if (!(val(hl[i]) > 0.0)) return false;
      return true;
    };
    int l = 0;
    bool stop = false;
    if (o.block_solver == 1) {
      // Newton on the block's implicit system R(W) = W - T(W), T the update of Part 1 with fluxes and widths
      // at W, whose fixed point is the dual-time limit. The Sec. 4 residual of an iterate W is
      // |R(W)| / (dt max(|W|, 1)) component by component (the pseudo step moves W by theta R / (1 + theta)),
      // so the same test stops Newton. Jacobian dR/dW = I - dT/dW by forward-mode dual numbers at the values
      // of the iterate (block_jacobian), linear solve with partial pivoting.
      const int n2 = 2 * (hi - lo + 1);
      std::vector<T> Tv(n2);
      auto target = [&](const std::vector<T>& Ar, const std::vector<T>& Am, std::vector<T>& out) -> bool {
        if (!fluxes(Ar, Am)) return false;
        for (int i = lo; i <= hi; ++i) {
          out[2 * (i - lo)] = wn[i] / hl[i] * rn[i] - dt / hl[i] * (Fc0[i + 1] - Fc0[i]);
          out[2 * (i - lo) + 1] = wn[i] / hl[i] * mn[i] - dt / hl[i] * (Fc1[i + 1] - Fc1[i]);
        }
        return true;
      };
      // plain values of everything the Jacobian depends on besides the iterate
      std::vector<Face<double>> fv(I.f.size());
      for (size_t g = 0; g < I.f.size(); ++g) fv[g] = Face<double>{I.f[g].pb, I.f[g].j, val(I.f[g].x)};
      std::vector<double> wnv(M), rnv(M), mnv(M), Wrv(M), Wmv(M);
      for (int i = 0; i < M; ++i) {
        wnv[i] = val(wn[i]);
        rnv[i] = val(rn[i]);
        mnv[i] = val(mn[i]);
      }
      const double FLv[2] = {val(FL[0]), val(FL[1])}, FRv[2] = {val(FR[0]), val(FR[1])};
      std::vector<std::vector<double>> dT(n2, std::vector<double>(n2, 0.0));
      double corr_prev = std::numeric_limits<double>::infinity();
      for (l = 0; l < o.l_max; ++l) {
        if (!target(Wr, Wm, Tv)) {
          I.status = ORC_ERR_VANISH;
          return;
        }
        double res_nb = 0.0, res_k = 0.0;
        const double dtv = val(dt);
        for (int i = lo; i <= hi; ++i) {
          double e0 = std::fabs(val(Wr[i]) - val(Tv[2 * (i - lo)])) / (dtv * std::max(std::fabs(val(Wr[i])), 1.0));
          double e1 = std::fabs(val(Wm[i]) - val(Tv[2 * (i - lo) + 1])) / (dtv * std::max(std::fabs(val(Wm[i])), 1.0));
          double res = std::max(e0, e1);
          if (o.res_mode == 1) res *= dtv;
          if (tiny[i])
            res_k = std::max(res_k, res);
          else
            res_nb = std::max(res_nb, res);
        }
        if (res_nb < o.tol_nb && res_k < o.tol_k) {
          stop = true;
          break;
        }
        for (int i = 0; i < M; ++i) {
          Wrv[i] = val(Wr[i]);
          Wmv[i] = val(Wm[i]);
        }
        if (!block_jacobian(F, o, val(I.tau), I.ph, fv, lo, hi, wnv, rnv, mnv, FLv, FRv, dtv, Wrv, Wmv, dT)) {
          I.status = ORC_ERR_VANISH;
          return;
        }
        std::vector<std::vector<T>> A(n2, std::vector<T>(n2 + 1));  // [dR/dW | -R]
        for (int r = 0; r < n2; ++r) {
          for (int j = 0; j < n2; ++j) A[r][j] = T((r == j ? 1.0 : 0.0) - dT[r][j]);
          A[r][n2] = Tv[r] - ((r % 2 == 0) ? Wr[lo + r / 2] : Wm[lo + r / 2]);
        }
        if (!gauss_solve(A, n2)) {
          I.status = ORC_ERR_PB_NOCONV;
          return;
        }
        // the floor rounding puts under the residual (a tiny cell's update amplifies a one-ulp change of W by
        // about 1/alpha): with c = max |correction| / max(|W|, 1), stop as at l_max when c <= 1e-14 (the
        // correction is below the iterate's own rounding) or when 1e-10 >= c > c_prev / 2 (the corrections no
        // longer contract, which quadratic convergence rules out; c_prev of the first step is infinite)
        double corr = 0.0;
        for (int r = 0; r < n2; ++r) {
          const double w = std::fabs(val((r % 2 == 0) ? Wr[lo + r / 2] : Wm[lo + r / 2]));
          corr = std::max(corr, std::fabs(val(A[r][n2])) / std::max(w, 1.0));
        }
        const bool at_floor = corr <= 1e-14 || (corr <= 1e-10 && corr > 0.5 * corr_prev);
        corr_prev = corr;
        for (int r = 0; r < n2; ++r) {
          if (r % 2 == 0)
            Wr[lo + r / 2] = Wr[lo + r / 2] + A[r][n2];
          else
            Wm[lo + r / 2] = Wm[lo + r / 2] + A[r][n2];
        }
        if (at_floor) {
          ++l;
          break;
        }
      }
    } else {
      for (l = 0; l < o.l_max && !stop; ++l) {
        // Part 1 (a): fluxes at the current iterate, (b) pseudo-time update.
        if (!fluxes(Wr, Wm)) {
          I.status = ORC_ERR_VANISH;
          return;
        }
        double res_nb = 0.0, res_k = 0.0;
        std::vector<T> Nr = Wr, Nm = Wm;
        for (int i = lo; i <= hi; ++i) {
          T th = theta[i];
          T tr = wn[i] / hl[i] * rn[i] - dt / hl[i] * (Fc0[i + 1] - Fc0[i]);
          T tm = wn[i] / hl[i] * mn[i] - dt / hl[i] * (Fc1[i + 1] - Fc1[i]);
          Nr[i] = (Wr[i] + th * tr) / (1.0 + th);
          Nm[i] = (Wm[i] + th * tm) / (1.0 + th);
          // residual of Sec. 4: ||(1 + dtau/dt)(W^{l+1} - W^l) / (dtau max(|W^l|, 1))||_inf
          double thv = val(th), dtv = val(dt);
          double dtau = thv * dtv;
          double e0 = (1.0 + thv) * std::fabs(val(Nr[i]) - val(Wr[i])) / (dtau * std::max(std::fabs(val(Wr[i])), 1.0));
          double e1 = (1.0 + thv) * std::fabs(val(Nm[i]) - val(Wm[i])) / (dtau * std::max(std::fabs(val(Wm[i])), 1.0));
          double res = std::max(e0, e1);
          if (o.res_mode == 1) res *= dtv;
          if (tiny[i])
            res_k = std::max(res_k, res);
          else
            res_nb = std::max(res_nb, res);
        }
        Wr = Nr;
        Wm = Nm;
        if (res_nb < o.tol_nb && res_k < o.tol_k) stop = true;
      }
    }
    int iters = l;
    if (!stop) I.maxiter++;
    I.dts_iters += iters;
    I.dts_max = std::max<long long>(I.dts_max, iters);
    // Part 2: fluxes and widths at U^{n,*}, conservative update with F_left/F_right from U^n.
    if (!fluxes(Wr, Wm)) {
      I.status = ORC_ERR_VANISH;
      return;
    }
    for (int i = lo; i <= hi; ++i) {
      // fixed-point defect of the implicit system at U^{n,*} (diagnostic)
      T gr = (wn[i] * rn[i] - dt * (Fc0[i + 1] - Fc0[i])) / hl[i];
      T gm = (wn[i] * mn[i] - dt * (Fc1[i + 1] - Fc1[i])) / hl[i];
      worst_defect = std::max(worst_defect, std::fabs(val(gr) - val(Wr[i])) / std::max(std::fabs(val(Wr[i])), 1.0));
      worst_defect = std::max(worst_defect, std::fabs(val(gm) - val(Wm[i])) / std::max(std::fabs(val(Wm[i])), 1.0));
      I.r[i] = gr;
      I.m[i] = gm;
      I.w[i] = hl[i];
    }
    for (int g = lo + 1; g <= hi; ++g)
      if (I.f[g].pb) {
        pb_moved[g] = 1;
        xpb_new[g] = I.f[g].x + wc[g] * dt;  // the grid follows the phase boundary (Sec. 2.3)
      }
  }
  I.last_implicit_res = worst_defect;
  for (int g = 1; g < M; ++g)
    if (pb_moved[g]) I.f[g].x = xpb_new[g];
  // (7) Insert created cells (App. B): width (w_right - w_left) dt between the two new boundaries.
  for (int g = M - 1; g >= 1; --g) {
    if (!create[g]) continue;
    const CreateResult<T>& R = cres[g];
    T xg = I.face_x(g);
    Face<T> f1{1, 0, xg + R.w1 * dt}, f2{1, 0, xg + R.w2 * dt};
    I.f[g] = f1;
    I.f.insert(I.f.begin() + g + 1, f2);
    I.w.insert(I.w.begin() + g, (R.w2 - R.w1) * dt);
    I.r.insert(I.r.begin() + g, R.rhoC);
    I.m.insert(I.m.begin() + g, R.rhoC * R.uC);
    I.ph.insert(I.ph.begin() + g, 1 - I.ph[g]);
    I.creations++;
  }
  // (8) Split cells next to a phase boundary that grew beyond split_ratio*h (Sec. 3.4).
  //     Reading: the split keeps every fixed face on the background lattice: a cell with a fixed
  //     left (right) face gives up its first (last) lattice cell; a cell between two phase
  //     boundaries is cut at the lattice face nearest its midpoint. Both parts keep the state.
  for (int i = 0; i < I.M(); ++i) {
    bool lpb = I.f[i].pb, rpb = I.f[i + 1].pb;
    if (!(lpb || rpb) || !(val(I.w[i]) > o.split_ratio * I.h)) continue;
    T w1, w2;
    long jc;
    if (!lpb) {
      jc = I.f[i].j + 1;
      w1 = I.h;
      w2 = I.w[i] - I.h;
    } else if (!rpb) {
      jc = I.f[i + 1].j - 1;
      w2 = I.h;
      w1 = I.w[i] - I.h;
    } else {
      double xm = 0.5 * (val(I.f[i].x) + val(I.f[i + 1].x));
      jc = std::lround((xm - I.xL) / I.h);
      w1 = (I.xL + (double)jc * I.h) - I.f[i].x;
      w2 = I.w[i] - w1;
      if (!(val(w1) > 0.0) || !(val(w2) > 0.0)) continue;
    }
    Face<T> fc{0, jc, T(0.0)};
    I.f.insert(I.f.begin() + i + 1, fc);
    I.w[i] = w1;
    I.w.insert(I.w.begin() + i + 1, w2);
    I.r.insert(I.r.begin() + i + 1, I.r[i]);
    I.m.insert(I.m.begin() + i + 1, I.m[i]);
    I.ph.insert(I.ph.begin() + i + 1, I.ph[i]);
    I.splits++;
    ++i;  // the new cell is not examined again in this step
  }
  I.t = clipped ? T(t_end) : T(I.t + dt);
  I.steps++;
  if (!finite_state(I)) I.status = ORC_ERR_NONPHYSICAL;
}

// Fully explicit moving-grid scheme used as a brute-force reference: every cell, including the
// phase-boundary cells, is updated by Eq. godunov_meth:nonunif with fluxes from U^n, and the time
// step obeys the CFL condition of the smallest cell.
void explicit_step(const Fluid& F, const orc_opts& o, Inst<double>& I, double t_end) {
  if (I.status != ORC_OK) return;
  int M = I.M();
  double S = 0.0, hmin = I.h;
  for (int i = 0; i < M; ++i) {
    S = std::max(S, std::fabs(I.m[i] / I.r[i]) + sound(F, I.ph[i]));
    hmin = std::min(hmin, I.w[i]);
  }
  // A cell shrinking towards zero would drive this step to zero: stop the instance instead.
  if (hmin < o.alpha_min * I.h) {
    I.status = ORC_ERR_VANISH;
    return;
  }
  double dt = o.cfl * hmin / S;
  bool clipped = false;
  if (t_end - I.t <= dt) {
    dt = t_end - I.t;
    clipped = true;
  }
  std::vector<double> F0(M + 1), F1(M + 1), wf(M + 1, 0.0);
  for (int g = 0; g <= M; ++g) {
    double Fx[2];
    if (g == 0)
      phys_flux(F.ph[I.ph[0]], I.r[0], I.m[0], Fx);
    else if (g == M)
      phys_flux(F.ph[I.ph[M - 1]], I.r[M - 1], I.m[M - 1], Fx);
    else if (I.f[g].pb) {
      PBResult<double> R = solve_face(F, o, I, I.ph[g - 1], I.r[g - 1], I.m[g - 1], I.ph[g], I.r[g], I.m[g]);
      if (!R.ok) {
        I.status = ORC_ERR_PB_NOCONV;
        return;
      }
      Fx[0] = R.F[0];
      Fx[1] = R.F[1];
      wf[g] = R.w;
    } else
      hll(F.ph[I.ph[g]], I.r[g - 1], I.m[g - 1], I.r[g], I.m[g], Fx);
    F0[g] = Fx[0];
    F1[g] = Fx[1];
  }
  for (int i = 0; i < M; ++i) {
    double hn = I.w[i], hnp1 = hn + (wf[i + 1] - wf[i]) * dt;
    if (!(hnp1 > 0.0)) {
      I.status = ORC_ERR_VANISH;
      return;
    }
    I.r[i] = (hn * I.r[i] - dt * (F0[i + 1] - F0[i])) / hnp1;
    I.m[i] = (hn * I.m[i] - dt * (F1[i + 1] - F1[i])) / hnp1;
    I.w[i] = hnp1;
  }
  for (int g = 1; g < M; ++g)
    if (I.f[g].pb) I.f[g].x += wf[g] * dt;
  I.t = clipped ? t_end : I.t + dt;
  I.steps++;
  if (!finite_state(I)) I.status = ORC_ERR_NONPHYSICAL;
}

struct Ctx {
  Fluid F;
  orc_opts o;
  std::vector<Inst<double>> inst;
  // tangent-linear results of the last orc_tangent call: per instance, per direction, the final
  // (width, rho, m) derivatives of every cell
  std::vector<std::vector<double>> tan_w, tan_r, tan_m;
  int tan_dirs = 0;
};

template <class Fn>
void parallel_for(int n, int n_threads, Fn fn) {
  if (n_threads <= 1 || n <= 1) {
    for (int i = 0; i < n; ++i) fn(i);
    return;
  }
  std::atomic<int> next(0);
  std::vector<std::thread> th;
  int nt = std::min(n_threads, n);
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&]() {
      for (;;) {
        int i = next.fetch_add(1);
        if (i >= n) break;
        fn(i);
      }
    });
  for (auto& x : th) x.join();
}

}  // namespace

// ---------------------------------------------------------------- C interface

extern "C" {

void orc_default_opts(orc_opts* o) {
  o->cfl = 0.5;
  o->theta_nb = 0.9;
  o->tol_nb = 1e-3;
  o->tol_k = 1e-1;
  o->res_mode = 0;
  o->l_max = 10000;
  o->newton_tol = 1e-12;
  o->newton_itmax = 50;
  o->alpha_min = 1e-8;
  o->split_ratio = 2.0;
  o->creation = 0;
  o->block_solver = 0;
}

void orc_hll(const orc_fluid* fl, int ph, double rl, double ml, double rr, double mr, double F[2]) {
  Fluid Fd = make_fluid(fl);
  hll(Fd.ph[ph], rl, ml, rr, mr, F);
}

void orc_pb_system(const orc_fluid* fl, double tau, int phl, double rl, double ul, int phr, double rr, double ur,
                   double pls, double prs, double out[7]) {
  Fluid Fd = make_fluid(fl);
  PBSys<double> S;
  bool ok = pb_eval(Fd, tau, phl, rl, ul, phr, rr, ur, pls, prs, &S);
  if (!ok) {
    for (int i = 0; i < 7; ++i) out[i] = NAN;
    return;
  }
  out[0] = S.G[0];
  out[1] = S.G[1];
  out[2] = S.z;
  out[3] = S.J[0][0];
  out[4] = S.J[0][1];
  out[5] = S.J[1][0];
  out[6] = S.J[1][1];
}

int orc_pb_solve(const orc_fluid* fl, const orc_opts* o, double tau, int phl, double rl, double ul, int phr,
                 double rr, double ur, double out[11]) {
  Fluid Fd = make_fluid(fl);
  PBResult<double> R = pb_solve(Fd, *o, tau, phl, rl, rl * ul, phr, rr, rr * ur);
  out[10] = R.iters;
  if (!R.ok) return ORC_ERR_PB_NOCONV;
  double v[10] = {R.pl, R.pr, R.rl, R.rr, R.ul, R.ur, R.z, R.w, R.F[0], R.F[1]};
  for (int i = 0; i < 10; ++i) out[i] = v[i];
  return ORC_OK;
}

double orc_nopt_star(const orc_fluid* fl, int ph, double rl, double ul, double rr, double ur) {
  Fluid Fd = make_fluid(fl);
  return nopt_star(Fd.ph[ph], rl, ul, rr, ur);
}

int orc_creation_solve(const orc_fluid* fl, const orc_opts* o, double tau, int ph, double rl, double ul, double rr,
                       double ur, double out[12]) {
  Fluid Fd = make_fluid(fl);
  CreateResult<double> R = creation_solve(Fd, *o, tau, ph, rl, rl * ul, rr, rr * ur);
  out[11] = R.iters;
  if (!R.ok) return ORC_ERR_PB_NOCONV;
  double v[11] = {R.pPl, R.pC, R.pPr, R.rhoC, R.uC, R.z1, R.z2, R.w1, R.w2, R.uPl, R.uPr};
  for (int i = 0; i < 11; ++i) out[i] = v[i];
  return ORC_OK;
}

int orc_exact_sample(const orc_fluid* fl, const orc_opts* o, double tau, int phl, double rl, double ul, int phr,
                     double rr, double ur, int n, const double* xi, double* rho, double* u, int* ph) {
  Fluid Fd = make_fluid(fl);
  PBResult<double> R = pb_solve(Fd, *o, tau, phl, rl, rl * ul, phr, rr, rr * ur);
  if (!R.ok) return ORC_ERR_PB_NOCONV;
  const Phase& El = Fd.ph[phl];
  const Phase& Er = Fd.ph[phr];
  double pl = pressure(El, rl), pr = pressure(Er, rr);
  for (int i = 0; i < n; ++i) {
    double s = xi[i];
    if (s < R.w) {  // left of the phase boundary: left outer wave, then the left star state
      ph[i] = phl;
      if (R.pl > pl) {  // shock with mass flux Q, speed u_l - Q v_l
        double Q = std::sqrt((R.pl - pl) / (1.0 / rl - 1.0 / R.rl));
        double S = ul - Q / rl;
        if (s < S) {
          rho[i] = rl;
          u[i] = ul;
        } else {
          rho[i] = R.rl;
          u[i] = R.ul;
        }
      } else {  // rarefaction: u - a = xi inside the fan, u + a ln rho constant across it
        double head = ul - El.a, tail = R.ul - El.a;
        if (s < head) {
          rho[i] = rl;
          u[i] = ul;
        } else if (s > tail) {
          rho[i] = R.rl;
          u[i] = R.ul;
        } else {
          u[i] = s + El.a;
          rho[i] = rl * std::exp((ul - u[i]) / El.a);
        }
      }
    } else {
      ph[i] = phr;
      if (R.pr > pr) {
        double Q = std::sqrt((R.pr - pr) / (1.0 / rr - 1.0 / R.rr));
        double S = ur + Q / rr;
        if (s > S) {
          rho[i] = rr;
          u[i] = ur;
        } else {
          rho[i] = R.rr;
          u[i] = R.ur;
        }
      } else {  // u + a = xi inside the fan, u - a ln rho constant across it
        double head = ur + Er.a, tail = R.ur + Er.a;
        if (s > head) {
          rho[i] = rr;
          u[i] = ur;
        } else if (s < tail) {
          rho[i] = R.rr;
          u[i] = R.ur;
        } else {
          u[i] = s - Er.a;
          rho[i] = rr * std::exp((u[i] - ur) / Er.a);
        }
      }
    }
  }
  return ORC_OK;
}

void* orc_create(int n_inst, const int* n_lattice, const double* x_left, const double* x_right, const double* tau,
                 const orc_fluid* fl, const orc_opts* o) {
  if (n_inst <= 0) return nullptr;
  Ctx* C = new Ctx();
  C->F = make_fluid(fl);
  if (o)
    C->o = *o;
  else
    orc_default_opts(&C->o);
  C->inst.resize(n_inst);
  for (int i = 0; i < n_inst; ++i) {
    Inst<double>& I = C->inst[i];
    I.N = n_lattice[i];
    I.xL = x_left[i];
    I.xR = x_right[i];
    I.h = (x_right[i] - x_left[i]) / (double)n_lattice[i];
    I.tau = tau[i];
  }
  return C;
}

void orc_destroy(void* H) { delete (Ctx*)H; }

int orc_set_states(void* H, const int* off, const double* widths, const double* rho, const double* m,
                   const unsigned char* phase, double t0) {
  Ctx* C = (Ctx*)H;
  int rc = ORC_OK;
  for (size_t k = 0; k < C->inst.size(); ++k) {
    Inst<double>& I = C->inst[k];
    int a = off[k], b = off[k + 1];
    int M = b - a;
    I.f.assign(M + 1, Face<double>{0, 0, 0.0});
    I.w.assign(widths + a, widths + b);
    I.r.assign(rho + a, rho + b);
    I.m.assign(m + a, m + b);
    I.ph.resize(M);
    for (int i = 0; i < M; ++i) I.ph[i] = phase[a + i];
    I.t = t0;
    I.status = ORC_OK;
    I.steps = I.dts_iters = I.dts_max = I.newton = I.merges = I.splits = I.creations = I.maxiter = I.pb_solves = 0;
    // Face positions: widths accumulate from the last fixed face, which sits on the lattice;
    // a face between cells of one phase must land on a lattice face (to 1e-9 h).
    long jfix = 0;
    double part = 0.0;
    I.f[0] = Face<double>{0, 0, 0.0};
    for (int i = 0; i < M; ++i) {
      part += I.w[i];
      if (i + 1 < M && I.ph[i + 1] != I.ph[i]) {
        I.f[i + 1] = Face<double>{1, 0, I.xL + (double)jfix * I.h + part};
      } else {
        double units = part / I.h;
        long j = jfix + std::lround(units);
        if (std::fabs(units - std::round(units)) > 1e-9 || j < 0 || j > I.N || j <= jfix) {
          I.status = ORC_ERR_ARG;
          rc = ORC_ERR_ARG;
        }
        I.f[i + 1] = Face<double>{0, j, 0.0};
        jfix = j;
        part = 0.0;
      }
    }
    if (I.f[M].pb || I.f[M].j != I.N) {
      I.status = ORC_ERR_ARG;
      rc = ORC_ERR_ARG;
    }
    // cells with two fixed faces are lattice cells: width (j_r - j_l) h exactly
    for (int i = 0; i < M; ++i)
      if (!I.f[i].pb && !I.f[i + 1].pb) I.w[i] = (double)(I.f[i + 1].j - I.f[i].j) * I.h;
  }
  return rc;
}

int orc_n_cells(void* H, int* counts) {
  Ctx* C = (Ctx*)H;
  for (size_t k = 0; k < C->inst.size(); ++k) counts[k] = C->inst[k].M();
  return ORC_OK;
}

int orc_get_states(void* H, int* off, double* widths, double* rho, double* m, unsigned char* phase, double* t,
                   int* status) {
  Ctx* C = (Ctx*)H;
  int o = 0;
  for (size_t k = 0; k < C->inst.size(); ++k) {
    const Inst<double>& I = C->inst[k];
    off[k] = o;
    for (int i = 0; i < I.M(); ++i, ++o) {
      widths[o] = I.w[i];
      rho[o] = I.r[i];
      m[o] = I.m[i];
      phase[o] = (unsigned char)I.ph[i];
    }
    t[k] = I.t;
    status[k] = I.status;
  }
  off[C->inst.size()] = o;
  return ORC_OK;
}

int orc_get_pbs(void* H, int* off, double* x) {
  Ctx* C = (Ctx*)H;
  int o = 0;
  for (size_t k = 0; k < C->inst.size(); ++k) {
    const Inst<double>& I = C->inst[k];
    off[k] = o;
    for (int g = 1; g < I.M(); ++g)
      if (I.f[g].pb) x[o++] = I.f[g].x;
  }
  off[C->inst.size()] = o;
  return ORC_OK;
}

int orc_get_stats(void* H, long long* s) {
  Ctx* C = (Ctx*)H;
  for (size_t k = 0; k < C->inst.size(); ++k) {
    const Inst<double>& I = C->inst[k];
    long long v[10] = {I.steps, I.dts_iters, I.dts_max, I.newton, I.merges, I.splits, I.creations, I.maxiter,
                       I.pb_solves, 0};
    for (int j = 0; j < 10; ++j) s[10 * k + j] = v[j];
  }
  return ORC_OK;
}

int orc_run_to(void* H, double t_end, int n_threads) {
  Ctx* C = (Ctx*)H;
  parallel_for((int)C->inst.size(), n_threads, [&](int k) {
    Inst<double>& I = C->inst[k];
    while (I.status == ORC_OK && I.t < t_end) step_instance(C->F, C->o, I, t_end);
  });
  return ORC_OK;
}

int orc_step(void* H, int n_steps, int n_threads) {
  Ctx* C = (Ctx*)H;
  parallel_for((int)C->inst.size(), n_threads, [&](int k) {
    Inst<double>& I = C->inst[k];
    for (int s = 0; s < n_steps && I.status == ORC_OK; ++s) step_instance(C->F, C->o, I, -1.0);
  });
  return ORC_OK;
}

int orc_explicit_run_to(void* H, double t_end, int n_threads) {
  Ctx* C = (Ctx*)H;
  parallel_for((int)C->inst.size(), n_threads, [&](int k) {
    Inst<double>& I = C->inst[k];
    while (I.status == ORC_OK && I.t < t_end) explicit_step(C->F, C->o, I, t_end);
  });
  return ORC_OK;
}

double orc_last_implicit_residual(void* H, int inst) { return ((Ctx*)H)->inst[inst].last_implicit_res; }

// Tangent-linear mode: every instance is re-run from its current states with K-direction dual
// numbers; the value parts reproduce the plain run bit for bit, the derivative parts are the
// directional derivatives of the computed final states (decisions frozen).
typedef orcdual::Dual<8> D8;

int orc_tangent(void* H, int n_dir, const double* seed_w, const double* seed_rho, const double* seed_m,
                const double* seed_tau, int n_prog, const int* prog_kind, const double* prog_arg, int n_threads) {
  Ctx* C = (Ctx*)H;
  const int n = (int)C->inst.size();
  if (n_dir < 1 || n_prog < 0) return ORC_ERR_ARG;
  std::vector<long> off(n + 1, 0);
  for (int k = 0; k < n; ++k) off[k + 1] = off[k] + C->inst[k].M();
  const long tot = off[n];
  std::vector<Inst<double>> start = C->inst;
  std::vector<Inst<double>> final_state(n);
  C->tan_w.assign(n, {});
  C->tan_r.assign(n, {});
  C->tan_m.assign(n, {});
  C->tan_dirs = n_dir;
  for (int d0 = 0; d0 < n_dir; d0 += 8) {
    parallel_for(n, n_threads, [&](int k) {
      const Inst<double>& S = start[k];
      Inst<D8> I;
      I.N = S.N;
      I.xL = S.xL;
      I.xR = S.xR;
      I.h = S.h;
      I.tau = S.tau;
      I.t = S.t;
      I.status = S.status;
      I.ph = S.ph;
      const int M = S.M();
      I.w.resize(M);
      I.r.resize(M);
      I.m.resize(M);
      I.f.resize(M + 1);
      for (int i = 0; i < M; ++i) {
        I.w[i] = S.w[i];
        I.r[i] = S.r[i];
        I.m[i] = S.m[i];
      }
      for (int i = 0; i <= M; ++i) I.f[i] = Face<D8>{S.f[i].pb, S.f[i].j, D8(S.f[i].x)};
      for (int q = 0; q < 8 && d0 + q < n_dir; ++q) {
        const long base = (long)(d0 + q) * tot + off[k];
        if (seed_tau) I.tau.d[q] = seed_tau[(long)(d0 + q) * n + k];
        // a phase boundary sits at the last fixed face plus the widths since it: its position moves
        // with the seeded widths
        double part = 0.0;
        for (int i = 0; i < M; ++i) {
          if (seed_w) I.w[i].d[q] = seed_w[base + i];
          if (seed_rho) I.r[i].d[q] = seed_rho[base + i];
          if (seed_m) I.m[i].d[q] = seed_m[base + i];
          part += seed_w ? seed_w[base + i] : 0.0;
          if (I.f[i + 1].pb)
            I.f[i + 1].x.d[q] = part;
          else
            part = 0.0;
        }
      }
      for (int p = 0; p < n_prog; ++p) {
        if (prog_kind[p] == 0) {
          for (long s = 0; s < (long)prog_arg[p] && I.status == ORC_OK; ++s) step_instance(C->F, C->o, I, -1.0);
        } else {
          while (I.status == ORC_OK && val(I.t) < prog_arg[p]) step_instance(C->F, C->o, I, prog_arg[p]);
        }
      }
      const int Mf = I.M();
      if (d0 == 0) {
        C->tan_w[k].assign((size_t)n_dir * Mf, 0.0);
        C->tan_r[k].assign((size_t)n_dir * Mf, 0.0);
        C->tan_m[k].assign((size_t)n_dir * Mf, 0.0);
        Inst<double>& O = final_state[k];
        O = S;
        O.w.resize(Mf);
        O.r.resize(Mf);
        O.m.resize(Mf);
        O.f.resize(Mf + 1);
        for (int i = 0; i < Mf; ++i) {
          O.w[i] = I.w[i].v;
          O.r[i] = I.r[i].v;
          O.m[i] = I.m[i].v;
        }
        for (int i = 0; i <= Mf; ++i) O.f[i] = Face<double>{I.f[i].pb, I.f[i].j, I.f[i].x.v};
        O.ph = I.ph;
        O.t = I.t.v;
        O.status = I.status;
        O.steps = S.steps + I.steps;
        O.dts_iters = S.dts_iters + I.dts_iters;
        O.dts_max = std::max(S.dts_max, I.dts_max);
        O.newton = S.newton + I.newton;
        O.merges = S.merges + I.merges;
        O.splits = S.splits + I.splits;
        O.creations = S.creations + I.creations;
        O.maxiter = S.maxiter + I.maxiter;
        O.pb_solves = S.pb_solves + I.pb_solves;
        O.last_implicit_res = I.last_implicit_res;
      }
      for (int q = 0; q < 8 && d0 + q < n_dir; ++q)
        for (int i = 0; i < Mf; ++i) {
          C->tan_w[k][(size_t)(d0 + q) * Mf + i] = I.w[i].d[q];
          C->tan_r[k][(size_t)(d0 + q) * Mf + i] = I.r[i].d[q];
          C->tan_m[k][(size_t)(d0 + q) * Mf + i] = I.m[i].d[q];
        }
    });
  }
  C->inst = final_state;
  return ORC_OK;
}

// Operation count: every instance is re-run from its current states with the counting scalar (values
// bit-identical to the plain run; the oracle's own states are left as they are). counts[0..6]: adds and
// subtracts, multiplies, divides, square roots, logarithms, exponentials, cell-steps (cells at the start
// of each step, summed).
typedef orcdual::Counted CT;

int orc_count_ops(void* H, int n_prog, const int* prog_kind, const double* prog_arg, long long* counts) {
  Ctx* C = (Ctx*)H;
  if (n_prog < 0 || !counts) return ORC_ERR_ARG;
  orcdual::op_count = orcdual::OpCount();
  long long cell_steps = 0;
  for (const Inst<double>& S : C->inst) {
    Inst<CT> I;
    I.N = S.N;
    I.xL = S.xL;
    I.xR = S.xR;
    I.h = S.h;
    I.tau = S.tau;
    I.t = S.t;
    I.status = S.status;
    I.ph = S.ph;
    const int M = S.M();
    I.w.resize(M);
    I.r.resize(M);
    I.m.resize(M);
    I.f.resize(M + 1);
    for (int i = 0; i < M; ++i) {
      I.w[i] = S.w[i];
      I.r[i] = S.r[i];
      I.m[i] = S.m[i];
    }
    for (int i = 0; i <= M; ++i) I.f[i] = Face<CT>{S.f[i].pb, S.f[i].j, CT(S.f[i].x)};
    for (int p = 0; p < n_prog; ++p) {
      if (prog_kind[p] == 0) {
        for (long s = 0; s < (long)prog_arg[p] && I.status == ORC_OK; ++s) {
          cell_steps += I.M();
          step_instance(C->F, C->o, I, -1.0);
        }
      } else {
        while (I.status == ORC_OK && val(I.t) < prog_arg[p]) {
          cell_steps += I.M();
          step_instance(C->F, C->o, I, prog_arg[p]);
        }
      }
    }
  }
  const orcdual::OpCount& q = orcdual::op_count;
  counts[0] = q.add;
  counts[1] = q.mul;
  counts[2] = q.div;
  counts[3] = q.sqrt;
  counts[4] = q.log;
  counts[5] = q.exp;
  counts[6] = cell_steps;
  return ORC_OK;
}

int orc_get_tangent(void* H, int dir, double* d_w, double* d_rho, double* d_m) {
  Ctx* C = (Ctx*)H;
  if (dir < 0 || dir >= C->tan_dirs) return ORC_ERR_ARG;
  long o = 0;
  for (size_t k = 0; k < C->inst.size(); ++k) {
    const long Mf = C->inst[k].M();
    for (long i = 0; i < Mf; ++i, ++o) {
      d_w[o] = C->tan_w[k][(size_t)dir * Mf + i];
      d_rho[o] = C->tan_r[k][(size_t)dir * Mf + i];
      d_m[o] = C->tan_m[k][(size_t)dir * Mf + i];
    }
  }
  return ORC_OK;
}

}  // extern "C"
