// Device physics of the explicit-implicit splitting scheme (arXiv 2211.00705): equations of state,
// HLL fluxes, the phase-boundary Riemann solver of App. A (Newton with the Armijo rule), the
// same-phase star pressure without transition and the phase-creation solve of App. B.
// Every routine runs in registers of one thread; FP64 throughout.
#pragma once
#include <cstdint>

#include "fastlog.cuh"

namespace imexds {

// Reciprocal refined from the hardware estimate (PTX rcp.approx.ftz.f64, ~23 correct bits) by one third-order
// step of the series 1/b = y / (b y) = y / (1 - e) = y (1 + e + e^2 + ...), e = 1 - b y: y' = y + y (e + e^2),
// three fused multiply-adds whose truncation error e^3 (~2^-66) lies far below double precision (two Newton-
// Raphson steps reach the same accuracy with four). a / b is then a times it, within 2 ulp of the correctly
// rounded quotient (checked against CUDA's division by imexds_check_div). Used where the same quotient is formed
// by several kernels (the lattice velocity m / rho, the HLL weight 1 / (S_R - S_L)), so that all of them produce
// the same bits. Arguments are normal, non-zero doubles (densities, wave-speed spans).
__device__ __forceinline__ double rcp_nr(double b) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(b));
  const double e = __fma_rn(-b, y, 1.0);
  return __fma_rn(y, __fma_rn(e, e, e), y);
}
__device__ __forceinline__ double div_nr(double a, double b) { return a * rcp_nr(b); }

// Comparisons decided on the IEEE-754 bit patterns, in integer instructions. On this GPU an FP64 compare
// or min/max issues to the narrow FP64 pipe that the sweep's arithmetic already saturates; the integer
// pipe is ~30x wider. Each helper returns what the FP64 comparison returns for every non-NaN argument.
// ord_key maps a double to an int64 with the same order (a negative double's magnitude bits inverted);
// -0 keys below +0, which no caller distinguishes (they only feed sums with a non-zero term).
__device__ __forceinline__ long long ord_key(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFll);
}
__device__ __forceinline__ bool lt_bits(double x, double y) { return ord_key(x) < ord_key(y); }
// x >= 0 (either zero, +inf included; false for NaN)
__device__ __forceinline__ bool ge0_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return b <= 0x7FF0000000000000ull || b == 0x8000000000000000ull;
}
// x <= 0 (either zero, -inf included; false for NaN)
__device__ __forceinline__ bool le0_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return b == 0ull || (b >= 0x8000000000000000ull && b <= 0xFFF0000000000000ull);
}
// 0 < x < inf (false for NaN)
__device__ __forceinline__ bool pos_finite_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) - 1ull < 0x7FEFFFFFFFFFFFFFull;
}
// x finite (false for +-inf and NaN)
__device__ __forceinline__ bool finite_bits(double x) {
  return (__double2hiint(x) & 0x7FF00000) != 0x7FF00000;
}
// x != 0 (+0 and -0 are zero; true for NaN, as the FP64 comparison)
__device__ __forceinline__ bool nonzero_bits(double x) { return (__double_as_longlong(x) << 1) != 0; }

// |d| < lim * max(|w|, 1) for lim >= 0, the Sec. 4 stop test of one component, with the maximum and the
// comparison decided on the bit patterns (non-negative doubles order as their bits); one FP64 multiply.
__device__ __forceinline__ bool below_tol(double d, double w, double lim) {
  const double aw = fabs(w);
  const double m = (__double_as_longlong(aw) > 0x3FF0000000000000ll) ? aw : 1.0;
  return __double_as_longlong(fabs(d)) < __double_as_longlong(lim * m);
}

constexpr int VAP = 0;
constexpr int LIQ = 1;

struct Phase {
  int kind;       // 0: p = a2 rho; 1: p = p0 + a2 (rho - rho0)
  double a2, a;   // squared sound speed, sound speed
  double p0, rho0;
  double rho_sat; // density at the saturation pressure (zero of g)
  double ia2, ia, ln_rho_sat, irho_sat;  // 1/a2, 1/a, ln(rho_sat), 1/rho_sat (set on the host)
};

struct Fluid {
  Phase ph[2];
  double p_sat, p_min, p_tilde;
};

struct Opts {
  double cfl, theta_nb, tol_nb, tol_k;
  int res_mode, l_max;
  double newton_tol;
  int newton_itmax;
  double alpha_min, split_ratio;
  int creation;
  int block_solver;  // 0: dual time stepping on each implicit block (Alg. 2); 1: Newton on the block's system
};

__host__ __device__ inline double pressure(const Phase& e, double rho) {
  return e.kind == 0 ? e.a2 * rho : e.p0 + e.a2 * (rho - e.rho0);
}
__host__ __device__ inline double density(const Phase& e, double p) {
  return e.kind == 0 ? p / e.a2 : e.rho0 + (p - e.p0) / e.a2;
}
__device__ inline bool valid_pressure(const Phase& e, double p) { return isfinite(p) && density(e, p) > 0.0; }
// Gibbs energy with dg = v dp: g = a2 ln(rho / rho_sat), zero at the saturation pressure (Sec. 2.1).
__device__ inline double gibbs(const Phase& e, double rho) { return e.a2 * log(rho / e.rho_sat); }

// HLL flux at a same-phase face (Toro), Davis wave speeds S_L = min(u_l, u_r) - a, S_R = max + a, physical
// flux (rho u, rho u^2 + p) (Eq. eeq:isoT both), arranged for the sweep: the physical fluxes come in
// precomputed (u = m/rho once per cell) and one reciprocal of S_R - S_L serves both components. With
// w = S_R / (S_R - S_L) (so -S_L / (S_R - S_L) = 1 - w) the HLL average
//   (S_R F_l - S_L F_r + S_L S_R (U_r - U_l)) / (S_R - S_L)  =  F_r + w ((F_l - F_r) + S_L (U_r - U_l)),
// two fused multiply-adds per component; for the mass component F_l - F_r = m_l - m_r = -(U_r - U_l)_m.
// Every product-sum is an explicit fused multiply-add so that every kernel computing a face flux gets the
// same bits.
__device__ inline double pressure_fma(const Phase& e, double rho) {
  return e.kind == 0 ? e.a2 * rho : __fma_rn(e.a2, rho - e.rho0, e.p0);
}
__device__ inline void hll_pre(double a, double rl, double ml, double ul, double fl1, double rr, double mr, double ur,
                               double fr1, double& F0, double& F1) {
  const bool lt = lt_bits(ul, ur);
  const double umin = lt ? ul : ur;
  const double umax = lt ? ur : ul;
  const double SL = umin - a, SR = umax + a;
  // branch-free: the HLL average is formed for every face (S_R - S_L >= 2a > 0) and the upwind cases
  // select the one-sided physical flux, the same values the three-way branch gives
  const double w = SR * rcp_nr(SR - SL);
  const double d0 = rr - rl, d1 = mr - ml;
  const double H0 = __fma_rn(w, __fma_rn(SL, d0, -d1), mr);
  const double H1 = __fma_rn(w, __fma_rn(SL, d1, fl1 - fr1), fr1);
  const bool up_l = ge0_bits(SL), up_r = le0_bits(SR);
  F0 = up_l ? ml : (up_r ? mr : H0);
  F1 = up_l ? fl1 : (up_r ? fr1 : H1);
}
__device__ inline void phys_flux_fast(const Phase& e, double r, double m, double& F0, double& F1) {
  double u = div_nr(m, r);
  F0 = m;
  F1 = __fma_rn(m, u, pressure_fma(e, r));
}
__device__ inline void hll_fast(const Phase& e, double rl, double ml, double rr, double mr, double& F0, double& F1) {
  double ul = div_nr(ml, rl), ur = div_nr(mr, rr);
  double fl1 = __fma_rn(ml, ul, pressure_fma(e, rl));
  double fr1 = __fma_rn(mr, ur, pressure_fma(e, rr));
  hll_pre(e.a, rl, ml, ul, fl1, rr, mr, ur, fr1, F0, F1);
}

// Outer-wave function f_K of App. A for an isothermal linear EOS: shock sqrt((p* - p_K)(v_K - v*)),
// rarefaction a ln(rho*/rho_K); derivative in dfdp.
__device__ inline double wave_f(const Phase& e, double pstar, double rhoK, double& dfdp) {
  double pK = pressure(e, rhoK);
  double rs = density(e, pstar);
  double vs = 1.0 / rs;
  if (pstar > pK) {
    double dv = 1.0 / rhoK - vs;
    double q = (pstar - pK) * dv;
    double f = sqrt(q);
    double dq = dv + (pstar - pK) * vs * vs / e.a2;
    dfdp = (f > 0.0) ? 0.5 * dq / f : vs / e.a;
    return f;
  }
  dfdp = vs / e.a;
  return e.a * log(rs / rhoK);
}

struct Side {
  double p, rho, v, g, dv;
};

__device__ inline Side side_at(const Phase& e, double p) {
  Side s;
  s.p = p;
  s.rho = density(e, p);
  s.v = 1.0 / s.rho;
  s.g = gibbs(e, s.rho);
  s.dv = -s.v * s.v / e.a2;
  return s;
}

// Kinetic relation z = tau p_V [[g + e_kin]] (Eq. isoT:kin_rel1) with e_kin relative to the moving
// boundary and z^2 = -[[p]]/[[v]], i.e. [[e_kin]] = -[[p]] (v_L + v_R) / 2; returns dz/dp per side.
__device__ inline double kinetic_z(double tau, bool left_is_vapour, const Side& L, const Side& R, double& dzl,
                                   double& dzr) {
  double pV = left_is_vapour ? L.p : R.p;
  double jp = R.p - L.p;
  double Q = (R.g - L.g) - 0.5 * jp * (L.v + R.v);
  double dQl = -L.v + 0.5 * (L.v + R.v) - 0.5 * jp * L.dv;
  double dQr = R.v - 0.5 * (L.v + R.v) - 0.5 * jp * R.dv;
  dzl = tau * ((left_is_vapour ? Q : 0.0) + pV * dQl);
  dzr = tau * ((left_is_vapour ? 0.0 : Q) + pV * dQr);
  return tau * pV * Q;
}

struct PBOut {
  double F0, F1, w, z, pl, pr;
  int iters;
  int ok;
};

// HLLC-based starting pressure of App. A (Eq. HLLC:2p_nopt), with a fallback when it is not positive.
__device__ inline void pb_initial_guess(const Fluid& F, int phl, double rl, double ul, int phr, double rr,
                                        double ur, double& pl0, double& pr0) {
  const Phase& El = F.ph[phl];
  const Phase& Er = F.ph[phr];
  double pl = pressure(El, rl), pr = pressure(Er, rr);
  double Sl = ul - El.a, Sr = ur + Er.a;
  double w = (pr - pl + rl * ul * (Sl - ul) - rr * ur * (Sr - ur)) / (rl * (Sl - ul) - rr * (Sr - ur));
  double rls = (phl == LIQ) ? rl * (Sl - ul) / (Sl - w) : rr * (Sr - ur) / (Sr - w);
  double p = pressure(F.ph[LIQ], rls);
  if (isfinite(p) && p > 0.0) {
    pl0 = p;
    pr0 = p;
    return;
  }
  double pv = (phl == VAP) ? pl : pr;
  double pliq = (phl == LIQ) ? pl : pr;
  double pvg = fmax(pv, 1e-3 * F.p_sat);
  pl0 = (phl == VAP) ? pvg : pliq;
  pr0 = (phr == VAP) ? pvg : pliq;
}

// ---- the phase-boundary Riemann problem of App. A: Newton's method with the Armijo rule on the 2x2 system
// G(p_l*, p_r*) (Eq. 2p_RP:ex_sys), flux F_PB = (-z, -z u_V* + p_V*) (Eq. pb_flux:pt) through the boundary
// moving at w = u_V* + z v_V*. Arranged for repeated calls: one (table-driven) logarithm per side and
// evaluation (ln(rho*/rho_K) = ln(rho*/rho_sat) + ln(rho_sat/rho_K) with the last term fixed per solve),
// reciprocals of the fixed data computed once, and an optional starting point (the previous solution) with
// the HLLC start of App. A as fallback.
struct SideData {
  const Phase* E;
  double rK, pK, invK, CK, aCK, ia2, ia, isat;
};

// invK: 1 / rho_K, the reciprocal the caller also forms the side's velocity with
__device__ inline SideData side_data(const Phase& e, double rK, double invK) {
  SideData s;
  s.E = &e;
  s.rK = rK;
  s.pK = pressure_fma(e, rK);
  s.invK = invK;
  s.isat = e.irho_sat;
  s.CK = e.ln_rho_sat - fast_log(rK);  // ln(rho_sat / rho_K), independent of 1/rho_K
  s.aCK = e.a * s.CK;
  s.ia2 = e.ia2;
  s.ia = e.ia;
  return s;
}

struct SideEval {
  double p, v, g, dv, f, df;
};

// Branch-free: both wave branches are formed and one is selected, so the two sides of a boundary can be
// interleaved by the instruction scheduler.
__device__ inline bool side_eval(const SideData& s, double p, SideEval& o) {
  const Phase& e = *s.E;
  double rs = e.kind == 0 ? p * s.ia2 : __fma_rn(p - e.p0, s.ia2, e.rho0);
  double v = rcp_nr(rs);
  double Ls = fast_log(rs * s.isat);
  o.p = p;
  o.v = v;
  o.g = e.a2 * Ls;
  const double vv = v * v;
  o.dv = -vv * s.ia2;
  // shock (p > p_K): f = sqrt(q), q = (p - p_K)(v_K - v); rarefaction: f = a ln(rho*/rho_K)
  double dvk = s.invK - v;
  double dp = p - s.pK;
  double q = dp * dvk;
  double dq = __fma_rn(dp * vv, s.ia2, dvk);
  const bool qpos = pos_finite_bits(q);  // q > 0 (finite), decided on the bit pattern
  double rq = rsqrt(qpos ? q : 1.0);
  bool shock = pos_finite_bits(dp) && qpos;
  o.f = shock ? q * rq : __fma_rn(e.a, Ls, s.aCK);
  o.df = shock ? 0.5 * dq * rq : v * s.ia;
  return pos_finite_bits(rs) && finite_bits(p);
}

struct PBFast {
  double G0, G1, J00, J01, J10, J11, z, dzl, dzr;
  SideEval L, R;
};

__device__ inline bool pbf_eval(const SideData& sl, const SideData& sr, bool left_vap, double tau, double du,
                                double pl, double pr, PBFast& S) {
  if (!side_eval(sl, pl, S.L) || !side_eval(sr, pr, S.R)) return false;
  const SideEval &L = S.L, &R = S.R;
  // G and its Jacobian with every product-sum fused (the same values to rounding; this is the dual-time
  // chain's inner loop): Q = (g_R - g_L) - jp vs / 2, z = tau p_V Q, G0 = jp + z^2 jv, G1 = f_L + f_R + z jv + du
  const double pV = left_vap ? pl : pr;
  const double jp = pr - pl, jv = R.v - L.v, vs = L.v + R.v;
  const double hj = 0.5 * jp, hv = 0.5 * vs;
  const double Q = __fma_rn(-hj, vs, R.g - L.g);
  const double dQl = __fma_rn(-hj, L.dv, hv - L.v);
  const double dQr = __fma_rn(-hj, R.dv, R.v - hv);
  const double tpV = tau * pV, tQ = tau * Q;
  const double dzl = __fma_rn(tpV, dQl, left_vap ? tQ : 0.0);
  const double dzr = __fma_rn(tpV, dQr, left_vap ? 0.0 : tQ);
  const double z = tpV * Q;
  const double zz = z * z, zj2 = 2.0 * z * jv;
  S.z = z;
  S.dzl = dzl;
  S.dzr = dzr;
  S.G0 = __fma_rn(zz, jv, jp);
  S.G1 = __fma_rn(z, jv, (L.f + R.f) + du);
  S.J00 = __fma_rn(-zz, L.dv, __fma_rn(zj2, dzl, -1.0));
  S.J01 = __fma_rn(zz, R.dv, __fma_rn(zj2, dzr, 1.0));
  S.J10 = __fma_rn(-z, L.dv, __fma_rn(dzl, jv, L.df));
  S.J11 = __fma_rn(z, R.dv, __fma_rn(dzr, jv, R.df));
  return finite_bits(S.G0) && finite_bits(S.G1);
}

// |d| <= 1e-8 max(|x|, p_sat) for finite x and p_sat > 0, the maximum and the comparison decided on bit patterns
// (non-negative doubles order as their bits; false for a NaN d, as the FP64 comparison).
__device__ __forceinline__ bool small_step(double d, double x, double p_sat) {
  const double ax = fabs(x);
  const double m = (__double_as_longlong(ax) > __double_as_longlong(p_sat)) ? ax : p_sat;
  return __double_as_longlong(fabs(d)) <= __double_as_longlong(1e-8 * m);
}

// Newton-Armijo from (x0, x1); returns 1 on convergence with S evaluated at the returned point. One
// evaluation state is kept: trial points are evaluated into S (the direction and the old norm are all
// the line search needs), and S is evaluated again at x only on the rare exits after a failed search.
__device__ inline int pbf_newton(const Fluid& F, const Opts& o, const SideData& sl, const SideData& sr, bool left_vap,
                                 double tau, double du, double imp, double& x0, double& x1, PBFast& S, int& iters) {
  if (!pbf_eval(sl, sr, left_vap, tau, du, x0, x1, S)) return 0;
  const double iimp = rcp_nr(imp);
  // the Armijo test on squared norms: |G_t|^2 <= (1 - 1e-4 lam)^2 |G|^2
  double g0 = S.G0 * iimp;
  double nrm2 = __fma_rn(g0, g0, S.G1 * S.G1);
  bool conv = (nrm2 == 0.0);
  int it = 0;
  while (!conv && it < o.newton_itmax) {
    ++it;
    double det = __fma_rn(S.J00, S.J11, -(S.J01 * S.J10));
    if (!finite_bits(det) || !nonzero_bits(det)) break;
    double idet = rcp_nr(det);
    double d0 = -__fma_rn(S.J11, S.G0, -(S.J01 * S.G1)) * idet;
    double d1 = -__fma_rn(S.J00, S.G1, -(S.J10 * S.G0)) * idet;
    {
      // A full Newton step below 1e-8 (relative) lands within O(1e-16) of the root (quadratic
      // convergence), the point the newton_tol test reaches: take it without the line-search evaluation
      // and carry the recovery quantities (f, v, z) to it to first order (their second-order terms are
      // O(1e-16) relative as well).
      // (tested without dividing: |d| <= 1e-8 max(|x|, p_sat) for both unknowns)
      if (small_step(d0, x0, F.p_sat) && small_step(d1, x1, F.p_sat)) {
        S.L.f = __fma_rn(S.L.df, d0, S.L.f);
        S.R.f = __fma_rn(S.R.df, d1, S.R.f);
        S.L.v = __fma_rn(S.L.dv, d0, S.L.v);
        S.R.v = __fma_rn(S.R.dv, d1, S.R.v);
        S.z = __fma_rn(S.dzl, d0, __fma_rn(S.dzr, d1, S.z));
        x0 += d0;
        x1 += d1;
        conv = true;
        break;
      }
    }
    double lam = 1.0;
    bool acc = false;
    for (int ls = 0; ls <= 20; ++ls) {
      if (pbf_eval(sl, sr, left_vap, tau, du, x0 + lam * d0, x1 + lam * d1, S)) {
        double t0 = S.G0 * iimp;
        double nt2 = __fma_rn(t0, t0, S.G1 * S.G1);
        double f = 1.0 - 1e-4 * lam;
        if (nt2 <= f * f * nrm2) {
          acc = true;
          nrm2 = nt2;
          break;
        }
      }
      lam *= 0.5;
    }
    double s0 = fabs(d0) / fmax(fabs(x0), F.p_sat);
    double s1 = fabs(d1) / fmax(fabs(x1), F.p_sat);
    if (!acc) {
      if (fmax(s0, s1) <= 1e-9) conv = pbf_eval(sl, sr, left_vap, tau, du, x0, x1, S);
      break;
    }
    x0 += lam * d0;
    x1 += lam * d1;
    // a full Newton step below 1e-8 (relative) leaves an error of order 1e-16 (quadratic convergence):
    // the same root the newton_tol test reaches, one evaluation earlier
    if (lam * fmax(s0, s1) <= o.newton_tol || nrm2 == 0.0 || (lam == 1.0 && fmax(s0, s1) <= 1e-8)) conv = true;
  }
  iters += it;
  return conv ? 1 : 0;
}

// Derivatives of one face's flux (F0, F1) and speed w with respect to the states next to it,
// d/d(rho_l, m_l, rho_r, m_r); the Jacobian rows of Newton's method on an implicit block.
struct FaceJac {
  double dF0[4], dF1[4], dw[4];
};

// d f_K / d rho_K at a fixed star pressure for the outer wave of App. A (isothermal linear EOS): rarefaction
// f = a ln(rho*/rho_K) gives -a / rho_K; shock f = (p* - p_K) / (a sqrt(rho_K rho*)) (the same function as
// sqrt((p* - p_K)(v_K - v*)), since p* - p_K = a^2 (rho* - rho_K)) gives -a / sqrt(rho_K rho*) - f / (2 rho_K).
// Both tend to -a / rho_K as p* -> p_K.
__device__ inline double dwave_drhoK(const Phase& e, const SideData& s, double p, double v, double f) {
  if (p > s.pK && f > 0.0) return -e.a * rsqrt(s.rK / v) - 0.5 * f * s.invK;
  return -e.a * s.invK;
}

// Boundary solve with an optional start (gl, gr > 0 ... valid pressures); writes the converged star
// pressures back to gl/gr for the next call. JAC: also the face Jacobian J by the implicit function theorem
// on the converged 2x2 system G(p; W_l, W_r) = 0 (Eq. 2p_RP:ex_sys): only the velocity-balance row G_2
// depends on the states (through u_l, u_r and the reference densities of the outer waves), so
// dp = -DG^{-1} (0, dG_2), and the recovery of App. A (z, u_V*, v_V*) is differentiated along.
template <bool JAC>
__device__ inline PBOut pb_solve_core(const Fluid& F, const Opts& o, double tau, int phl, double rl, double ml, int phr,
                                      double rr, double mr, double& gl, double& gr, FaceJac* J) {
  PBOut R;
  R.ok = 0;
  R.iters = 0;
  R.F0 = R.F1 = R.w = R.z = R.pl = R.pr = 0.0;
  const double irl0 = rcp_nr(rl), irr0 = rcp_nr(rr);  // one reciprocal per side: velocity and 1/rho_K
  double ul = ml * irl0, ur = mr * irr0;
  const SideData sl = side_data(F.ph[phl], rl, irl0), sr = side_data(F.ph[phr], rr, irr0);
  const bool left_vap = (phl == VAP);
  const double imp = __fma_rn(rl, F.ph[phl].a, rr * F.ph[phr].a), du = ur - ul;
  PBFast S;
  double x0 = gl, x1 = gr;
  int ok = 0;
  if (nonzero_bits(gl) || nonzero_bits(gr)) ok = pbf_newton(F, o, sl, sr, left_vap, tau, du, imp, x0, x1, S, R.iters);
  if (!ok) {
    pb_initial_guess(F, phl, rl, ul, phr, rr, ur, x0, x1);
    ok = pbf_newton(F, o, sl, sr, left_vap, tau, du, imp, x0, x1, S, R.iters);
  }
  if (!ok) return R;
  double ulS = ul - S.L.f, urS = ur + S.R.f;
  double uV = left_vap ? ulS : urS;
  double vV = left_vap ? S.L.v : S.R.v;
  double pV = left_vap ? x0 : x1;
  R.z = S.z;
  R.w = __fma_rn(R.z, vV, uV);
  R.F0 = -R.z;
  R.F1 = __fma_rn(-R.z, uV, pV);
  R.pl = x0;
  R.pr = x1;
  R.ok = 1;
  gl = x0;
  gr = x1;
  if (JAC) {
    const double irl = irl0, irr = irr0;
    const double fKl = dwave_drhoK(F.ph[phl], sl, x0, S.L.v, S.L.f);
    const double fKr = dwave_drhoK(F.ph[phr], sr, x1, S.R.v, S.R.f);
    // dG_2 / d(rho_l, m_l, rho_r, m_r): f_l(p_l; rho_l) + f_r(p_r; rho_r) + z [[v]] + u_r - u_l
    const double g2[4] = {fKl + ul * irl, -irl, fKr - ur * irr, irr};
    const double det = __fma_rn(S.J00, S.J11, -(S.J01 * S.J10));
    if (!nonzero_bits(det) || !finite_bits(det)) {
      R.ok = 0;
      return R;
    }
    const double idet = rcp_nr(det);
    const double cl = S.J01 * idet, cr = -S.J00 * idet;  // dp_l = cl g2, dp_r = cr g2
    const double dul[4] = {-ul * irl, irl, 0.0, 0.0};
    const double dur[4] = {0.0, 0.0, -ur * irr, irr};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const double dpl = cl * g2[k], dpr = cr * g2[k];
      const double dz = __fma_rn(S.dzl, dpl, S.dzr * dpr);
      double duV, dpV, dvV;
      if (left_vap) {
        duV = dul[k] - __fma_rn(S.L.df, dpl, k == 0 ? fKl : 0.0);
        dpV = dpl;
        dvV = S.L.dv * dpl;
      } else {
        duV = dur[k] + __fma_rn(S.R.df, dpr, k == 2 ? fKr : 0.0);
        dpV = dpr;
        dvV = S.R.dv * dpr;
      }
      J->dF0[k] = -dz;
      J->dF1[k] = __fma_rn(-R.z, duV, __fma_rn(-dz, uV, dpV));
      J->dw[k] = __fma_rn(R.z, dvV, __fma_rn(dz, vV, duV));
    }
  }
  return R;
}

__device__ inline PBOut pb_solve_warm(const Fluid& F, const Opts& o, double tau, int phl, double rl, double ml, int phr,
                                      double rr, double mr, double& gl, double& gr) {
  return pb_solve_core<false>(F, o, tau, phl, rl, ml, phr, rr, mr, gl, gr, nullptr);
}

// Jacobian of the HLL flux of hll_pre / hll_fast (Davis speeds, the same branch and the same min/max choice)
// with respect to (rho_l, m_l, rho_r, m_r); the face does not move (dw = 0).
__device__ inline void hll_jac(const Phase& e, double rl, double ml, double rr, double mr, FaceJac& J) {
  const double irl = rcp_nr(rl), irr = rcp_nr(rr);
  const double ul = ml * irl, ur = mr * irr;
  const double a2 = e.a2, a = e.a;
  const double dul[4] = {-ul * irl, irl, 0.0, 0.0};
  const double dur[4] = {0.0, 0.0, -ur * irr, irr};
  // physical fluxes (m, m u + p) and their derivatives: dF1/drho = a^2 - u^2, dF1/dm = 2u
  const double fl1 = ml * ul + pressure(e, rl), fr1 = mr * ur + pressure(e, rr);
  const double dFl0[4] = {0.0, 1.0, 0.0, 0.0}, dFr0[4] = {0.0, 0.0, 0.0, 1.0};
  const double dFl1[4] = {a2 - ul * ul, 2.0 * ul, 0.0, 0.0};
  const double dFr1[4] = {0.0, 0.0, a2 - ur * ur, 2.0 * ur};
  const bool lt = lt_bits(ul, ur);
  const double SL = (lt ? ul : ur) - a, SR = (lt ? ur : ul) + a;
#pragma unroll
  for (int k = 0; k < 4; ++k) J.dw[k] = 0.0;
  if (ge0_bits(SL)) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      J.dF0[k] = dFl0[k];
      J.dF1[k] = dFl1[k];
    }
    return;
  }
  if (le0_bits(SR)) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      J.dF0[k] = dFr0[k];
      J.dF1[k] = dFr1[k];
    }
    return;
  }
  // H = (S_R F_l - S_L F_r + S_L S_R (U_r - U_l)) / (S_R - S_L): dH = (dN - H (dS_R - dS_L)) / (S_R - S_L)
  const double iw = rcp_nr(SR - SL);
  const double H0 = (SR * ml - SL * mr + SL * SR * (rr - rl)) * iw;
  const double H1 = (SR * fl1 - SL * fr1 + SL * SR * (mr - ml)) * iw;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double dSL = lt ? dul[k] : dur[k];
    const double dSR = lt ? dur[k] : dul[k];
    const double dss = __fma_rn(dSL, SR, SL * dSR);
    const double dU0 = (k == 2 ? 1.0 : 0.0) - (k == 0 ? 1.0 : 0.0);
    const double dU1 = (k == 3 ? 1.0 : 0.0) - (k == 1 ? 1.0 : 0.0);
    // dN = dS_R F_l + S_R dF_l - dS_L F_r - S_L dF_r + d(S_L S_R) (U_r - U_l) + S_L S_R dU, fused
    const double dN0 = __fma_rn(dSR, ml, __fma_rn(SR, dFl0[k], __fma_rn(-dSL, mr, __fma_rn(-SL, dFr0[k],
                                          __fma_rn(dss, rr - rl, SL * SR * dU0)))));
    const double dN1 = __fma_rn(dSR, fl1, __fma_rn(SR, dFl1[k], __fma_rn(-dSL, fr1, __fma_rn(-SL, dFr1[k],
                                          __fma_rn(dss, mr - ml, SL * SR * dU1)))));
    const double dsd = dSR - dSL;
    J.dF0[k] = __fma_rn(-H0, dsd, dN0) * iw;
    J.dF1[k] = __fma_rn(-H1, dsd, dN1) * iw;
  }
}

// |x| > |y| on the bit patterns (integer pipe), for non-NaN arguments: the pivot choice of the block solves.
__device__ __forceinline__ bool absgt_bits(double x, double y) {
  const unsigned long long m = 0x7FFFFFFFFFFFFFFFull;
  return ((unsigned long long)__double_as_longlong(x) & m) > ((unsigned long long)__double_as_longlong(y) & m);
}

// Dense N x N solve of A x = b (b in column N) by Gaussian elimination with partial pivoting, fully unrolled
// so that A stays in registers: each candidate row is compared with the pivot row and the two are swapped by
// selects when it is larger, which leaves the largest entry in the pivot row. The solution replaces column N.
template <int N>
__device__ inline bool solve_dense(double (&A)[N][N + 1]) {
#pragma unroll
  for (int c = 0; c < N; ++c) {
#pragma unroll
    for (int r = c + 1; r < N; ++r) {
      const bool sw = absgt_bits(A[r][c], A[c][c]);
#pragma unroll
      for (int j = c; j <= N; ++j) {
        const double t = sw ? A[r][j] : A[c][j];
        A[r][j] = sw ? A[c][j] : A[r][j];
        A[c][j] = t;
      }
    }
    if (!nonzero_bits(A[c][c]) || !finite_bits(A[c][c])) return false;
    const double ip = rcp_nr(A[c][c]);
#pragma unroll
    for (int r = c + 1; r < N; ++r) {
      const double f = A[r][c] * ip;
#pragma unroll
      for (int j = c + 1; j <= N; ++j) A[r][j] = __fma_rn(-f, A[c][j], A[r][j]);
    }
    A[c][N] *= ip;
#pragma unroll
    for (int j = c + 1; j < N; ++j) A[c][j] *= ip;
  }
#pragma unroll
  for (int c = N - 1; c >= 0; --c) {
#pragma unroll
    for (int j = c + 1; j < N; ++j) A[c][N] = __fma_rn(-A[c][j], A[j][N], A[c][N]);
  }
  return true;
}

// Banded solve for the implicit systems of general blocks: n unknowns (two per cell), lower and upper
// bandwidth 3 (a cell couples to its neighbours only), partial pivoting among the 4 rows that reach the
// pivot column, which widens the upper band to 6. Row r stores columns r-3 .. r+6 in A[r][0..9]
// (column j at A[r][j - r + 3]); b is the right-hand side and receives the solution.
constexpr int BAND_W = 10;
__device__ inline bool solve_band(double (*A)[BAND_W], double* b, int n) {
  for (int c = 0; c < n; ++c) {
    const int rmax = min(c + 3, n - 1), jmax = min(c + 6, n - 1);
    int p = c;
    for (int r = c + 1; r <= rmax; ++r)
      if (absgt_bits(A[r][c - r + 3], A[p][c - p + 3])) p = r;
    const double piv = A[p][c - p + 3];
    if (!nonzero_bits(piv) || !finite_bits(piv)) return false;
    if (p != c) {
      for (int j = c; j <= jmax; ++j) {
        const double t = A[c][j - c + 3];
        A[c][j - c + 3] = A[p][j - p + 3];
        A[p][j - p + 3] = t;
      }
      const double t = b[c];
      b[c] = b[p];
      b[p] = t;
    }
    const double ip = rcp_nr(A[c][3]);
    for (int r = c + 1; r <= rmax; ++r) {
      const double f = A[r][c - r + 3] * ip;
      for (int j = c + 1; j <= jmax; ++j) A[r][j - r + 3] = __fma_rn(-f, A[c][j - c + 3], A[r][j - r + 3]);
      b[r] = __fma_rn(-f, b[c], b[r]);
    }
  }
  for (int c = n - 1; c >= 0; --c) {
    double s = b[c];
    const int jmax = min(c + 6, n - 1);
    for (int j = c + 1; j <= jmax; ++j) s = __fma_rn(-A[c][j - c + 3], b[j], s);
    b[c] = s / A[c][3];
  }
  return true;
}

// Star pressure of the same-phase Riemann problem without transition: closed form for two
// rarefactions, otherwise bisection on [min(p_l, p_r), p_TR] (the shock curve lies above the
// rarefaction curve).
__device__ inline double nopt_star(const Phase& e, double rl, double ul, double rr, double ur) {
  double pl = pressure(e, rl), pr = pressure(e, rr);
  double pm = fmin(pl, pr);
  double rs = sqrt(rl * rr) * exp((ul - ur) / (2.0 * e.a));
  double ptr = pressure(e, rs);
  if (ptr <= pm) return ptr;
  double lo = pm, hi = ptr, d;
  for (int i = 0; i < 200; ++i) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    double phi = wave_f(e, mid, rl, d) + wave_f(e, mid, rr, d) + (ur - ul);
    if (phi > 0.0)
      hi = mid;
    else
      lo = mid;
  }
  return 0.5 * (lo + hi);
}

// Creation test of App. B at a same-phase face: the no-transition star pressure p* below p_min (liquid,
// cavitation) or above p_tilde (vapour, nucleation). Same decision as comparing nopt_star, without its
// bisection where the bracket already decides: when the two-rarefaction value p_TR exceeds
// min(p_l, p_r), p* lies in [min(p_l, p_r), p_TR] (and the bisection returns a point of that bracket).
__device__ inline bool creation_detect(const Fluid& F, int P, double rl, double ul, double rr, double ur) {
  const Phase& e = F.ph[P];
  const double pl = pressure(e, rl), pr = pressure(e, rr);
  const double pm = fmin(pl, pr);
  const double ptr = pressure(e, sqrt(rl * rr) * exp((ul - ur) / (2.0 * e.a)));
  if (ptr <= pm) return (P == LIQ) ? (ptr < F.p_min) : (ptr > F.p_tilde);
  if (P == LIQ) {
    if (pm >= F.p_min) return false;
  } else {
    if (ptr <= F.p_tilde) return false;
    if (pm > F.p_tilde) return true;
  }
  const double ps = nopt_star(e, rl, ul, rr, ur);
  return (P == LIQ) ? (ps < F.p_min) : (ps > F.p_tilde);
}

struct CreateOut {
  double pC, rhoC, uC, z1, z2, w1, w2;
  double pPl, pPr;  // converged parent-side pressures
  int iters;
  int ok;
};

struct CrSys {
  double E[3], J[3][3];
  Side Pl, C, Pr;
  double z1, z2, fl, fr;
};

__device__ inline bool cr_eval(const Fluid& F, double tau, int P, double rl, double ul, double rr, double ur,
                               const double x[3], CrSys& S) {
  int Cph = 1 - P;
  const Phase& EP = F.ph[P];
  const Phase& EC = F.ph[Cph];
  if (!valid_pressure(EP, x[0]) || !valid_pressure(EC, x[1]) || !valid_pressure(EP, x[2])) return false;
  S.Pl = side_at(EP, x[0]);
  S.C = side_at(EC, x[1]);
  S.Pr = side_at(EP, x[2]);
  double dz1a, dz1b, dz2a, dz2b;
  S.z1 = kinetic_z(tau, P == VAP, S.Pl, S.C, dz1a, dz1b);
  S.z2 = kinetic_z(tau, Cph == VAP, S.C, S.Pr, dz2a, dz2b);
  double dfl, dfr;
  S.fl = wave_f(EP, x[0], rl, dfl);
  S.fr = wave_f(EP, x[2], rr, dfr);
  double jv1 = S.C.v - S.Pl.v, jv2 = S.Pr.v - S.C.v;
  double z1 = S.z1, z2 = S.z2;
  S.E[0] = (x[1] - x[0]) + z1 * z1 * jv1;
  S.E[1] = (x[2] - x[1]) + z2 * z2 * jv2;
  S.E[2] = S.fl + S.fr + z1 * jv1 + z2 * jv2 + (ur - ul);
  S.J[0][0] = -1.0 + 2.0 * z1 * dz1a * jv1 - z1 * z1 * S.Pl.dv;
  S.J[0][1] = 1.0 + 2.0 * z1 * dz1b * jv1 + z1 * z1 * S.C.dv;
  S.J[0][2] = 0.0;
  S.J[1][0] = 0.0;
  S.J[1][1] = -1.0 + 2.0 * z2 * dz2a * jv2 - z2 * z2 * S.C.dv;
  S.J[1][2] = 1.0 + 2.0 * z2 * dz2b * jv2 + z2 * z2 * S.Pr.dv;
  S.J[2][0] = dfl + dz1a * jv1 - z1 * S.Pl.dv;
  S.J[2][1] = dz1b * jv1 + z1 * S.C.dv + dz2a * jv2 - z2 * S.C.dv;
  S.J[2][2] = dfr + dz2b * jv2 + z2 * S.Pr.dv;
  return isfinite(S.E[0]) && isfinite(S.E[1]) && isfinite(S.E[2]);
}

// 3x3 solve by elimination with partial pivoting.
__device__ inline bool solve3(const double A[3][3], const double b[3], double x[3]) {
  double M[3][4];
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) M[i][j] = A[i][j];
    M[i][3] = b[i];
  }
  for (int c = 0; c < 3; ++c) {
    int p = c;
    for (int r = c + 1; r < 3; ++r)
      if (fabs(M[r][c]) > fabs(M[p][c])) p = r;
    if (M[p][c] == 0.0 || !isfinite(M[p][c])) return false;
    if (p != c)
      for (int j = 0; j < 4; ++j) {
        double t = M[p][j];
        M[p][j] = M[c][j];
        M[c][j] = t;
      }
    for (int r = c + 1; r < 3; ++r) {
      double f = M[r][c] / M[c][c];
      for (int j = c; j < 4; ++j) M[r][j] -= f * M[c][j];
    }
  }
  for (int i = 2; i >= 0; --i) {
    double s = M[i][3];
    for (int j = i + 1; j < 3; ++j) s -= M[i][j] * x[j];
    x[i] = s / M[i][i];
  }
  return true;
}

// Single-phase Riemann problem with creation of the other phase (App. B): unknowns
// (p_parent-, p_created, p_parent+), two boundary momentum jumps and the chained velocity balance,
// solved by Newton with the Armijo rule from the saturation pressure.
__device__ __noinline__ CreateOut creation_solve(const Fluid& F, const Opts& o, double tau, int P, double rl, double ml,
                                           double rr, double mr) {
  CreateOut R;
  R.ok = 0;
  R.iters = 0;
  double ul = ml / rl, ur = mr / rr;
  double imp = (rl + rr) * F.ph[P].a;
  double x[3] = {F.p_sat, F.p_sat, F.p_sat};
  CrSys S;
  if (!cr_eval(F, tau, P, rl, ul, rr, ur, x, S)) return R;
  double nrm = sqrt((S.E[0] / imp) * (S.E[0] / imp) + (S.E[1] / imp) * (S.E[1] / imp) + S.E[2] * S.E[2]);
  bool conv = (nrm == 0.0);
  int it = 0;
  while (!conv && it < o.newton_itmax) {
    ++it;
    double b[3] = {-S.E[0], -S.E[1], -S.E[2]}, d[3];
    if (!solve3(S.J, b, d)) break;
    double lam = 1.0;
    bool acc = false;
    CrSys T;
    for (int ls = 0; ls <= 20; ++ls) {
      double xt[3] = {x[0] + lam * d[0], x[1] + lam * d[1], x[2] + lam * d[2]};
      if (cr_eval(F, tau, P, rl, ul, rr, ur, xt, T)) {
        double nt = sqrt((T.E[0] / imp) * (T.E[0] / imp) + (T.E[1] / imp) * (T.E[1] / imp) + T.E[2] * T.E[2]);
        if (nt <= (1.0 - 1e-4 * lam) * nrm) {
          acc = true;
          nrm = nt;
          break;
        }
      }
      lam *= 0.5;
    }
    double s = 0.0;
    for (int i = 0; i < 3; ++i) s = fmax(s, fabs(d[i]) / fmax(fabs(x[i]), F.p_sat));
    if (!acc) {
      if (s <= 1e-9) conv = true;
      break;
    }
    for (int i = 0; i < 3; ++i) x[i] += lam * d[i];
    S = T;
    if (lam * s <= o.newton_tol || nrm == 0.0) conv = true;
  }
  R.iters = it;
  if (!conv) return R;
  R.pC = x[1];
  R.pPl = x[0];
  R.pPr = x[2];
  R.rhoC = S.C.rho;
  R.z1 = S.z1;
  R.z2 = S.z2;
  double uPl = ul - S.fl;
  R.uC = uPl - S.z1 * (S.C.v - S.Pl.v);
  R.w1 = R.uC + S.z1 * S.C.v;
  R.w2 = R.uC + S.z2 * S.C.v;
  R.ok = (R.w2 > R.w1) ? 1 : 0;
  return R;
}

// Two ways the block Newton iteration reaches the floor that rounding puts under the residual before the Sec. 4
// test holds (for a tiny cell of fraction alpha the update T amplifies a one-ulp change of W by about 1/alpha, which
// can exceed a tight stop tolerance; the iterate then cycles among a few points ulps apart). With the correction
// measured as c = max over components |d| / max(|W|, 1):
//   (a) c <= 1e-14: the correction cannot move the iterate further than its own rounding;
//   (b) c <= 1e-10 and c > c_prev / 2: the corrections stopped contracting; Newton's quadratic convergence
//       takes small corrections to much smaller ones, so only rounding (or a kink of the flux exactly at the
//       root) can keep them from shrinking.
// Either ends the iteration as l_max would: the corrected iterate is used and counted among the blocks that did
// not meet the test. c_prev of the first step is +infinity, so (b) needs two corrections.
constexpr double kNewtonFloor = 1e-14;
constexpr double kNewtonStallBelow = 1e-10;
__device__ inline double newton_corr(int nb, const double* W0, const double* W1, const double* d0, const double* d1) {
  double c = 0.0;
  for (int q = 0; q < nb; ++q) {
    c = fmax(c, fabs(d0[q]) * rcp_nr(fmax(fabs(W0[q]), 1.0)));
    c = fmax(c, fabs(d1[q]) * rcp_nr(fmax(fabs(W1[q]), 1.0)));
  }
  return c;
}
__device__ inline bool newton_at_floor(double c, double c_prev) {
  return c <= kNewtonFloor || (c <= kNewtonStallBelow && c > 0.5 * c_prev);
}

// One Newton step on a block's implicit system R(W) = W - T(W) = 0 (Algorithm 2 Part 1's update T with fluxes and
// widths at W; the option block_solver = 1): dR/dW = I - dT/dW assembled from the face Jacobians,
//   dT_q/dW = -(dt / h_q) [(dF_{q+1/2} - dF_{q-1/2}) + T_q (dw_{q+1/2} - dw_{q-1/2})],
// rows and columns (cell q, component c) = 2q + c, then the solve of dR/dW d = T - W. Cells 0..nb-1 of the block;
// ih[q] = 1 / h_q(W); fj[g] the Jacobian of interior face g = 1..nb-1 (between cells g-1 and g). Blocks of three
// cells (the common one) use the dense 6 x 6 solve, larger blocks the banded one, so that every kernel that solves
// a block of a given size (the forward kernels and the adjoint's replay) produces the same bits. False if the
// system is singular.
__device__ inline bool newton_block_step(int nb, double dt, const double* ih, const double* T0, const double* T1,
                                         const double* W0, const double* W1, const FaceJac* fj, double* d0,
                                         double* d1) {
  if (nb == 3) {
    double A[6][7];
#pragma unroll
    for (int r = 0; r < 6; ++r) {
#pragma unroll
      for (int c = 0; c < 6; ++c) A[r][c] = (r == c) ? 1.0 : 0.0;
      A[r][6] = (r & 1) ? T1[r >> 1] - W1[r >> 1] : T0[r >> 1] - W0[r >> 1];
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const double coef = dt * ih[q];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const double Tq = c ? T1[q] : T0[q];
        if (q + 1 <= 2) {  // right face q+1: + coef (dF + T dw), columns of cells q, q+1
          const FaceJac& J = fj[q + 1];
#pragma unroll
          for (int k = 0; k < 4; ++k)
            A[2 * q + c][2 * q + k] = __fma_rn(coef, __fma_rn(Tq, J.dw[k], c ? J.dF1[k] : J.dF0[k]), A[2 * q + c][2 * q + k]);
        }
        if (q >= 1) {  // left face q: - coef (dF + T dw), columns of cells q-1, q
          const FaceJac& J = fj[q];
#pragma unroll
          for (int k = 0; k < 4; ++k)
            A[2 * q + c][2 * (q - 1) + k] =
                __fma_rn(-coef, __fma_rn(Tq, J.dw[k], c ? J.dF1[k] : J.dF0[k]), A[2 * q + c][2 * (q - 1) + k]);
        }
      }
    }
    if (!solve_dense<6>(A)) return false;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      d0[q] = A[2 * q][6];
      d1[q] = A[2 * q + 1][6];
    }
    return true;
  }
  constexpr int NMAX = 2 * 18;
  const int n2 = 2 * nb;
  if (n2 > NMAX) return false;
  double A[NMAX][BAND_W], rhs[NMAX];
  for (int r = 0; r < n2; ++r) {
    for (int k = 0; k < BAND_W; ++k) A[r][k] = 0.0;
    A[r][3] = 1.0;  // the identity (column r)
  }
  for (int q = 0; q < nb; ++q) {
    const double coef = dt * ih[q];
    rhs[2 * q] = T0[q] - W0[q];
    rhs[2 * q + 1] = T1[q] - W1[q];
    for (int c = 0; c < 2; ++c) {
      const int row = 2 * q + c;
      const double Tq = c ? T1[q] : T0[q];
      if (q + 1 < nb) {
        const FaceJac& J = fj[q + 1];
        for (int k = 0; k < 4; ++k)
          A[row][2 * q + k - row + 3] =
              __fma_rn(coef, __fma_rn(Tq, J.dw[k], c ? J.dF1[k] : J.dF0[k]), A[row][2 * q + k - row + 3]);
      }
      if (q >= 1) {
        const FaceJac& J = fj[q];
        for (int k = 0; k < 4; ++k)
          A[row][2 * (q - 1) + k - row + 3] =
              __fma_rn(-coef, __fma_rn(Tq, J.dw[k], c ? J.dF1[k] : J.dF0[k]), A[row][2 * (q - 1) + k - row + 3]);
      }
    }
  }
  if (!solve_band(A, rhs, n2)) return false;
  for (int q = 0; q < nb; ++q) {
    d0[q] = rhs[2 * q];
    d1[q] = rhs[2 * q + 1];
  }
  return true;
}

}  // namespace imexds
