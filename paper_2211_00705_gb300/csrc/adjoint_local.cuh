// Local derivatives for the discrete adjoint: forward-mode dual numbers on the device and the face
// functions of the scheme written once for a generic scalar (double or dual). They give the exact
// Jacobians of one face (HLL at a same-phase face, the physical flux at a domain end, and the
// phase-boundary flux of App. A through the implicit function theorem on the converged 2x2 system).
// Values are not used from here (the forward pass supplies them); only derivatives are.
#pragma once
#include "physics.cuh"

namespace imexds {
namespace adj {

template <int K>
struct Dual {
  double v;
  double d[K];
};

template <int K>
__device__ __forceinline__ Dual<K> dconst(double x) {
  Dual<K> r;
  r.v = x;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = 0.0;
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> dvar(double x, int k0) {
  Dual<K> r = dconst<K>(x);
  r.d[k0] = 1.0;
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator+(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator-(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator-(const Dual<K>& a) {
  Dual<K> r;
  r.v = -a.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = -a.d[k];
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator*(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = __fma_rn(a.d[k], b.v, a.v * b.d[k]);
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator/(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r;
  const double ib = rcp_nr(b.v);  // within 1 ulp of 1 / b
  r.v = a.v * ib;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = __fma_rn(-r.v, b.d[k], a.d[k]) * ib;
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator*(double a, const Dual<K>& b) {
  Dual<K> r;
  r.v = a * b.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a * b.d[k];
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator+(const Dual<K>& a, double b) {
  Dual<K> r = a;
  r.v = a.v + b;
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator-(const Dual<K>& a, double b) {
  Dual<K> r = a;
  r.v = a.v - b;
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator-(double a, const Dual<K>& b) {
  return dconst<K>(a) - b;
}
template <int K>
__device__ __forceinline__ Dual<K> operator/(const Dual<K>& a, double b) {
  Dual<K> r;
  const double ib = rcp_nr(b);
  r.v = a.v * ib;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * ib;
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator/(double a, const Dual<K>& b) {
  return dconst<K>(a) / b;
}
template <int K>
__device__ __forceinline__ Dual<K> dsqrt(const Dual<K>& a) {
  Dual<K> r;
  r.v = sqrt(a.v);
  const double s = 0.5 * rcp_nr(r.v);
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * s;
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> dlog(const Dual<K>& a) {
  Dual<K> r;
  r.v = log(a.v);
  const double s = rcp_nr(a.v);
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * s;
  return r;
}

// ---- face functions on dual numbers (Sec. 2.1, Sec. 4, App. A) ----
template <int K>
__device__ __forceinline__ Dual<K> pressure_d(const Phase& e, const Dual<K>& rho) {
  return e.kind == 0 ? e.a2 * rho : (e.a2 * rho + (e.p0 - e.a2 * e.rho0));
}
template <int K>
__device__ __forceinline__ Dual<K> density_d(const Phase& e, const Dual<K>& p) {
  return e.kind == 0 ? p / e.a2 : (p - e.p0) / e.a2 + e.rho0;
}

// Physical flux (rho u, rho u^2 + p).
template <int K>
__device__ __forceinline__ void phys_flux_d(const Phase& e, const Dual<K>& r, const Dual<K>& m, Dual<K>& F0,
                                            Dual<K>& F1) {
  F0 = m;
  F1 = m * (m / r) + pressure_d(e, r);
}

// HLL flux with Davis wave speeds; the branch and the min/max are taken on values.
template <int K>
__device__ void hll_d(const Phase& e, const Dual<K>& rl, const Dual<K>& ml, const Dual<K>& rr, const Dual<K>& mr,
                      Dual<K>& F0, Dual<K>& F1) {
  Dual<K> ul = ml / rl, ur = mr / rr;
  Dual<K> Fl0 = ml, Fl1 = ml * ul + pressure_d(e, rl);
  Dual<K> Fr0 = mr, Fr1 = mr * ur + pressure_d(e, rr);
  Dual<K> SL = (ur.v - e.a < ul.v - e.a) ? (ur - e.a) : (ul - e.a);
  Dual<K> SR = (ul.v + e.a < ur.v + e.a) ? (ur + e.a) : (ul + e.a);
  if (SL.v >= 0.0) {
    F0 = Fl0;
    F1 = Fl1;
  } else if (SR.v <= 0.0) {
    F0 = Fr0;
    F1 = Fr1;
  } else {
    Dual<K> iw = 1.0 / (SR - SL);
    F0 = (SR * Fl0 - SL * Fr0 + SL * SR * (rr - rl)) * iw;
    F1 = (SR * Fl1 - SL * Fr1 + SL * SR * (mr - ml)) * iw;
  }
}

template <int K>
struct SideD {
  Dual<K> p, rho, v, g, dv;
};
template <int K>
__device__ __forceinline__ SideD<K> side_d(const Phase& e, const Dual<K>& p) {
  SideD<K> s;
  s.p = p;
  s.rho = density_d(e, p);
  s.v = 1.0 / s.rho;
  s.g = e.a2 * dlog(s.rho / e.rho_sat);
  s.dv = -(s.v * s.v) / e.a2;
  return s;
}
// Outer-wave function f_K(p*) (shock / rarefaction branch on values) and df/dp*. Shock branch: for both
// linear EOS p* - p_K = a^2 (rho* - rho_K), so (p* - p_K)(v_K - v*) = (p* - p_K)^2 / (a^2 rho_K rho*) and
// f = (p* - p_K) / (a sqrt(rho_K rho*)): the same function without the product of two vanishing factors
// under a square root, whose derivative turns into 0/0 where p* -> p_K (cells next to a boundary sit in
// the star region once the outer waves have left).
template <int K>
__device__ Dual<K> wave_f_d(const Phase& e, const Dual<K>& ps, const Dual<K>& rK, Dual<K>& dfdp) {
  Dual<K> pK = pressure_d(e, rK);
  Dual<K> rs = density_d(e, ps);
  Dual<K> vs = 1.0 / rs;
  if (ps.v > pK.v) {
    Dual<K> den = e.a * dsqrt(rK * rs);
    Dual<K> dp = ps - pK;
    Dual<K> f = dp / den;
    dfdp = (1.0 - dp * vs / (2.0 * e.a2)) / den;
    return f;
  }
  dfdp = vs / e.a;
  return e.a * dlog(rs / rK);
}
// Kinetic relation z = tau p_V [[g + e_kin]] with [[e_kin]] = -[[p]] (v_L + v_R)/2, and dz/dp per side.
template <int K>
__device__ Dual<K> kinetic_z_d(const Dual<K>& tau, bool left_vap, const SideD<K>& L, const SideD<K>& R,
                               Dual<K>& dzl, Dual<K>& dzr) {
  Dual<K> pV = left_vap ? L.p : R.p;
  Dual<K> jp = R.p - L.p;
  Dual<K> vs = L.v + R.v;
  Dual<K> Q = (R.g - L.g) - 0.5 * (jp * vs);
  Dual<K> dQl = 0.5 * vs - L.v - 0.5 * (jp * L.dv);
  Dual<K> dQr = R.v - 0.5 * vs - 0.5 * (jp * R.dv);
  dzl = tau * (left_vap ? Q + pV * dQl : pV * dQl);
  dzr = tau * (left_vap ? pV * dQr : Q + pV * dQr);
  return tau * (pV * Q);
}

// Phase-boundary face: the flux (F0, F1) and boundary speed w as functions of the adjacent states and
// tau, differentiated at the converged star pressures (pl, pr) of G(p; W_l, W_r, tau) = 0 (Eq.
// 2p_RP:ex_sys): dp = -DG^{-1} (dG/dtheta) dtheta, then the recovery of App. A on duals. Inputs are
// duals over the caller's directions; returns false if DG is singular.
template <int K>
__device__ bool pb_face_d(const Fluid& F, int phl, int phr, const Dual<K>& rl, const Dual<K>& ml, const Dual<K>& rr,
                          const Dual<K>& mr, const Dual<K>& tau, double pl, double pr, Dual<K>& F0, Dual<K>& F1,
                          Dual<K>& w) {
  const Phase& El = F.ph[phl];
  const Phase& Er = F.ph[phr];
  const bool left_vap = (phl == VAP);
  Dual<K> ul = ml / rl, ur = mr / rr;
  // G at fixed p (derivatives with respect to the inputs only) and its p-Jacobian (values)
  Dual<K> P0 = dconst<K>(pl), P1 = dconst<K>(pr);
  SideD<K> L = side_d(El, P0), R = side_d(Er, P1);
  Dual<K> dzl, dzr;
  Dual<K> z = kinetic_z_d(tau, left_vap, L, R, dzl, dzr);
  Dual<K> dfl, dfr;
  Dual<K> fl = wave_f_d(El, P0, rl, dfl);
  Dual<K> fr = wave_f_d(Er, P1, rr, dfr);
  Dual<K> jv = R.v - L.v;
  Dual<K> G0 = (P1 - P0) + z * z * jv;
  Dual<K> G1 = fl + fr + z * jv + (ur - ul);
  const double J00 = -1.0 + 2.0 * z.v * dzl.v * jv.v - z.v * z.v * L.dv.v;
  const double J01 = 1.0 + 2.0 * z.v * dzr.v * jv.v + z.v * z.v * R.dv.v;
  const double J10 = dfl.v + dzl.v * jv.v - z.v * L.dv.v;
  const double J11 = dfr.v + dzr.v * jv.v + z.v * R.dv.v;
  const double det = J00 * J11 - J01 * J10;
  if (!(det != 0.0) || !isfinite(det)) return false;
  const double id = 1.0 / det;
  // p as duals: value p*, derivative -J^{-1} dG
#pragma unroll
  for (int k = 0; k < K; ++k) {
    P0.d[k] = -(J11 * G0.d[k] - J01 * G1.d[k]) * id;
    P1.d[k] = -(-J10 * G0.d[k] + J00 * G1.d[k]) * id;
  }
  // recovery on duals: z from the kinetic relation, u* from the outer waves, w from z = -rho (u - w)
  L = side_d(El, P0);
  R = side_d(Er, P1);
  z = kinetic_z_d(tau, left_vap, L, R, dzl, dzr);
  fl = wave_f_d(El, P0, rl, dfl);
  fr = wave_f_d(Er, P1, rr, dfr);
  Dual<K> uV = left_vap ? (ul - fl) : (ur + fr);
  Dual<K> vV = left_vap ? L.v : R.v;
  Dual<K> pV = left_vap ? P0 : P1;
  w = uV + z * vV;
  F0 = -z;
  F1 = pV - z * uV;
  return true;
}

// Phase creation at a same-phase face (App. B): the outputs (z1, z2, u_C, p_C, rho_C, w1, w2) as functions of
// the adjacent states and tau, differentiated at the converged pressures x = (p_P-, p_C, p_P+) of the 3x3
// system E(x; W_l, W_r, tau) = 0: dx = -DE^{-1} (dE/dtheta) dtheta, then the recovery on duals.
template <int K>
__device__ bool creation_d(const Fluid& F, int P, const Dual<K>& rl, const Dual<K>& ml, const Dual<K>& rr,
                           const Dual<K>& mr, const Dual<K>& tau, const double x[3], Dual<K> out[7]) {
  const int Cph = 1 - P;
  const Phase& EP = F.ph[P];
  const Phase& EC = F.ph[Cph];
  Dual<K> ul = ml / rl, ur = mr / rr;
  Dual<K> X[3] = {dconst<K>(x[0]), dconst<K>(x[1]), dconst<K>(x[2])};
  double J[3][3];
  Dual<K> E[3];
  for (int pass = 0; pass < 2; ++pass) {
    SideD<K> Pl = side_d(EP, X[0]), C = side_d(EC, X[1]), Pr = side_d(EP, X[2]);
    Dual<K> dz1a, dz1b, dz2a, dz2b, dfl, dfr;
    Dual<K> z1 = kinetic_z_d(tau, P == VAP, Pl, C, dz1a, dz1b);
    Dual<K> z2 = kinetic_z_d(tau, Cph == VAP, C, Pr, dz2a, dz2b);
    Dual<K> fl = wave_f_d(EP, X[0], rl, dfl);
    Dual<K> fr = wave_f_d(EP, X[2], rr, dfr);
    Dual<K> jv1 = C.v - Pl.v, jv2 = Pr.v - C.v;
    if (pass == 0) {
      E[0] = (X[1] - X[0]) + z1 * z1 * jv1;
      E[1] = (X[2] - X[1]) + z2 * z2 * jv2;
      E[2] = fl + fr + z1 * jv1 + z2 * jv2 + (ur - ul);
      J[0][0] = -1.0 + 2.0 * z1.v * dz1a.v * jv1.v - z1.v * z1.v * Pl.dv.v;
      J[0][1] = 1.0 + 2.0 * z1.v * dz1b.v * jv1.v + z1.v * z1.v * C.dv.v;
      J[0][2] = 0.0;
      J[1][0] = 0.0;
      J[1][1] = -1.0 + 2.0 * z2.v * dz2a.v * jv2.v - z2.v * z2.v * C.dv.v;
      J[1][2] = 1.0 + 2.0 * z2.v * dz2b.v * jv2.v + z2.v * z2.v * Pr.dv.v;
      J[2][0] = dfl.v + dz1a.v * jv1.v - z1.v * Pl.dv.v;
      J[2][1] = dz1b.v * jv1.v + z1.v * C.dv.v + dz2a.v * jv2.v - z2.v * C.dv.v;
      J[2][2] = dfr.v + dz2b.v * jv2.v + z2.v * Pr.dv.v;
      for (int k = 0; k < K; ++k) {
        double b[3] = {-E[0].d[k], -E[1].d[k], -E[2].d[k]}, dx[3];
        if (!solve3(J, b, dx)) return false;
        for (int i = 0; i < 3; ++i) X[i].d[k] = dx[i];
      }
    } else {
      Dual<K> uPl = ul - fl;
      Dual<K> uC = uPl - z1 * (C.v - Pl.v);
      out[0] = z1;
      out[1] = z2;
      out[2] = uC;
      out[3] = X[1];
      out[4] = C.rho;
      out[5] = uC + z1 * C.v;
      out[6] = uC + z2 * C.v;
    }
  }
  return true;
}

}  // namespace adj
}  // namespace imexds
