"""Plant plausible mistakes in a copy of the oracle, one at a time, and report which CPU test catches each
(a check of the oracle's pins; a tool run by hand, not a test: pytest does not collect this file).

Each entry names a mistake and replaces one exact string of oracle.cpp (or dual.h) that occurs once. For each
entry the oracle's sources are copied to a temporary directory, the copy is edited and compiled, and the
oracle tests run against that library (ORACLE_LIB, stopping at the first failure). The tracked sources are
never written. Run from anywhere:

    python tests/plant_mistakes.py            # every batch (a few minutes)
    python tests/plant_mistakes.py dual        # one batch: scheme, batch2, batch3, batch4, dual, residual, newton
"""
import os
import subprocess
import sys

import shutil
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
ORACLE = os.path.join(ROOT, "oracle")
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
TESTS = ["tests/test_oracle_pins.py", "tests/test_oracle_residual.py", "tests/test_oracle_scheme.py",
         "tests/test_oracle_tangent.py", "tests/test_oracle_newton_floor.py"]

SCHEME = [
 ("kinetic relation: sign of the kinetic-energy jump", "T Q = (R.g - L.g) - 0.5 * jp * (L.v + R.v);", "T Q = (R.g - L.g) + 0.5 * jp * (L.v + R.v);"),
 ("kinetic relation: liquid pressure instead of vapour", "T pV = left_is_vapour ? L.p : R.p;", "T pV = left_is_vapour ? R.p : L.p;"),
 ("Gibbs energy: factor a^2 dropped", "return e.a2 * tlog(T(rho / e.rho_sat));", "return tlog(T(rho / e.rho_sat));"),
 ("rarefaction wave: density ratio inverted", "return e.a * tlog(T(rs / rhoK));", "return e.a * tlog(T(rhoK / rs));"),
 ("shock wave: factor 2 in the jump product", "T q = (pstar - pK) * dv;", "T q = 2.0 * (pstar - pK) * dv;"),
 ("shock wave derivative: sign of the second term", "T dq = dv + (pstar - pK) * vs * vs / e.a2;", "T dq = dv - (pstar - pK) * vs * vs / e.a2;"),
 ("boundary system G1: sign of z^2 [[v]]", "S->G[0] = jp + z * z * jv;", "S->G[0] = jp - z * z * jv;"),
 ("boundary system G2: sign of z [[v]]", "S->G[1] = S->fl + S->fr + z * jv + (ur - ul);", "S->G[1] = S->fl + S->fr - z * jv + (ur - ul);"),
 ("boundary system G2: velocity jump transposed", "S->G[1] = S->fl + S->fr + z * jv + (ur - ul);", "S->G[1] = S->fl + S->fr + z * jv + (ul - ur);"),
 ("HLL: sign of the dissipation term", "SL * Fr[c] + SL * SR * (Ur[c] - Ul[c])", "SL * Fr[c] - SL * SR * (Ur[c] - Ul[c])"),
 ("HLL: left and right physical fluxes transposed", "(SR * Fl[c] - SL * Fr[c] +", "(SR * Fr[c] - SL * Fl[c] +"),
 ("merge: wrong width weighting", "T rm = (I.w[a] * I.r[a] + I.w[b] * I.r[b]) / wm;", "T rm = (I.w[a] * I.r[a] + I.w[a] * I.r[b]) / wm;"),
 ("dual time: wrong pseudo-time denominator", "Nr[i] = (Wr[i] + th * tr) / (1.0 + th);", "Nr[i] = (Wr[i] + th * tr) / (1.0 + 2.0 * th);"),
 ("dual time: theta from the current width (convergence only)", "theta[i] = tmin(T(o.theta_nb), T(hpred[i] / I.h));", "theta[i] = tmin(T(o.theta_nb), T(val(I.w[i]) / I.h));"),
 ("CFL: half the time step", "T dt = o.cfl * I.h / S;", "T dt = 0.5 * o.cfl * I.h / S;"),
 ("creation: sign of the second boundary's z [[v]] in the velocity balance", "S->E[2] = S->fl + S->fr + z1 * jv1 + z2 * jv2 + (ur - ul);", "S->E[2] = S->fl + S->fr + z1 * jv1 - z2 * jv2 + (ur - ul);"),
 ("creation: sign of z2^2 [[v]]", "S->E[1] = (x[2] - x[1]) + z2 * z2 * jv2;", "S->E[1] = (x[2] - x[1]) - z2 * z2 * jv2;"),
 ("split: cut at the quarter point", "double xm = 0.5 * (val(I.f[i].x) + val(I.f[i + 1].x));", "double xm = 0.25 * (val(I.f[i].x) + 3.0 * val(I.f[i + 1].x));"),
]
BATCH2 = [
 ("boundary flux: sign of p* in the momentum flux", "R.F[1] = -R.z * uV + pV;", "R.F[1] = -R.z * uV - pV;"),
 ("boundary flux: sign of the mass flux", "R.F[0] = -R.z;", "R.F[0] = R.z;"),
 ("boundary speed: w from the liquid side volume", "T vV = (phl == VAP) ? S.L.v : S.R.v;", "T vV = (phl == VAP) ? S.R.v : S.L.v;"),
 ("no-transition star: exponent sign", "double rs = std::sqrt(rl * rr) * std::exp((ul - ur) / (2.0 * e.a));", "double rs = std::sqrt(rl * rr) * std::exp((ur - ul) / (2.0 * e.a));"),
 ("creation detection: thresholds swapped", "det[g] = (P == LIQ) ? (ps < F.p_min) : (ps > F.p_tilde);", "det[g] = (P == LIQ) ? (ps > F.p_tilde) : (ps < F.p_min);"),
 ("regular update: flux difference transposed", "I.r[i] = (hn * I.r[i] - dt * (F0[i + 1] - F0[i])) / hnp1;", "I.r[i] = (hn * I.r[i] - dt * (F0[i] - F0[i + 1])) / hnp1;"),
 ("physical flux: pressure dropped", "F[1] = m * u + pressure(e, r);", "F[1] = m * u;"),
]
BATCH3 = [
 ("explicit ALE update: face speeds transposed", "T hnp1 = wn[i] + (wl[i + 1] - wr[i]) * dt;", "T hnp1 = wn[i] + (wr[i] - wl[i + 1]) * dt;"),
 ("created cell: width from one boundary speed", "I.w.insert(I.w.begin() + g, (R.w2 - R.w1) * dt);", "I.w.insert(I.w.begin() + g, R.w2 * dt);"),
 ("created cell: momentum with the parent velocity sign", "I.m.insert(I.m.begin() + g, R.rhoC * R.uC);", "I.m.insert(I.m.begin() + g, -R.rhoC * R.uC);"),
 ("transmissive left end: flux of the second cell", "phys_flux(F.ph[I.ph[0]], I.r[0], I.m[0], Fx);  // transmissive boundary", "phys_flux(F.ph[I.ph[1]], I.r[1], I.m[1], Fx);  // transmissive boundary"),
 ("boundary position: moved against its speed", "xpb_new[g] = I.f[g].x + wc[g] * dt;", "xpb_new[g] = I.f[g].x - wc[g] * dt;"),
 ("Part 2: block widths not updated", "      I.w[i] = hl[i];\n    }\n    for (int g = lo + 1; g <= hi; ++g)", "    }\n    for (int g = lo + 1; g <= hi; ++g)"),
 ("creation flux: created-state pressure dropped", "Fl1[g] = -R.z1 * R.uC + R.pC;", "Fl1[g] = -R.z1 * R.uC;"),
 ("predicted widths: boundary speeds transposed", "for (int i = 0; i < M; ++i) hpred[i] = I.w[i] + (wf[i + 1] - wf[i]) * dt;", "for (int i = 0; i < M; ++i) hpred[i] = I.w[i] + (wf[i] - wf[i + 1]) * dt;"),
]
BATCH4 = [
 ("tangent shock form: factor 2 dropped in df/dp", "T((1.0 - (pstar - pK) * vs / (2.0 * e.a2)) / den)", "T((1.0 - (pstar - pK) * vs / e.a2) / den)"),
 ("tangent shock form: sound speed dropped from the denominator", "T den = e.a * tsqrt(T(rhoK * rs));", "T den = tsqrt(T(rhoK * rs));"),
]
DUAL = [
 ("dual numbers: quotient rule sign", "r.d[k] = (a.d[k] - r.v * b.d[k]) / b.v;", "r.d[k] = (a.d[k] + r.v * b.d[k]) / b.v;"),
 ("dual numbers: logarithm derivative", "r.d[k] = a.d[k] / a.v;", "r.d[k] = a.d[k] * a.v;"),
 ("dual numbers: product rule term dropped", "r.d[k] = a.d[k] * b.v + a.v * b.d[k];", "r.d[k] = a.d[k] * b.v;"),
 ("dual numbers: square-root derivative factor", "r.d[k] = 0.5 * a.d[k] / r.v;", "r.d[k] = a.d[k] / r.v;"),
]

RESIDUAL = [
 ("dual-time residual: (1 + theta) dropped from the density term", "double e0 = (1.0 + thv) * std::fabs(val(Nr[i]) - val(Wr[i]))", "double e0 = std::fabs(val(Nr[i]) - val(Wr[i]))"),
 ("dual-time residual: (1 + theta) dropped from the momentum term", "double e1 = (1.0 + thv) * std::fabs(val(Nm[i]) - val(Wm[i]))", "double e1 = std::fabs(val(Nm[i]) - val(Wm[i]))"),
 ("dual-time residual: |W| instead of max(|W|, 1) (density)", "(dtau * std::max(std::fabs(val(Wr[i])), 1.0));", "(dtau * std::fabs(val(Wr[i])));"),
 ("dual-time residual: |W| instead of max(|W|, 1) (momentum)", "(dtau * std::max(std::fabs(val(Wm[i])), 1.0));", "(dtau * std::fabs(val(Wm[i])));"),
 ("dual-time residual: times dt in the printed mode", "          double res = std::max(e0, e1);\n          if (o.res_mode == 1) res *= dtv;\n          if (tiny[i])\n            res_k = std::max(res_k, res);\n          else\n            res_nb = std::max(res_nb, res);\n        }\n        Wr = Nr;", "          double res = std::max(e0, e1);\n          if (o.res_mode == 0) res *= dtv;\n          if (tiny[i])\n            res_k = std::max(res_k, res);\n          else\n            res_nb = std::max(res_nb, res);\n        }\n        Wr = Nr;"),
 ("dual-time stop: either tolerance met instead of both", "        Wm = Nm;\n        if (res_nb < o.tol_nb && res_k < o.tol_k) stop = true;", "        Wm = Nm;\n        if (res_nb < o.tol_nb || res_k < o.tol_k) stop = true;"),
 ("dual-time stop: tiny and other cells' residuals exchanged", "          if (tiny[i])\n            res_k = std::max(res_k, res);\n          else\n            res_nb = std::max(res_nb, res);\n        }\n        Wr = Nr;", "          if (!tiny[i])\n            res_k = std::max(res_k, res);\n          else\n            res_nb = std::max(res_nb, res);\n        }\n        Wr = Nr;"),
]

NEWTON = [
 ("block Newton: the stall rule dropped", "const bool at_floor = corr <= 1e-14 || (corr <= 1e-10 && corr > 0.5 * corr_prev);", "const bool at_floor = corr <= 1e-14;"),
 ("block Newton: the stall rule's contraction test reversed", "(corr <= 1e-10 && corr > 0.5 * corr_prev)", "(corr <= 1e-10 && corr < 0.5 * corr_prev)"),
 ("block Newton: the correction's sign", "Wr[lo + r / 2] = Wr[lo + r / 2] + A[r][n2];", "Wr[lo + r / 2] = Wr[lo + r / 2] - A[r][n2];"),
]

BATCHES = {"scheme": ("oracle.cpp", SCHEME), "batch2": ("oracle.cpp", BATCH2), "batch3": ("oracle.cpp", BATCH3),
           "batch4": ("oracle.cpp", BATCH4), "dual": ("dual.h", DUAL), "residual": ("oracle.cpp", RESIDUAL),
           "newton": ("oracle.cpp", NEWTON)}


def run_batch(fname, mutations):
    from oracle import build as ob
    with open(os.path.join(ORACLE, fname)) as f:
        orig = f.read()
    for name, old, new in mutations:
        n = orig.count(old)
        if n != 1:
            print(f"{name}: text found {n} times, skipped", flush=True)
            continue
        with tempfile.TemporaryDirectory() as tmp:
            for f in os.listdir(ORACLE):
                if f.endswith((".cpp", ".h")):
                    shutil.copy(os.path.join(ORACLE, f), tmp)
            with open(os.path.join(tmp, fname), "w") as f:
                f.write(orig.replace(old, new))
            lib = os.path.join(tmp, "liboracle_planted.so")
            try:
                ob.compile_to(tmp, lib)
            except subprocess.CalledProcessError:
                print(f"{name}: build failed", flush=True)
                continue
            env = dict(os.environ, ORACLE_LIB=lib)
            r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"] + TESTS,
                               cwd=ROOT, capture_output=True, text=True, env=env)
        first = [l for l in r.stdout.splitlines() if l.startswith(("FAILED", "ERROR"))]
        if r.returncode:
            print(f"{name}: CAUGHT ({first[0].split()[1] if first else 'pytest exit %d' % r.returncode})", flush=True)
        else:
            print(f"{name}: not caught", flush=True)


if __name__ == "__main__":
    names = sys.argv[1:] or list(BATCHES)
    for nm in names:
        run_batch(*BATCHES[nm])
