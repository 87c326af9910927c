"""Study behind the next solver choice (Newton on each block instead of dual time, the paper's own outlook):
one block's implicit system (3 cells around a phase boundary, the tiny cell in the middle) is assembled
from the oracle's pointwise pieces (the App. A boundary solve and HLL) on states of the 4096-instance
workload after 5 and 40 steps. Dual time (Alg. 2, local steps theta_i = min(theta_nb, h_pred/h), the
scaled stop test of Sec. 4) and Newton (finite-difference Jacobian, stopped at the same residual levels)
reach the same solution; Newton needs 1-3 iterations where dual time needs 12-73."""
import math

import numpy as np
from paper_2211_00705_gb300 import inputs as I
from oracle import pyoracle as P

TINY = np.array([False, True, False])   # the block is {k-1, k, k+1}, the tiny cell k in the middle


def block_case(b, k_inst, n_steps):
    o = P.Oracle(b.subset([k_inst]))
    o.step(n_steps)
    s = o.states()
    ph, w, r, m = s["phase"], s["widths"], s["rho"], s["m"]
    f = int(np.nonzero(ph[:-1] != ph[1:])[0][0]) + 1        # boundary face between cells f-1 and f
    k = f - 1 if w[f - 1] < w[f] else f                    # tiny cell
    h = 1.0 / b.n_lattice[k_inst]
    S = np.max(np.abs(m / r) + np.where(ph == 0, math.sqrt(b.fluid.a2_vap), math.sqrt(b.fluid.a2_liq)))
    dt = b.options.cfl * h / S
    return dict(ph=ph, w=w, r=r, m=m, f=f, k=k, h=h, dt=dt, tau=float(b.tau[k_inst]))


def make_T(fl, opts, c):
    ph, w, r, m, f, k, h, dt, tau = (c[x] for x in ("ph", "w", "r", "m", "f", "k", "h", "dt", "tau"))
    lo, hi = k - 1, k + 1
    FL = P.hll(fl, ph[lo], r[lo - 1], m[lo - 1], r[lo], m[lo])   # outer faces at U^n
    FR = P.hll(fl, ph[hi], r[hi], m[hi], r[hi + 1], m[hi + 1])
    def T(W):
        Wr, Wm = W[0::2], W[1::2]
        F = [FL]
        wf = [0.0]
        for g in range(lo + 1, hi + 1):                          # interior faces between g-1 and g
            a, bb = g - 1 - lo, g - lo
            if g == f:
                R = P.pb_solve(fl, opts, tau, int(ph[g - 1]), Wr[a], Wm[a] / Wr[a], int(ph[g]), Wr[bb], Wm[bb] / Wr[bb])
                F.append(np.array([R["F0"], R["F1"]])); wf.append(R["w"])
            else:
                F.append(P.hll(fl, ph[g], Wr[a], Wm[a], Wr[bb], Wm[bb])); wf.append(0.0)
        F.append(FR); wf.append(0.0)
        out = np.zeros(6)
        hn1 = np.zeros(3)
        for q in range(3):
            i = lo + q
            hn1[q] = w[i] + (wf[q + 1] - wf[q]) * dt
            out[2 * q] = (w[i] * r[i] - dt * (F[q + 1][0] - F[q][0])) / hn1[q]
            out[2 * q + 1] = (w[i] * m[i] - dt * (F[q + 1][1] - F[q][1])) / hn1[q]
        return out, hn1
    W0 = np.array([x for i in range(lo, hi + 1) for x in (r[i], m[i])])
    return T, W0


def dts(T, W0, c, opts, hpred):
    th = np.minimum(opts.theta_nb, hpred / c["h"])
    W = W0.copy()
    for l in range(1, 20001):
        TW, _ = T(W)
        N = W.copy()
        ok = True
        for q in range(3):
            for j in (0, 1):
                N[2 * q + j] = (W[2 * q + j] + th[q] * TW[2 * q + j]) / (1 + th[q])
                # scaled residual (reading R10): (1 + theta)|W^{l+1} - W^l| / (theta dt max(|W^l|, 1)) times dt
                res = (1 + th[q]) * abs(N[2 * q + j] - W[2 * q + j]) / (th[q] * max(abs(W[2 * q + j]), 1.0))
                ok = ok and res < (opts.tol_k if TINY[q] else opts.tol_nb)
        W = N
        if ok:
            return W, l
    return W, -1


def newton(T, W0, c, opts):
    W = W0.copy()
    for it in range(1, 50):
        TW, _ = T(W)
        R = W - TW
        tol = np.repeat(np.where(TINY, opts.tol_k, opts.tol_nb), 2) * np.maximum(np.abs(W), 1.0)
        if (np.abs(R) <= tol).all():
            return W, it - 1
        J = np.eye(6)
        for j in range(6):
            e = 1e-7 * max(abs(W[j]), 1.0)
            Wp, Wm_ = W.copy(), W.copy(); Wp[j] += e; Wm_[j] -= e
            J[:, j] -= (T(Wp)[0] - T(Wm_)[0]) / (2 * e)
        W = W - np.linalg.solve(J, R)
    return W, -1


def test_newton_on_a_block_needs_far_fewer_iterations_than_dual_time():
    b = I.workload(1, scale=16 / 4096)
    fl, opts = b.fluid, b.options
    for ki in range(b.n_inst):
        for n in (5, 40):
            c = block_case(b, ki, n)
            T, W0 = make_T(fl, opts, c)
            _, hp = T(W0)                      # widths predicted from the boundary speed at U^n
            Wd, ld = dts(T, W0, c, opts, hp)
            Wn, ln = newton(T, W0, c, opts)
            assert 10 <= ld and 1 <= ln <= 3, (ki, n, ld, ln)
            assert np.max(np.abs(Wd - Wn) / np.maximum(np.abs(Wd), 1.0)) <= 1e-7, (ki, n)
