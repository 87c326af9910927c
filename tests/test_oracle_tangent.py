"""Pins of the oracle's tangent-linear mode (its forward-mode derivative by dual numbers), the reference
for the CUDA adjoint: the value part reproduces the plain oracle bit for bit, and the derivative parts
match central finite differences of the plain oracle (a computation that shares no derivative code),
direction by direction, on the jittered adjoint workload at small size."""
import dataclasses

import numpy as np
import pytest

from oracle import pyoracle as P
from paper_2211_00705_gb300 import inputs as I


def _run(b, steps):
    o = P.Oracle(b)
    o.step(steps)
    return o.states()


def _dirs(b):
    rng = np.random.default_rng(3)
    M = int(b.cell_offsets[-1])
    z = np.zeros(M)
    out = [dict(tau=b.tau.copy(), rho=z, m=z, widths=z)]
    for c in rng.choice(M, 2, replace=False):
        e = np.zeros(M)
        e[c] = b.rho[c]
        out.append(dict(tau=np.zeros(b.n_inst), rho=e, m=z, widths=z))
    for c in rng.choice(M, 2, replace=False):
        e = np.zeros(M)
        e[c] = max(abs(b.m[c]), b.rho[c])
        out.append(dict(tau=np.zeros(b.n_inst), rho=z, m=e, widths=z))
    dw = np.zeros(M)
    f = int(np.where(b.phase[:-1] != b.phase[1:])[0][0])
    dw[f], dw[f + 1] = 0.1 * b.widths[f + 1], -0.1 * b.widths[f + 1]   # the boundary moves right
    out.append(dict(tau=np.zeros(b.n_inst), rho=z, m=z, widths=dw))
    return out


def test_tangent_values_are_the_plain_oracle():
    b = I.adjoint_batch(n_inst=2, n_lattice=60, n_steps=40)
    plain = _run(b, 40)
    st, _ = P.Oracle(b).tangent([("step", 40)], seed_rho=np.ones((1, int(b.cell_offsets[-1]))))
    for k in ("offsets", "widths", "rho", "m", "phase", "t", "status"):
        np.testing.assert_array_equal(plain[k], st[k])


def test_tangent_matches_central_differences():
    """Final-state derivatives in the directions tau, rho and m of single cells, and the boundary
    position, against central differences (relative step 1e-6 for states, 1e-4 for tau and the
    boundary, whose effect on the states is ~1e-7 relative and needs the larger step to rise above
    round-off)."""
    b = I.adjoint_batch(n_inst=1, n_lattice=60, n_steps=40)
    dirs = _dirs(b)
    st, d = P.Oracle(b).tangent([("step", 40)], seed_w=np.stack([x["widths"] for x in dirs]),
                               seed_rho=np.stack([x["rho"] for x in dirs]), seed_m=np.stack([x["m"] for x in dirs]),
                               seed_tau=np.stack([x["tau"] for x in dirs]))
    for q, dd in enumerate(dirs):
        eps = 1e-4 if (dd["tau"].any() or dd["widths"].any()) else 1e-6
        sp = _run(dataclasses.replace(b, tau=b.tau + eps * dd["tau"], rho=b.rho + eps * dd["rho"],
                                      m=b.m + eps * dd["m"], widths=b.widths + eps * dd["widths"]), 40)
        sm = _run(dataclasses.replace(b, tau=b.tau - eps * dd["tau"], rho=b.rho - eps * dd["rho"],
                                      m=b.m - eps * dd["m"], widths=b.widths - eps * dd["widths"]), 40)
        assert len(sp["rho"]) == len(st["rho"]) == len(sm["rho"])
        for key in ("rho", "m"):
            fd = (sp[key] - sm[key]) / (2 * eps)
            tg = d[key][q]
            err = np.max(np.abs(fd - tg)) / np.max(np.abs(tg))
            assert err <= 2e-5, (q, key, err)


def test_tangent_of_a_uniform_state_is_exact():
    """Closed form: a uniform liquid state is left unchanged by a step (every face flux is the same
    physical flux), and so is a uniform shift of its momentum (every face flux shifts by the same amount,
    HLL being consistent): d rho_T / d m0 = 0 and d m_T / d m0 = 1 in every cell, whatever dt is."""
    N = 40
    fl = I.workload_fluid()
    b = I.Batch(n_lattice=np.array([N], np.int32), x_left=np.zeros(1), x_right=np.ones(1),
                tau=np.array([1e-7]), cell_offsets=np.array([0, N], np.int32), widths=np.full(N, 1.0 / N),
                rho=np.full(N, 1000.0), m=np.full(N, 5000.0), phase=np.ones(N, np.uint8), fluid=fl,
                options=I.Options(), t_end=0.0, n_steps=3, name="uniform liquid")
    st, d = P.Oracle(b).tangent([("step", 3)], seed_m=np.ones((1, N)))
    np.testing.assert_allclose(d["rho"][0], 0.0, atol=1e-12)
    np.testing.assert_allclose(d["m"][0], 1.0, atol=1e-12)


@pytest.mark.parametrize("kind", ["cavitation", "nucleation"])
def test_tangent_through_phase_creation(kind):
    """Phase creation (App. B), liquid pulled apart (cavitation) or vapour driven together (nucleation):
    the derivative of the final states with respect to V (the initial momentum rho0 (-+V)) through the
    creation step, the created cell and its two boundaries, against central differences of the plain
    oracle (relative step 1e-6). The nucleated liquid cell starts ~1e-7 wide, its boundaries see star
    pressures within rounding of the side pressures: the shock branch's derivative at p* -> p_K."""
    if kind == "cavitation":
        b = I.cavitation_batch(4, 2, n_range=(64, 96), n_steps=40)
    else:
        b = I.nucleation_batch(5, 2, n_range=(64, 96), n_steps=40)
    b = dataclasses.replace(b, options=I.scaled_options(creation=1, tol_nb=3e-13, tol_k=3e-11))
    dm = np.zeros(int(b.cell_offsets[-1]))
    V = np.zeros(b.n_inst)
    for i in range(b.n_inst):
        sl = slice(b.cell_offsets[i], b.cell_offsets[i + 1])
        u = b.m[sl] / b.rho[sl]
        V[i] = abs(u[0])
        dm[sl] = np.sign(u) * b.rho[sl] * V[i]          # d m0 for a relative change of V
    st, d = P.Oracle(b).tangent([("step", 40)], seed_m=dm[None, :])
    assert (st["status"] == 0).all()
    assert (np.diff(st["phase"].astype(int)) != 0).sum() >= 2 * b.n_inst   # a created cell in every instance
    eps = 1e-6
    sp = _run(dataclasses.replace(b, m=b.m + eps * dm), 40)
    sm = _run(dataclasses.replace(b, m=b.m - eps * dm), 40)
    assert len(sp["rho"]) == len(st["rho"]) == len(sm["rho"])
    # A nucleated liquid cell is stiff (a_L >> a_V): its density moves by ~1e-9 relative per unit of eps and
    # its momentum derivative is ~1e-10, both below what a difference of solves stopped at tol resolves. That
    # cell is checked through its width and mass rho w; every other cell element by element.
    stiff = (st["phase"] == 1) & (st["phase"] != b.phase[0])
    for key in ("rho", "m", "widths"):
        fd = (sp[key] - sm[key]) / (2 * eps)
        tg = d[key][0]
        sel = ~stiff if key != "widths" else np.ones_like(stiff)
        err = np.max(np.abs(fd - tg)[sel]) / np.max(np.abs(tg[sel]))
        assert err <= 2e-5, (key, err)
    if stiff.any():
        mass = lambda s: s["rho"] * s["widths"]
        fd = (mass(sp) - mass(sm)) / (2 * eps)
        tg = d["rho"][0] * st["widths"] + st["rho"] * d["widths"][0]
        err = np.max(np.abs(fd - tg)[stiff] / np.abs(tg[stiff]))
        assert err <= 2e-5, ("created liquid mass", err)


def test_tangent_through_the_split_of_a_cell_between_two_boundaries():
    """Split of a cell between two phase boundaries (Sec. 3.4, cut at the lattice face nearest its midpoint):
    a vapour cell of 2.4h between boundaries at 7.1h and 9.5h, perturbed states, split in the first step.
    Derivatives of the final states after 3 steps in the directions rho of the vapour cell and m of a liquid
    cell against central differences of the plain oracle (relative step 1e-4)."""
    N = 20
    h = 1.0 / N
    fl = I.workload_fluid()
    rv = fl.p_sat / fl.a2_vap
    widths = np.array([h] * 7 + [0.1 * h, 2.4 * h, 0.5 * h] + [h] * 10)
    phase = np.array([1] * 8 + [0] + [1] * 11, np.uint8)
    rng = np.random.default_rng(4)
    M = len(widths)
    rho = np.where(phase == 1, fl.rho0_liq * (1 + 1e-4 * rng.uniform(-1, 1, M)), rv * (1 + 1e-2 * rng.uniform(-1, 1, M)))
    m = rho * rng.uniform(-2, 2, M)
    b = I.Batch(n_lattice=np.array([N], np.int32), x_left=np.zeros(1), x_right=np.ones(1),
                tau=np.array([I.tau_paper()]), cell_offsets=np.array([0, M], np.int32), widths=widths, rho=rho, m=m,
                phase=phase, fluid=fl, options=I.scaled_options(tol_nb=3e-13, tol_k=3e-11), t_end=0.0, n_steps=3,
                name="vapour cell between two boundaries")
    o = P.Oracle(b)
    o.step(3)
    assert o.states()["status"][0] == 0 and o.stats()["splits"][0] == 1
    dr, dm = np.zeros(M), np.zeros(M)
    dr[8] = rho[8]
    dm[12] = rho[12]
    st, d = P.Oracle(b).tangent([("step", 3)], seed_rho=np.stack([dr, np.zeros(M)]), seed_m=np.stack([np.zeros(M), dm]))
    eps = 1e-4
    for q, (er, em) in enumerate(((dr, 0 * dm), (0 * dr, dm))):
        sp = _run(dataclasses.replace(b, rho=b.rho + eps * er, m=b.m + eps * em), 3)
        sm = _run(dataclasses.replace(b, rho=b.rho - eps * er, m=b.m - eps * em), 3)
        assert len(sp["rho"]) == len(st["rho"]) == len(sm["rho"])
        for key in ("rho", "m", "widths"):
            fd = (sp[key] - sm[key]) / (2 * eps)
            tg = d[key][q]
            err = np.max(np.abs(fd - tg)) / np.max(np.abs(tg))
            assert err <= 2e-5, (q, key, err)
