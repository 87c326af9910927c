"""The discrete adjoint (imexds_adjoint) against the oracle's own derivative (forward mode through the
oracle, an independent computation) and against central finite differences of the CUDA forward run, on
the adjoint workload (Riemann instances, jittered states, tight dual-time tolerances) scaled down."""
import dataclasses

import numpy as np
import pytest

from oracle import pyoracle as P
from paper_2211_00705_gb300 import inputs as I
from tests.adjoint_util import directions, grad_dot, misfit, target_samples

pytestmark = pytest.mark.gpu

# adjoint vs the oracle's tangent: both are exact derivatives of the discrete map, the adjoint at the
# converged implicit system (implicit function theorem), the tangent of the iterations as computed; the
# tangent itself moves by up to 1.3e-7 (relative) when the dual-time tolerances go from 1e-4 to 1e-6
# times the scaled ones (measured on this batch), so the bar is 1e-6
TOL_TANGENT = 1e-6
TOL_FD = 1e-5        # adjoint vs central differences (the target relative error)


def _forward(batch, program, k=16, **kw):
    from paper_2211_00705_gb300.imexds import Imexds
    ctx = Imexds.from_batch(batch, **kw)
    ctx.set_adjoint_checkpoint(k)
    for kind, arg in program:
        ctx.step(arg) if kind == "step" else ctx.run_to(arg)
    return ctx


def _target(batch, program):
    tb = dataclasses.replace(batch, tau=batch.tau * 1.1)
    ctx = _forward(tb, program)
    s = ctx.get_states()
    ctx.close()
    return target_samples(s, tb)


def _grad(batch, program, k=16, **kw):
    tgt = _target(batch, program)
    ctx = _forward(batch, program, k, **kw)
    s = ctx.get_states()
    assert (s["status"] == 0).all()
    J, gr = misfit(s, tgt, batch)
    g = ctx.adjoint(gr, np.zeros_like(gr))
    info = ctx.adjoint_info()
    stats = ctx.stats()
    ctx.close()
    return tgt, s, J, g, info, stats


def _oracle_dirs(batch, program, tgt, dirs):
    o = P.Oracle(batch)
    st, d = o.tangent(program, seed_w=np.stack([x["widths"] for x in dirs]),
                      seed_rho=np.stack([x["rho"] for x in dirs]), seed_m=np.stack([x["m"] for x in dirs]),
                      seed_tau=np.stack([x["tau"] for x in dirs]), threads=8)
    J, gr = misfit(st, tgt, batch)
    off = st["offsets"]
    out = []
    for q in range(len(dirs)):
        v = np.zeros(batch.n_inst)
        for i in range(batch.n_inst):
            s = slice(off[i], off[i + 1])
            v[i] = float(np.dot(gr[s], d["rho"][q][s]))
        out.append(v)
    return out


def _rel(a, b, scale):
    return np.abs(a - b) / np.maximum(scale, 1e-300)


@pytest.mark.parametrize("program", [[("step", 150)], [("step", 60), ("step", 90)]])
def test_adjoint_matches_oracle_tangent(program):
    """Every directional derivative (tau, random rho and m fields, the boundary position) of every
    instance agrees with the oracle's forward-mode derivative of the same run."""
    b = I.adjoint_batch(n_inst=6, n_lattice=120, n_steps=150)
    tgt, s, J, g, info, stats = _grad(b, program)
    assert (g["status"] == 0).all(), g["status"]
    assert info["replay_err"] <= 1e-9, info
    assert stats["merges"].sum() + stats["splits"].sum() > 0  # grid management is differentiated too
    dirs = directions(b)
    ref = _oracle_dirs(b, program, tgt, dirs)
    for q, d in enumerate(dirs):
        got = grad_dot(b, g, d)
        scale = np.max(np.abs(ref[q]))
        err = _rel(got, ref[q], scale)
        print(q, np.max(err), scale)
        assert np.max(err) <= TOL_TANGENT, (q, got, ref[q])


def test_adjoint_through_the_split_of_a_cell_between_two_boundaries():
    """Split of a cell between two phase boundaries (Sec. 3.4: cut at the lattice face nearest its midpoint): a
    vapour cell of 2.4h between boundaries at 7.1h and 9.5h, perturbed states, split in the first of 3 steps.
    Random seeds on the final densities, momenta and widths; the adjoint's directional derivatives (tau,
    density and momentum fields, each boundary position on its own) against the oracle's forward-mode
    derivative of the same run."""
    from paper_2211_00705_gb300.imexds import Imexds
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
    ctx = Imexds.from_batch(b)
    ctx.set_adjoint_checkpoint(2)
    ctx.step(3)
    s, st = ctx.get_states(), ctx.stats()
    assert s["status"][0] == 0 and st["splits"][0] == 1
    n = int(s["offsets"][-1])
    sr, sm, sw = rng.standard_normal(n), rng.standard_normal(n) * 1e-2, rng.standard_normal(n) * 1e3
    g = ctx.adjoint(sr, sm, sw)
    ctx.close()
    assert (g["status"] == 0).all(), g["status"]
    zero, z1 = np.zeros(M), np.zeros(1)
    dirs = [{"tau": b.tau.copy(), "rho": zero, "m": zero, "widths": zero}]
    for _ in range(2):
        dirs.append({"tau": z1, "rho": rng.standard_normal(M) * rho, "m": zero, "widths": zero})
        dirs.append({"tau": z1, "rho": zero, "m": rng.standard_normal(M) * np.maximum(np.abs(m), rho), "widths": zero})
    for f in (7, 8):  # the boundaries at faces 8 and 9: cells f | f+1, moved by 1e-3 of the smaller width
        dw = np.zeros(M)
        d = 1e-3 * min(widths[f], widths[f + 1])
        dw[f], dw[f + 1] = d, -d
        dirs.append({"tau": z1, "rho": zero, "m": zero, "widths": dw})
    so, d = P.Oracle(b).tangent([("step", 3)], seed_w=np.stack([x["widths"] for x in dirs]),
                                 seed_rho=np.stack([x["rho"] for x in dirs]), seed_m=np.stack([x["m"] for x in dirs]),
                                 seed_tau=np.stack([x["tau"] for x in dirs]))
    assert int(so["offsets"][-1]) == n
    np.testing.assert_array_equal(so["phase"], s["phase"])
    for q, x in enumerate(dirs):
        terms = np.concatenate([sr * d["rho"][q], sm * d["m"][q], sw * d["widths"][q]])
        ref, scale = float(terms.sum()), float(np.abs(terms).sum())
        got = float(grad_dot(b, g, x)[0])
        print(q, got, ref, scale)
        assert abs(got - ref) <= TOL_TANGENT * scale, (q, got, ref, scale)


# central-difference steps (relative) and bars per parameter kind. The oracle's own central differences
# against its own exact tangent (same code, same run) show the floor of the measurement on this loss:
# momentum derivatives at step 1e-6 are off by up to 2e-4 (round-off of the final states, ~1e-16 rho,
# times the misfit, against a loss change of ~1e-11), at 1e-5 by up to 1.5e-5; tau at 1e-6 by up to
# 9e-5 (its effect on the states is ~1e-7 relative), at 1e-4 by < 1e-6; density at 1e-6 by < 1e-5.
FD_STEP = {"tau": 1e-4, "rho": 1e-6, "m": 1e-5}
FD_BAR = {"tau": TOL_FD, "rho": TOL_FD, "m": 5e-5}


def fd_cases(b, g, rng, per_kind=3):
    """tau of every instance and, per instance and state kind, cells among those whose derivative is within a
    factor 10 of the instance's largest of that kind."""
    cases = [("tau", i, None) for i in range(b.n_inst)]
    for i in range(b.n_inst):
        a0, a1 = b.cell_offsets[i], b.cell_offsets[i + 1]
        for kind in ("rho", "m"):
            gk = np.abs(g[kind][a0:a1])
            cand = a0 + np.nonzero(gk >= 0.1 * gk.max())[0]
            for c in rng.choice(cand, min(per_kind, len(cand)), replace=False):
                cases.append((kind, i, int(c)))
    return cases


def test_adjoint_matches_central_differences():
    """dJ/dtau and dJ/d(rho, m) at sampled cells against central differences of the CUDA forward run, for
    every instance, with the steps and bars of FD_STEP / FD_BAR (the measurement's own floor, see above);
    the median error over all cases must also meet 1e-5."""
    program = [("step", 150)]
    b = I.adjoint_batch(n_inst=4, n_lattice=120, n_steps=150)
    tgt, s, J, g, info, stats = _grad(b, program)
    cases = fd_cases(b, g, np.random.default_rng(11))
    from paper_2211_00705_gb300.imexds import Imexds
    from paper_2211_00705_gb300.inputs import sample_density
    h = np.repeat((b.x_right - b.x_left) / b.n_lattice, b.n_lattice)
    inst = np.repeat(np.arange(b.n_inst), b.n_lattice)
    errs = []
    for kind, i, c in cases:
        vals = []
        for sgn in (+1, -1):
            bb = dataclasses.replace(b, tau=b.tau.copy(), rho=b.rho.copy(), m=b.m.copy())
            if kind == "tau":
                eps = FD_STEP[kind] * b.tau[i]
                bb.tau[i] += sgn * eps
            elif kind == "rho":
                eps = FD_STEP[kind] * b.rho[c]
                bb.rho[c] += sgn * eps
            else:
                eps = FD_STEP[kind] * max(abs(b.m[c]), b.rho[c])
                bb.m[c] += sgn * eps
            ctx = Imexds.from_batch(bb)
            ctx.step(150)
            ss = ctx.get_states()
            ctx.close()
            vals.append(sample_density(ss, ss["offsets"], b.n_lattice, b.x_left, b.x_right)[0])
        # J(+) - J(-) = 1/2 h sum (rho+ - rho-)(rho+ + rho- - 2 rho_tgt): the state difference is formed
        # first, so the difference of two nearly equal losses does not cancel digits
        sel = inst == i
        dp, sm_ = vals[0][sel] - vals[1][sel], vals[0][sel] + vals[1][sel] - 2.0 * tgt[sel]
        fd = float(np.sum(0.5 * h[sel] * dp * sm_)) / (2 * eps)
        ad = g["tau"][i] if kind == "tau" else g[kind][c]
        err = abs(fd - ad) / abs(ad)
        print(kind, i, c, ad, fd, err)
        assert err <= FD_BAR[kind], (kind, i, c, ad, fd, err)
        errs.append(err)
    assert np.median(errs) <= TOL_FD


def test_autograd_function():
    """torch.autograd.Function over the library: the gradient of the misfit through backward() is the
    adjoint's. Inputs, outputs and gradients are CUDA tensors passed to the device-resident calls; a second
    call reuses the RunSpec's context and gives the same gradients."""
    import torch
    from paper_2211_00705_gb300.autograd import ImexdsFunction, RunSpec
    program = [("step", 60)]
    b = I.adjoint_batch(n_inst=3, n_lattice=100, n_steps=60)
    tgt, s, J, g, info, stats = _grad(b, program)
    spec = RunSpec(b.n_lattice, b.x_left, b.x_right, b.cell_offsets, b.widths, b.phase, b.fluid, b.options,
                   program, checkpoint_every=16)
    dev = torch.device("cuda", 0)
    grads = []
    for _ in range(2):
        rho0 = torch.tensor(b.rho, device=dev, requires_grad=True)
        m0 = torch.tensor(b.m, device=dev, requires_grad=True)
        tau = torch.tensor(b.tau, device=dev, requires_grad=True)
        rT, mT = ImexdsFunction.apply(rho0, m0, tau, spec)
        assert rT.is_cuda and mT.is_cuda
        st = {"offsets": spec.last_offsets, "widths": spec.last_widths.cpu().numpy(),
              "rho": rT.detach().cpu().numpy()}
        _, gr = misfit(st, tgt, b)
        (rT * torch.tensor(gr, device=dev)).sum().backward()
        assert rho0.grad.is_cuda
        np.testing.assert_allclose(rho0.grad.cpu().numpy(), g["rho"], rtol=0, atol=1e-14 * np.max(np.abs(g["rho"])))
        np.testing.assert_allclose(m0.grad.cpu().numpy(), g["m"], rtol=0, atol=1e-14 * np.max(np.abs(g["m"])))
        np.testing.assert_allclose(tau.grad.cpu().numpy(), g["tau"], rtol=1e-14)
        grads.append((rho0.grad.cpu().numpy(), m0.grad.cpu().numpy(), tau.grad.cpu().numpy()))
    for a, c in zip(grads[0], grads[1]):
        np.testing.assert_array_equal(a, c)


def test_device_resident_calls_match_the_host_ones():
    """imexds_get_states_device and imexds_adjoint_device against imexds_get_states and imexds_adjoint on a run
    with splits, merges and created cells (cavitation): the same cell lists and the same gradients, bit for bit
    (the same kernels; only the staging differs), widths included."""
    import torch
    from paper_2211_00705_gb300.imexds import Imexds
    b = I.cavitation_batch(4, 4, n_range=(64, 128), n_steps=60)
    b = dataclasses.replace(b, options=I.scaled_options(creation=1, tol_nb=3e-13, tol_k=3e-11))
    ctx = Imexds.from_batch(b)
    ctx.set_adjoint_checkpoint(16)
    ctx.step(60)
    s = ctx.get_states()
    assert (ctx.stats()["creations"] >= 1).all()
    dev = torch.device("cuda", 0)
    n = int(s["offsets"][-1])
    wd, rd, md = (torch.empty(n, dtype=torch.float64, device=dev) for _ in range(3))
    phd = torch.empty(n, dtype=torch.uint8, device=dev)
    sd = ctx.get_states_device(wd, rd, md, phd)
    np.testing.assert_array_equal(sd["offsets"], s["offsets"])
    np.testing.assert_array_equal(sd["t"], s["t"])
    np.testing.assert_array_equal(wd.cpu().numpy(), s["widths"])
    np.testing.assert_array_equal(rd.cpu().numpy(), s["rho"])
    np.testing.assert_array_equal(md.cpu().numpy(), s["m"])
    np.testing.assert_array_equal(phd.cpu().numpy(), s["phase"])
    rng = np.random.default_rng(4)
    sr, sm, sw = rng.standard_normal(n), rng.standard_normal(n), rng.standard_normal(n)
    g = ctx.adjoint(sr, sm, sw)
    n0 = int(b.cell_offsets[-1])
    out = [torch.empty(n0, dtype=torch.float64, device=dev) for _ in range(3)]
    out_t = torch.empty(b.n_inst, dtype=torch.float64, device=dev)
    t = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    st = ctx.adjoint_device(t(sr), t(sm), out[0], out[1], out_t, dJ_dw_T=t(sw), out_w=out[2])
    ctx.close()
    assert (st == 0).all() and (g["status"] == 0).all()
    np.testing.assert_array_equal(out[0].cpu().numpy(), g["rho"])
    np.testing.assert_array_equal(out[1].cpu().numpy(), g["m"])
    np.testing.assert_array_equal(out[2].cpu().numpy(), g["widths"])
    np.testing.assert_array_equal(out_t.cpu().numpy(), g["tau"])


def test_adjoint_segments_do_not_change_the_gradient():
    """Checkpoint intervals 7, 45 (two segments that end with the run), 90 and 1000 (one segment) give the same
    gradient bit for bit. The last segment is taped during the replay and not recomputed; the others are
    recomputed from their checkpoints; with one segment the adjoint is one taped replay and the reverse sweep."""
    program = [("step", 90)]
    b = I.adjoint_batch(n_inst=3, n_lattice=100, n_steps=90)
    _, _, _, g1, _, _ = _grad(b, program, k=7)
    for k in (45, 90, 1000):
        _, _, _, g2, _, _ = _grad(b, program, k=k)
        for key in ("rho", "m", "widths", "tau"):
            np.testing.assert_array_equal(g1[key], g2[key], err_msg=f"k={k} {key}")


def test_adjoint_run_to_clipped_last_step():
    """run_to: the last step of each instance is shortened to land on t_end, so t^n enters that step's dt;
    the adjoint carries it back (checked against the oracle tangent)."""
    b = I.adjoint_batch(n_inst=4, n_lattice=100, n_steps=0)
    b = dataclasses.replace(b, t_end=3.3e-5)
    program = [("run_to", 3.3e-5)]
    tgt, s, J, g, info, stats = _grad(b, program)
    assert (g["status"] == 0).all()
    dirs = directions(b, n_rand=2)
    ref = _oracle_dirs(b, program, tgt, dirs)
    for q, d in enumerate(dirs):
        got = grad_dot(b, g, d)
        err = _rel(got, ref[q], np.max(np.abs(ref[q])))
        assert np.max(err) <= TOL_TANGENT, (q, got, ref[q])


def _mean_pressure(st, b):
    """J_i = sum_c w_c p(rho_c) / sum_c w_c over the final cells of instance i; gradients w.r.t. rho and w."""
    f = b.fluid
    off = st["offsets"]
    J = np.zeros(b.n_inst)
    gr = np.zeros(int(off[-1]))
    gw = np.zeros(int(off[-1]))
    for i in range(b.n_inst):
        sl = slice(off[i], off[i + 1])
        ph, r, w = st["phase"][sl], st["rho"][sl], st["widths"][sl]
        a2 = np.where(ph == 0, f.a2_vap, f.a2_liq)
        p = np.where(ph == 0, f.a2_vap * r, f.p_sat + f.a2_liq * (r - f.rho0_liq))
        W = w.sum()
        J[i] = float((w * p).sum() / W)
        gr[sl] = w * a2 / W
        gw[sl] = (p - J[i]) / W
    return J, gr, gw


@pytest.mark.parametrize("kind", ["cavitation", "nucleation"])
def test_adjoint_through_phase_creation_dJ_dV(kind):
    """Phase creation (App. B): liquid pulled apart at +-V creates a vapour cell (cavitation), vapour driven
    together at +-V nucleates a liquid cell (nucleation). dJ/dV of the mean final pressure (V enters the
    initial momentum, m0 = rho0 (-+V)) from the adjoint against the oracle's tangent in the V direction and
    against central differences of the CUDA forward run. Step 1e-6 relative for cavitation; 1e-4 for
    nucleation, whose created liquid cell carries its solves' stop-test noise into J amplified by a_L^2
    (central differences of the oracle's J reach the tangent to 5e-8 at 1e-4 and only to 1e-5 at 1e-6)."""
    from paper_2211_00705_gb300.imexds import Imexds
    if kind == "cavitation":
        b = I.cavitation_batch(4, 4, n_range=(64, 128), n_steps=60)
    else:
        b = I.nucleation_batch(5, 4, n_range=(64, 128), n_steps=60)
    b = dataclasses.replace(b, options=I.scaled_options(creation=1, tol_nb=3e-13, tol_k=3e-11))
    program = [("step", 60)]
    ctx = _forward(b, program)
    s = ctx.get_states()
    st = ctx.stats()
    assert (s["status"] == 0).all() and (st["creations"] >= 1).all()
    J, gr, gw = _mean_pressure(s, b)
    g = ctx.adjoint(gr, np.zeros_like(gr), gw)
    info = ctx.adjoint_info()
    ctx.close()
    assert (g["status"] == 0).all(), g["status"]
    assert info["replay_err"] <= 1e-9, info
    dmdV = np.zeros(int(b.cell_offsets[-1]))
    V = np.zeros(b.n_inst)
    for i in range(b.n_inst):
        sl = slice(b.cell_offsets[i], b.cell_offsets[i + 1])
        u = b.m[sl] / b.rho[sl]
        V[i] = abs(u[0])
        dmdV[sl] = np.sign(u) * b.rho[sl]
    adj = np.array([np.dot(g["m"][b.cell_offsets[i]:b.cell_offsets[i + 1]],
                           dmdV[b.cell_offsets[i]:b.cell_offsets[i + 1]]) for i in range(b.n_inst)])
    o = P.Oracle(b)
    sto, d = o.tangent(program, seed_m=dmdV[None, :], threads=4)
    Jo, gro, gwo = _mean_pressure(sto, b)
    off = sto["offsets"]
    tang = np.array([np.dot(gro[off[i]:off[i + 1]], d["rho"][0][off[i]:off[i + 1]])
                     + np.dot(gwo[off[i]:off[i + 1]], d["widths"][0][off[i]:off[i + 1]]) for i in range(b.n_inst)])
    print("adjoint", adj, "tangent", tang)
    assert np.max(np.abs(adj - tang) / np.abs(tang)) <= TOL_TANGENT
    eps = 1e-6 if kind == "cavitation" else 1e-4
    vals = []
    for sgn in (1.0, -1.0):
        bb = dataclasses.replace(b, m=b.m + sgn * eps * np.repeat(V, np.diff(b.cell_offsets)) * dmdV)
        c = Imexds.from_batch(bb)
        c.step(60)
        vals.append(_mean_pressure(c.get_states(), bb)[0])
        c.close()
    fd = (vals[0] - vals[1]) / (2 * eps * V)
    print("fd", fd)
    assert np.max(np.abs(adj - fd) / np.abs(adj)) <= 1e-5
