"""C-ABI argument checks that need a context (and so a GPU): imexds_set_states rejects malformed cell lists
with IMEXDS_ERR_ARG and leaves the states it had loaded as they were."""
import numpy as np
import pytest

from paper_2211_00705_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _malformed(b):
    """(name, overrides of the valid cell lists of batch b) for each kind of malformed list."""
    pad = lambda x: np.concatenate([x[:1], x])   # one leading cell that the shifted offsets skip
    cases = [("first offset not 0", dict(offsets=b.cell_offsets + 1, widths=pad(b.widths), rho=pad(b.rho),
                                         m=pad(b.m), phase=pad(b.phase)))]
    m = b.m.copy()
    m[3] = np.nan
    cases.append(("NaN momentum", dict(m=m)))
    m = b.m.copy()
    m[3] = np.inf
    cases.append(("infinite momentum", dict(m=m)))
    r = b.rho.copy()
    r[0] = np.inf
    cases.append(("infinite density", dict(rho=r)))
    r = b.rho.copy()
    r[0] = -1.0
    cases.append(("negative density", dict(rho=r)))
    w = b.widths.copy()
    w[0] *= 1.5
    cases.append(("fixed face off the lattice", dict(widths=w)))
    ph = b.phase.copy()
    ph[0] = 2
    cases.append(("unknown phase", dict(phase=ph)))
    return cases


def test_set_states_rejects_malformed_lists_and_keeps_the_loaded_states():
    from paper_2211_00705_gb300.imexds import Imexds, ImexdsError
    b = I.workload(0)
    ctx = Imexds.from_batch(b)
    for name, over in _malformed(b):
        a = dict(offsets=b.cell_offsets, widths=b.widths, rho=b.rho, m=b.m, phase=b.phase)
        a.update(over)
        with pytest.raises(ImexdsError, match=r"status 1 "):
            ctx.set_states(a["offsets"], a["widths"], a["rho"], a["m"], a["phase"])
    # lists whose lengths disagree with the offsets are refused by the binding before the library reads them
    with pytest.raises(ValueError, match="rho"):
        ctx.set_states(b.cell_offsets, b.widths, b.rho[:-1], b.m, b.phase)
    # the context still holds the valid lists loaded first: 5 steps equal those of a fresh context
    ctx.step(5)
    s = ctx.get_states()
    ctx.close()
    ref = Imexds.from_batch(b)
    ref.step(5)
    r = ref.get_states()
    ref.close()
    for k in ("offsets", "widths", "rho", "m", "phase", "t", "status"):
        np.testing.assert_array_equal(s[k], r[k], err_msg=k)


def test_adjoint_checks_the_seed_lengths():
    """The binding refuses seeds whose length differs from the final cell lists (the library would read
    one entry per final cell)."""
    from paper_2211_00705_gb300.imexds import Imexds
    b = I.adjoint_batch(n_inst=2, n_lattice=60, n_steps=10)
    ctx = Imexds.from_batch(b)
    ctx.set_adjoint_checkpoint(4)
    ctx.step(10)
    n = int(ctx.cell_counts().sum())
    with pytest.raises(ValueError, match="dJ_drho_T"):
        ctx.adjoint(np.zeros(n - 1), np.zeros(n))
    with pytest.raises(ValueError, match="dJ_dw_T"):
        ctx.adjoint(np.zeros(n), np.zeros(n), np.zeros(n + 1))
    g = ctx.adjoint(np.ones(n), np.zeros(n))
    ctx.close()
    assert (g["status"] == 0).all()


def _collapsing_bubble(fl, N=40, V=100.0):
    """Liquid converging at +-V onto a vapour cell of half a lattice cell between two boundaries: the cell
    between the two boundaries would vanish (IMEXDS_ERR_VANISH in the oracle, at step 6)."""
    h = 1.0 / N
    widths = np.array([h] * 19 + [0.5 * h, 0.5 * h, h] + [h] * (N - 21))
    phase = np.array([1] * 20 + [0] + [1] * (N - 20), np.uint8)
    rho = np.where(phase == 1, 1000.0, fl.p_sat / fl.a2_vap)
    x = np.cumsum(widths) - widths / 2
    m = rho * np.where(x < 0.5, V, -V)
    return I.Batch(n_lattice=np.array([N], np.int32), x_left=np.zeros(1), x_right=np.ones(1),
                   tau=np.array([I.tau_paper()]), cell_offsets=np.array([0, len(widths)], np.int32), widths=widths,
                   rho=rho, m=m, phase=phase, fluid=fl, options=I.scaled_options(), t_end=0.0, n_steps=40,
                   name="collapsing bubble")


def _concat(parts):
    """One batch holding the instances of single-instance batches (same fluid and options)."""
    off = np.zeros(len(parts) + 1, np.int32)
    off[1:] = np.cumsum([p.cell_offsets[-1] for p in parts])
    cat = lambda f: np.concatenate([getattr(p, f) for p in parts])
    return I.Batch(n_lattice=cat("n_lattice"), x_left=cat("x_left"), x_right=cat("x_right"), tau=cat("tau"),
                   cell_offsets=off, widths=cat("widths"), rho=cat("rho"), m=cat("m"), phase=cat("phase"),
                   fluid=parts[0].fluid, options=parts[0].options, t_end=0.0, n_steps=parts[0].n_steps)


def _with_a_failing_instance():
    fl = I.workload_fluid(rho0_liq=1000.0)
    r = I.riemann_batch(7, 2, n_range=(60, 90), alpha_range=(1e-3, 1e-2), fluid=fl, options=I.scaled_options(),
                        t_end=0.0, n_steps=40)
    return _concat([r.subset([0]), _collapsing_bubble(fl), r.subset([1])]), _concat([r.subset([0]), r.subset([1])])


def test_an_instance_that_fails_stops_alone():
    """Fault isolation on data: an instance driven into an error (a vanishing cell between two boundaries)
    stops with its status, the call returns IMEXDS_OK, and the other instances of the batch end exactly as
    in a batch without it."""
    from paper_2211_00705_gb300.imexds import Imexds
    b3, b2 = _with_a_failing_instance()
    c3 = Imexds.from_batch(b3)
    c3.step(40)
    s3 = c3.get_states()
    c3.close()
    c2 = Imexds.from_batch(b2)
    c2.step(40)
    s2 = c2.get_states()
    c2.close()
    assert s3["status"][1] != 0 and s3["status"][0] == 0 and s3["status"][2] == 0
    for k, j in ((0, 0), (2, 1)):
        a = slice(s3["offsets"][k], s3["offsets"][k + 1])
        b = slice(s2["offsets"][j], s2["offsets"][j + 1])
        for f in ("widths", "rho", "m", "phase"):
            np.testing.assert_array_equal(s3[f][a], s2[f][b], err_msg=f"instance {k}: {f}")
        assert s3["t"][k] == s2["t"][j]


def test_forced_caps_report_through_status_and_counters():
    """Caps forced by the options (no GPU fault): one Newton iteration cannot converge a boundary solve from
    its cold start, so every instance stops with IMEXDS_ERR_PB_NOCONV while the call returns IMEXDS_OK; one
    dual-time iteration per step ends every step on the cap, which is counted (maxiter) and is not an
    error (reading R18). The oracle gives the same statuses and counters."""
    import dataclasses
    from paper_2211_00705_gb300.imexds import Imexds
    b = I.riemann_batch(8, 3, n_range=(60, 90), alpha_range=(1e-3, 1e-2), options=I.scaled_options(), t_end=0.0,
                        n_steps=10)
    c = Imexds.from_batch(dataclasses.replace(b, options=dataclasses.replace(b.options, newton_itmax=1)))
    c.step(10)
    assert (c.get_states()["status"] == 4).all()
    c.close()
    c = Imexds.from_batch(dataclasses.replace(b, options=dataclasses.replace(b.options, l_max=1)))
    c.step(10)
    s, st = c.get_states(), c.stats()
    c.close()
    assert (s["status"] == 0).all() and (st["steps"] == 10).all()
    assert (st["maxiter"] >= st["steps"]).all() and (st["dts_iters"] == st["steps"]).all()


def test_set_states_again_with_the_same_or_another_layout():
    """imexds_set_states on a loaded context: with the layout of the loaded states it keeps the device buffers,
    with another number of boundaries (other zone slots) it allocates anew. Either way the run that follows is
    bit for bit the run of a fresh context on the same states."""
    from paper_2211_00705_gb300.imexds import Imexds
    b = I.workload(1, scale=16 / 4096)
    N = b.n_lattice
    h = (b.x_right - b.x_left) / N
    off_u = np.concatenate([[0], np.cumsum(N)]).astype(np.int32)   # every instance one liquid phase, at rest
    w_u = np.repeat(h, N)
    uniform = dict(offsets=off_u, widths=w_u, rho=np.full(w_u.shape, 998.0), m=np.zeros(w_u.shape),
                   phase=np.ones(w_u.shape, np.uint8))
    riemann = dict(offsets=b.cell_offsets, widths=b.widths, rho=b.rho, m=b.m, phase=b.phase)

    def run(ctx, st):
        ctx.set_states(st["offsets"], st["widths"], st["rho"], st["m"], st["phase"])
        ctx.step(50)
        return ctx.get_states()

    def fresh(st):  # a context whose only imexds_set_states is this one
        ctx = Imexds(b.n_lattice, b.x_left, b.x_right, b.tau, b.fluid, b.options)
        s = run(ctx, st)
        ctx.close()
        return s

    ref_r, ref_u = fresh(riemann), fresh(uniform)
    ctx = Imexds.from_batch(b)   # loaded with the same layout: the first call below keeps the buffers
    got = [run(ctx, riemann), run(ctx, uniform), run(ctx, riemann), run(ctx, riemann)]
    ctx.close()
    for s, ref in zip(got, (ref_r, ref_u, ref_r, ref_r)):
        for key in ("offsets", "widths", "rho", "m", "phase", "t", "status"):
            np.testing.assert_array_equal(s[key], ref[key], err_msg=key)
    assert (ref_r["status"] == 0).all() and (ref_u["status"] == 0).all()
