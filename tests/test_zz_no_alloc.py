"""The entry point that allocates no GPU memory (imexds_step_uniform_noalloc), for callers that cannot
call cudaMalloc, against the regular context entry point (imexds_step) on the same single-phase
instances: two calls in a row, each compared with one step of the context path; then the checks it makes
on its device inputs (bad phase bytes, densities and momenta, mixed-phase instances), which must reject the
call without writing the outputs and leave the next call unaffected.

This file sorts last so that a run stopping at the first failure has run every other test first."""
import numpy as np
import pytest

from paper_2211_00705_gb300 import inputs as I
from tests.parity import TOL

pytestmark = pytest.mark.gpu


def _single_phase_batch():
    rng = np.random.default_rng(11)
    fluid = I.workload_fluid()
    ns = [100, 333, 1000, 64]   # 64: the last lane of a tile takes the domain end (N divisible by 32)
    widths, rho, m, phase = [], [], [], []
    for k, n in enumerate(ns):
        x = (np.arange(n) + 0.5) / n
        if k == 1:   # vapour instance
            r = 0.6 + 0.2 * np.sin(2 * np.pi * x) + 0.05 * rng.random(n)
            ph = np.zeros(n, np.uint8)
        else:        # liquid instances
            r = 970.0 + 20.0 * np.sin(2 * np.pi * x) + rng.random(n)
            ph = np.ones(n, np.uint8)
        u = 30.0 * np.cos(3 * np.pi * x) + rng.uniform(-5, 5, n)
        widths.append(np.full(n, 1.0 / n))
        rho.append(r)
        m.append(r * u)
        phase.append(ph)
    off = np.zeros(len(ns) + 1, np.int32)
    off[1:] = np.cumsum(ns)
    return I.Batch(n_lattice=np.array(ns, np.int32), x_left=np.zeros(len(ns)), x_right=np.ones(len(ns)),
                   tau=np.full(len(ns), I.tau_paper()), cell_offsets=off, widths=np.concatenate(widths),
                   rho=np.concatenate(rho), m=np.concatenate(m), phase=np.concatenate(phase), fluid=fluid,
                   options=I.Options(), t_end=0.0, n_steps=1, name="single-phase instances")


def test_no_alloc_step_matches_context_step_twice():
    torch = pytest.importorskip("torch")
    from paper_2211_00705_gb300.imexds import Imexds, step_uniform_noalloc
    b = _single_phase_batch()
    ctx = Imexds.from_batch(b)
    ref = []
    for _ in range(2):
        ctx.step(1)
        ref.append(ctx.get_states())
    ctx.close()
    dev = torch.device("cuda", 0)
    r = torch.tensor(b.rho, dtype=torch.float64, device=dev)
    m = torch.tensor(b.m, dtype=torch.float64, device=dev)
    ph = torch.tensor(b.phase, dtype=torch.uint8, device=dev)
    t = np.zeros(b.n_inst)
    for call in range(2):
        r_out = torch.empty_like(r)
        m_out = torch.empty_like(m)
        dt = torch.empty(b.n_inst, dtype=torch.float64, device=dev)
        step_uniform_noalloc(b.fluid, b.options.cfl, b.n_lattice, b.x_left, b.x_right, r, m, ph, r_out, m_out, dt)
        torch.cuda.synchronize()
        s = ref[call]
        rr, mm = r_out.cpu().numpy(), m_out.cpu().numpy()
        for k in range(b.n_inst):
            a0, a1 = s["offsets"][k], s["offsets"][k + 1]
            assert np.max(np.abs(rr[a0:a1] - s["rho"][a0:a1])) <= TOL * np.max(np.abs(s["rho"][a0:a1]))
            mscale = max(np.max(np.abs(s["m"][a0:a1])), np.max(np.abs(s["rho"][a0:a1])))
            assert np.max(np.abs(mm[a0:a1] - s["m"][a0:a1])) <= TOL * mscale
        t += dt.cpu().numpy()
        np.testing.assert_allclose(t, s["t"], rtol=1e-14)
        r, m = r_out, m_out


def test_no_alloc_rejects_bad_device_inputs():
    """Inputs the kernels check on the device (the host never sees them): a phase byte above 1, a density
    that is not positive, a non-finite momentum, an instance with cells of both phases. Each call returns
    IMEXDS_ERR_ARG with its reason, leaves rho_out and m_out unwritten, and the next valid call on the same
    scratch gives the same result as a first call."""
    torch = pytest.importorskip("torch")
    from paper_2211_00705_gb300.imexds import ImexdsError, last_error, step_uniform_noalloc
    b = _single_phase_batch()
    dev = torch.device("cuda", 0)

    def call(rho, m, ph):
        """One call into outputs filled with -7; returns the outputs (host copies) and the error, if any."""
        r_out = torch.full_like(rho, -7.0)
        m_out = torch.full_like(m, -7.0)
        dt = torch.empty(b.n_inst, dtype=torch.float64, device=dev)
        err = None
        try:
            step_uniform_noalloc(b.fluid, b.options.cfl, b.n_lattice, b.x_left, b.x_right, rho, m, ph, r_out, m_out,
                                 dt)
        except ImexdsError as e:
            err = str(e)
        torch.cuda.synchronize()
        return (r_out.cpu().numpy(), m_out.cpu().numpy(), dt.cpu().numpy()), err

    r = torch.tensor(b.rho, dtype=torch.float64, device=dev)
    m = torch.tensor(b.m, dtype=torch.float64, device=dev)
    ph = torch.tensor(b.phase, dtype=torch.uint8, device=dev)
    good, err = call(r, m, ph)
    assert err is None, err
    k = int(b.cell_offsets[2]) + 5   # a cell of the third instance
    ph2 = ph.clone()
    ph2[k] = 2
    r2 = r.clone()
    r2[k] = -1.0
    m2 = m.clone()
    m2[k] = float("nan")
    ph3 = ph.clone()
    ph3[k] = 1 - int(b.phase[k])
    for name, rr, mm, pp in [("phase byte", r, m, ph2), ("density", r2, m, ph), ("momentum", r, m2, ph),
                             ("both phases", r, m, ph3)]:
        out, err = call(rr, mm, pp)
        assert err is not None and "status 1 " in err, (name, err)
        assert "not written" in last_error(), (name, last_error())
        assert (out[0] == -7.0).all() and (out[1] == -7.0).all(), name   # a rejected call writes no state
    again, err = call(r, m, ph)
    assert err is None, err
    for x, y in zip(good, again):
        np.testing.assert_array_equal(x, y)
