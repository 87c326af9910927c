"""The entry point that allocates no GPU memory (imexds_step_uniform_noalloc), for callers that cannot
call cudaMalloc, against the regular context entry point (imexds_step) on the same single-phase
instances: two calls in a row, each compared with one step of the context path.

This file sorts last so that a run stopping at the first failure has run every other test first."""
import numpy as np
import pytest

from paper_2211_00705_gb300 import inputs as I
from tests.parity import TOL

pytestmark = pytest.mark.gpu


def _single_phase_batch():
    rng = np.random.default_rng(11)
    fluid = I.workload_fluid()
    ns = [100, 333, 1000]
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
