"""Newton's method on each implicit block (options.block_solver = 1; the paper's outlook, Sec. 5) on the CUDA
path against the oracle's Newton option, element by element (relative L-infinity per conserved variable and
instance <= 1e-9, identical cell lists and grid events), on every workload shape and schedule; the iteration
counts against the oracle's and against dual time; and the adjoint of a Newton run.

Both Newton iterations stop on the same test (the Sec. 4 residual of the iterate) and take the same steps up to
rounding: both use the exact Jacobian, the CUDA path by the implicit function theorem at the boundary and HLL in
closed form, the oracle by forward-mode dual numbers of its block update. (With a central-difference Jacobian in
the oracle, the two iterations landed at different points inside the stop tolerance: on the bubble domain the
oracle disagreed with itself by 2.6e-8 between difference steps of 1e-7 and 1e-8.) The states are held to the
1e-9 parity bar and the Newton-step counts to 1 % (plus two)."""
import dataclasses

import numpy as np
import pytest

from paper_2211_00705_gb300 import inputs as I
from tests.parity import compare, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

SCHEDULES = [pytest.param(1, id="per-step-kernels"), pytest.param(2, id="instance-groups"),
             pytest.param(3, id="independent-instance-groups")]


def newton(batch):
    return dataclasses.replace(batch, options=dataclasses.replace(batch.options, block_solver=1))


def _check(batch, **kw):
    b = newton(batch)
    a, sa = run_oracle(b)
    g, sg = run_gpu(b, **kw)
    recs = compare(a, g)
    for k in ("steps", "merges", "splits", "creations"):
        np.testing.assert_array_equal(sa[k], sg[k], err_msg=k)
    ia, ig = float(sa["dts_iters"].sum()), float(sg["dts_iters"].sum())
    # where a residual sits at the stop tolerance, the two roundings decide whether one more Newton step is taken
    assert abs(ia - ig) <= 0.02 * ia + 2, (ia, ig)
    # no block runs on to l_max; a block may end at the rounding floor (the floor rules of the block Newton
    # iteration), which the two implementations' roundings reach in different blocks, rarely
    assert int(sg["dts_max"].max()) <= 8, sg["dts_max"]
    assert float(sg["maxiter"].sum()) <= 0.01 * ig, (float(sg["maxiter"].sum()), ig)
    return recs, sa, sg


def test_single_instance_workload():
    """One Riemann instance (N = 100, alpha = 1e-3) to t_end with the printed residual."""
    _, sa, sg = _check(I.workload(0))
    # about one and a half Newton steps per time step, where dual time takes ~31 iterations
    steps = float(sg["steps"].sum())
    assert float(sg["dts_iters"].sum()) / steps < 3.0


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_batched_riemann_subset(schedule):
    """32 instances of the batched Riemann workload (N in [200, 2000], alpha in [1e-6, 1e-1]) to t_end."""
    _check(I.workload(1, scale=32 / 4096), schedule=schedule)


def test_batched_riemann_subset_wide_groups():
    _check(I.workload(1, scale=32 / 4096), schedule=2, group_threads=256)


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_fixed_step_count(schedule):
    b = I.workload(3, scale=8 / 1024)
    b.n_steps = 300
    _check(b, schedule=schedule)


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_cavitation_creation(schedule):
    """A created vapour cell between two boundaries: blocks with two boundary faces (the general path)."""
    b = I.workload(4, scale=8 / 16384)
    b.n_steps = 200
    _, _, sg = _check(b, schedule=schedule)
    assert (sg["creations"] >= 1).all()


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_nucleation_creation(schedule):
    """A nucleated liquid cell (~1e-7 of a lattice cell at first): where dual time needs ~1e3 iterations."""
    b = I.nucleation_batch(5, 8, n_steps=200)
    _, _, sg = _check(b, schedule=schedule)
    assert (sg["creations"] >= 1).all()


def test_bubbles_small_domain():
    """Many boundaries in one domain, blocks of two boundaries joined (4096 cells, 64 bubbles)."""
    _check(I.bubbles_domain(2, n_cells=4096, n_bubbles=64, n_steps=60))


def test_newton_and_dual_time_reach_the_same_solution():
    """Both solvers solve one implicit system per block: on the CUDA path their results differ by the
    dual-time stop tolerance only (tight tolerances here: x 1e-4), while Newton takes far fewer iterations."""
    b = I.workload(1, scale=16 / 4096)
    b = dataclasses.replace(b, options=dataclasses.replace(b.options, tol_nb=b.options.tol_nb * 1e-4,
                                                           tol_k=b.options.tol_k * 1e-4))
    d, sd = run_gpu(b)
    n, sn = run_gpu(newton(b))
    compare(d, n, tol=1e-7)
    assert float(sn["dts_iters"].sum()) * 5 < float(sd["dts_iters"].sum())


def test_adjoint_of_a_newton_run():
    """The adjoint replays the forward run with the context's solver and differentiates the converged block
    systems (independent of the solver that converged them): a Newton run's gradient equals a dual-time run's
    on the adjoint workload (tight tolerances), and its replay reproduces the forward states."""
    from paper_2211_00705_gb300.imexds import Imexds
    from tests.adjoint_util import misfit, target_samples
    b = I.adjoint_batch(n_inst=4, n_lattice=100, n_steps=120)
    grads = []
    for bb in (b, newton(b)):
        tctx = Imexds.from_batch(dataclasses.replace(bb, tau=bb.tau * 1.1))
        tctx.step(bb.n_steps)
        tgt = target_samples(tctx.get_states(), bb)
        tctx.close()
        ctx = Imexds.from_batch(bb)
        ctx.set_adjoint_checkpoint(16)
        ctx.step(bb.n_steps)
        s = ctx.get_states()
        assert (s["status"] == 0).all()
        J, gr = misfit(s, tgt, bb)
        g = ctx.adjoint(gr, np.zeros_like(gr))
        info = ctx.adjoint_info()
        ctx.close()
        assert (g["status"] == 0).all(), g["status"]
        assert info["replay_err"] <= 1e-9, info
        grads.append(g)
    for key in ("rho", "m", "tau"):
        a, n = grads[0][key], grads[1][key]
        scale = np.max(np.abs(a))
        assert np.max(np.abs(a - n)) <= 1e-6 * scale, (key, np.max(np.abs(a - n)) / scale)


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_creation_at_a_face_inside_a_joined_zone(schedule):
    """Creation at a face between two explicit cells of a joined zone (see tests/test_parity_gpu.py), with
    Newton on the blocks around the created cells (a nucleated droplet is where dual time hits l_max)."""
    _, _, sg = _check(I.slab_creation_batch(n_steps=30), schedule=schedule)
    assert (sg["creations"] >= 1).all()
