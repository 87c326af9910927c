"""Newton on the implicit blocks (the paper's outlook, Sec. 5) at the floor that rounding puts under the Sec. 4
residual, in the oracle. For a tiny cell of fraction alpha the update T amplifies a one-ulp change of the iterate
by about 1/alpha, so a stop tolerance can lie below every residual double precision can reach; the iterate then
cycles among points a few ulps apart. The iteration ends there by its floor rules (correction below 1e-14 of the
iterate, or corrections at most 1e-10 that no longer contract), as l_max would end it, and must not end early
where the test can be met."""
import dataclasses

import numpy as np

from oracle import pyoracle as P
from paper_2211_00705_gb300 import inputs as I
from tests.parity import compare


def _newton(batch, **opts):
    return dataclasses.replace(batch, options=dataclasses.replace(batch.options, block_solver=1, **opts))


def _run(batch, n_steps):
    o = P.Oracle(batch)
    o.step(n_steps, 8)
    return o.states(), o.stats()


def test_newton_ends_at_the_rounding_floor_in_a_few_steps():
    """16 Riemann instances (alpha in [1e-6, 1e-1]), 40 steps, with tolerances 1e-18 (no residual in double
    precision is that small) and l_max = 200: every block ends by the floor rules within a few Newton steps,
    and the states equal those of the workload's own tolerances (which the iteration meets) to 1e-9."""
    b = I.workload(1, scale=16 / 4096)
    ref, st_ref = _run(_newton(b), 40)
    s, st = _run(_newton(b, tol_nb=1e-18, tol_k=1e-18, l_max=200), 40)
    assert (st_ref["maxiter"] == 0).all()               # the floor rules do not end a block that can converge
    assert (st["maxiter"] > 0).all()                     # the 1e-18 test is never met ...
    assert int(st["dts_max"].max()) <= 8, st["dts_max"]  # ... and no block iterates on to l_max
    # every block-step ended by a floor rule: the iterations per block-step stay a few
    assert float(st["dts_iters"].sum()) <= 6.0 * float(st["maxiter"].sum())
    compare(ref, s)


def test_tight_tolerances_of_the_adjoint_workload_reach_the_floor_rules_only_in_a_few_blocks():
    """The adjoint workload's tolerances (the scaled ones x 1e-4: 3e-13 and 3e-11) lie near the floor: 64 of its
    instances, 200 steps. Newton needs at most a handful of steps per block; the blocks that end by the floor
    rules are rare; the states equal the dual-time ones (Alg. 2 at the same tolerances) to 1e-9."""
    b = I.adjoint_batch(n_inst=64, n_steps=200)
    sn, stn = _run(_newton(b), 200)
    sd, std = _run(b, 200)
    assert int(stn["dts_max"].max()) <= 8, stn["dts_max"]
    assert float(stn["maxiter"].sum()) <= 1e-3 * float(stn["dts_iters"].sum())
    compare(sd, sn)
