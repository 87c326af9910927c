"""The group kernel's per-phase SM cycle counters (timing mode) are consistent: for the slowest group the
boundary solves + plan, the concurrent phase (sweep beside the block solves) and the grid management add up to
the launch's own cycles, the sweep and the block solves each fit inside the concurrent phase, and the launch's
cycles over its event-timed duration give an SM clock rate."""
import numpy as np
import pytest

from paper_2211_00705_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("block_solver", [0, 1], ids=["dual-time", "newton"])
def test_group_phase_cycles_add_up(block_solver):
    import dataclasses
    from paper_2211_00705_gb300.imexds import Imexds
    b = I.workload(1, scale=64 / 4096)
    b = dataclasses.replace(b, options=dataclasses.replace(b.options, block_solver=block_solver))
    ctx = Imexds.from_batch(b, schedule=2)
    ctx.set_kernel_timing(True)
    ctx.run_to(b.t_end)
    ph = ctx.group_phase_cycles()["slowest"]
    ms, n = ctx.kernel_times()["k_group"]
    assert (ctx.get_states()["status"] == 0).all()
    ctx.close()
    assert n == 1 and ph["launch"] > 0
    total = ph["plan"] + ph["concurrent"] + ph["post"]
    assert abs(total - ph["launch"]) <= 0.02 * ph["launch"], ph
    assert ph["sweep"] <= 1.01 * ph["concurrent"] and ph["block_solve"] <= 1.01 * ph["concurrent"], ph
    ghz = ph["launch"] / (ms * 1e-3) / 1e9
    assert 0.8 < ghz < 2.2, (ghz, ph, ms)
