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
