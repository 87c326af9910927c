"""Helpers shared by the GPU parity tests: run a batch on the oracle and on the CUDA library and
compare cell lists instance by instance (relative L-infinity per conserved variable)."""
import numpy as np

from oracle import pyoracle as P

TOL = 1e-9   # relative L-infinity per conserved variable and instance
U_REF = 1.0  # m/s: momentum is normalised by max(|m|_inf, |rho|_inf * U_REF) (a fluid at rest has |m| ~ 0)


def run_oracle(batch, threads=8):
    o = P.Oracle(batch)
    assert o.set_rc == 0
    if batch.t_end > 0:
        o.run_to(batch.t_end, threads)
    else:
        o.step(batch.n_steps, threads)
    return o.states(), o.stats()


def run_gpu(batch, **kw):
    from paper_2211_00705_gb300.imexds import Imexds
    ctx = Imexds.from_batch(batch, **kw)
    if batch.t_end > 0:
        ctx.run_to(batch.t_end)
    else:
        ctx.step(batch.n_steps)
    s, st = ctx.get_states(), ctx.stats()
    ctx.close()
    return s, st


def compare(a, b, tol=TOL, skip_status=False):
    """Per-instance errors: returns list of dicts; raises AssertionError with details on mismatch."""
    n = len(a["t"])
    out = []
    for k in range(n):
        a0, a1 = a["offsets"][k], a["offsets"][k + 1]
        b0, b1 = b["offsets"][k], b["offsets"][k + 1]
        rec = {"inst": k, "status_a": int(a["status"][k]), "status_b": int(b["status"][k])}
        if not skip_status:
            assert a["status"][k] == b["status"][k], rec
        if a["status"][k] != 0 and b["status"][k] != 0:
            out.append(rec)   # both stopped with the same error; states after an error are not compared
            continue
        assert a1 - a0 == b1 - b0, (k, "cell counts", a1 - a0, b1 - b0)
        np.testing.assert_array_equal(a["phase"][a0:a1], b["phase"][b0:b1])
        ra, rb = a["rho"][a0:a1], b["rho"][b0:b1]
        ma, mb = a["m"][a0:a1], b["m"][b0:b1]
        wa, wb = a["widths"][a0:a1], b["widths"][b0:b1]
        rec["rho"] = float(np.max(np.abs(ra - rb)) / np.max(np.abs(ra)))
        rec["m"] = float(np.max(np.abs(ma - mb)) / max(np.max(np.abs(ma)), np.max(np.abs(ra)) * U_REF))
        rec["w"] = float(np.max(np.abs(wa - wb)) / np.max(wa))
        rec["t"] = float(abs(a["t"][k] - b["t"][k]))
        out.append(rec)
        assert rec["rho"] <= tol and rec["m"] <= tol and rec["w"] <= tol, rec
        assert rec["t"] <= 1e-15 * max(1.0, abs(a["t"][k])) * 1e3, rec
    return out
