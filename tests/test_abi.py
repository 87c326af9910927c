"""The C-ABI library builds for sm_103a, loads and exports every function declared in include/imexds.h.
No device calls (runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "imexds.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(imexds_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2211_00705_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "imexds_create" in names and "imexds_run_to" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_lists_every_declared_symbol():
    from paper_2211_00705_gb300 import imexds
    assert sorted(imexds.EXPORTED) == declared_functions()


def test_status_strings_without_device(lib):
    lib.imexds_status_string.restype = ctypes.c_char_p
    assert lib.imexds_status_string(0) == b"ok"
    assert b"capacity" in lib.imexds_status_string(9)


def _problem(**kw):
    """A valid two-instance problem (the workload fluid and options), fields overridable."""
    import numpy as np
    from paper_2211_00705_gb300 import inputs as I
    p = dict(n_lattice=np.array([40, 60]), x_left=np.zeros(2), x_right=np.ones(2), tau=np.full(2, 1e-7),
             fluid=I.workload_fluid(), options=I.Options())
    p.update(kw)
    return p


@pytest.mark.parametrize("bad", [
    dict(n_lattice=[1, 60]),                      # fewer than two lattice cells
    dict(x_right=[1.0, 0.0]),                     # empty domain
    dict(tau=[1e-7, -1.0]),                       # negative kinetic coefficient
    dict(cfl=0.0), dict(l_max=0), dict(newton_itmax=0), dict(split_ratio=1.0),
    dict(schedule=4), dict(group_threads=48), dict(group_threads=288), dict(group_threads=100),
])
def test_create_rejects_malformed_problems(lib, bad):
    """imexds_create checks its arguments before any device call: IMEXDS_ERR_ARG on every malformed problem
    or option (runs without a GPU)."""
    import dataclasses
    import numpy as np
    from paper_2211_00705_gb300.imexds import Imexds, ImexdsError
    p = _problem()
    kw = {}
    for k, v in bad.items():
        if k in p:
            p[k] = np.asarray(v)
        elif k in ("schedule", "group_threads"):
            kw[k] = v
        else:
            p["options"] = dataclasses.replace(p["options"], **{k: v})
    with pytest.raises(ImexdsError, match=r"status 1 "):
        Imexds(p["n_lattice"], p["x_left"], p["x_right"], p["tau"], p["fluid"], p["options"], **kw)


def test_create_without_gpu_fails_loudly(lib):
    """No host fallback: on a machine without a GPU a valid problem is refused with IMEXDS_ERR_CUDA."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2211_00705_gb300.imexds import Imexds, ImexdsError
    p = _problem()
    with pytest.raises(ImexdsError, match=r"status 2 "):
        Imexds(p["n_lattice"], p["x_left"], p["x_right"], p["tau"], p["fluid"], p["options"])


def test_binding_refuses_cell_lists_shorter_than_the_offsets():
    """The library reads offsets[n_inst] entries of every cell array: the binding checks the lengths first
    (host-side logic, no context needed)."""
    import numpy as np
    from paper_2211_00705_gb300.imexds import Imexds
    ctx = object.__new__(Imexds)
    ctx.n_inst = 2
    off = np.array([0, 3, 7], dtype=np.int32)
    ok = np.zeros(7)
    ctx._check_lists(off, [("widths", ok), ("rho", ok)])
    with pytest.raises(ValueError, match="rho has 6 entries"):
        ctx._check_lists(off, [("widths", ok), ("rho", ok[:6])])
    with pytest.raises(ValueError, match="offsets has 2 entries"):
        ctx._check_lists(off[:2], [("widths", ok[:3])])


class _FakeDevicePtr:
    """Stands in for a device tensor in calls that are rejected before any pointer is used."""

    def data_ptr(self):
        return 16


def test_noalloc_rejects_oversized_and_malformed_batches_before_any_device_call(lib):
    """The allocation-free step checks its host arguments first: more instances than its fixed scratch holds
    gives IMEXDS_ERR_CAPACITY, a malformed instance IMEXDS_ERR_ARG, each with its reason in
    imexds_last_error_string, and neither touches the (here fake) device pointers or needs a GPU."""
    import numpy as np
    from paper_2211_00705_gb300 import inputs as I
    from paper_2211_00705_gb300.imexds import ImexdsError, last_error, step_uniform_noalloc
    f = _FakeDevicePtr()
    n = 16385
    with pytest.raises(ImexdsError, match=r"status 9 "):
        step_uniform_noalloc(I.workload_fluid(), 0.5, np.full(n, 64), np.zeros(n), np.ones(n), f, f, f, f, f, f)
    assert "16384" in last_error()
    with pytest.raises(ImexdsError, match=r"status 1 "):
        step_uniform_noalloc(I.workload_fluid(), 0.5, np.array([64, 1]), np.zeros(2), np.ones(2), f, f, f, f, f, f)
    assert "fewer than 2 cells" in last_error()
    with pytest.raises(ImexdsError, match=r"status 1 "):
        step_uniform_noalloc(I.workload_fluid(), 0.5, np.array([64, 64]), np.zeros(2), np.array([1.0, 0.0]),
                             f, f, f, f, f, f)
    assert "x_right <= x_left" in last_error()
