"""ctypes wrapper of the CPU oracle (TEST INFRASTRUCTURE ONLY).

Only the tests, the smoke check and the CPU-baseline leg of the benchmark use this module.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


class OEos(C.Structure):
    _fields_ = [("kind", C.c_int), ("a2", C.c_double), ("p0", C.c_double), ("rho0", C.c_double)]


class OFluid(C.Structure):
    _fields_ = [("ph", OEos * 2), ("p_sat", C.c_double), ("p_min", C.c_double), ("p_tilde", C.c_double)]


class OOpts(C.Structure):
    _fields_ = [("cfl", C.c_double), ("theta_nb", C.c_double), ("tol_nb", C.c_double), ("tol_k", C.c_double),
                ("res_mode", C.c_int), ("l_max", C.c_int), ("newton_tol", C.c_double),
                ("newton_itmax", C.c_int), ("alpha_min", C.c_double), ("split_ratio", C.c_double),
                ("creation", C.c_int), ("block_solver", C.c_int)]


def lib():
    global _lib
    if _lib is None:
        # ORACLE_LIB: a library built from a modified copy of the oracle's source (the planted-mistake check of
        # tests/plant_mistakes.py); otherwise the oracle built from this directory
        path = os.environ.get("ORACLE_LIB") or _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.c_int, ip, dp, dp, dp, C.POINTER(OFluid), C.POINTER(OOpts)]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_set_states.argtypes = [C.c_void_p, ip, dp, dp, dp, C.POINTER(C.c_ubyte), C.c_double]
        L.orc_n_cells.argtypes = [C.c_void_p, ip]
        L.orc_get_states.argtypes = [C.c_void_p, ip, dp, dp, dp, C.POINTER(C.c_ubyte), dp, ip]
        L.orc_get_pbs.argtypes = [C.c_void_p, ip, dp]
        L.orc_get_stats.argtypes = [C.c_void_p, C.POINTER(C.c_longlong)]
        L.orc_run_to.argtypes = [C.c_void_p, C.c_double, C.c_int]
        L.orc_step.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.orc_explicit_run_to.argtypes = [C.c_void_p, C.c_double, C.c_int]
        L.orc_last_implicit_residual.restype = C.c_double
        L.orc_last_implicit_residual.argtypes = [C.c_void_p, C.c_int]
        L.orc_hll.argtypes = [C.POINTER(OFluid), C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, dp]
        L.orc_pb_system.argtypes = [C.POINTER(OFluid), C.c_double, C.c_int, C.c_double, C.c_double, C.c_int,
                                    C.c_double, C.c_double, C.c_double, C.c_double, dp]
        L.orc_pb_solve.argtypes = [C.POINTER(OFluid), C.POINTER(OOpts), C.c_double, C.c_int, C.c_double,
                                   C.c_double, C.c_int, C.c_double, C.c_double, dp]
        L.orc_nopt_star.restype = C.c_double
        L.orc_nopt_star.argtypes = [C.POINTER(OFluid), C.c_int, C.c_double, C.c_double, C.c_double, C.c_double]
        L.orc_creation_solve.argtypes = [C.POINTER(OFluid), C.POINTER(OOpts), C.c_double, C.c_int, C.c_double,
                                         C.c_double, C.c_double, C.c_double, dp]
        if hasattr(L, "orc_tangent"):
            L.orc_tangent.argtypes = [C.c_void_p, C.c_int, dp, dp, dp, dp, C.c_int, ip, dp, C.c_int]
            L.orc_get_tangent.argtypes = [C.c_void_p, C.c_int, dp, dp, dp]
        if hasattr(L, "orc_count_ops"):
            L.orc_count_ops.argtypes = [C.c_void_p, C.c_int, ip, dp, C.POINTER(C.c_longlong)]
        L.orc_exact_sample.argtypes = [C.POINTER(OFluid), C.POINTER(OOpts), C.c_double, C.c_int, C.c_double,
                                       C.c_double, C.c_int, C.c_double, C.c_double, C.c_int, dp, dp, dp, ip]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def make_fluid(f) -> OFluid:
    """From an inputs.Fluid."""
    of = OFluid()
    of.ph[0] = OEos(0, f.a2_vap, 0.0, 0.0)
    of.ph[1] = OEos(1, f.a2_liq, f.p_sat, f.rho0_liq)
    of.p_sat, of.p_min, of.p_tilde = f.p_sat, f.p_min, f.p_tilde
    return of


def make_opts(o, block_solver=None) -> OOpts:
    """block_solver: 0 dual time stepping (Alg. 2), 1 Newton on each block's implicit system; None takes the
    options' own block_solver (0 when they have none)."""
    bs = getattr(o, "block_solver", 0) if block_solver is None else block_solver
    return OOpts(o.cfl, o.theta_nb, o.tol_nb, o.tol_k, o.res_mode, o.l_max, o.newton_tol, o.newton_itmax,
                 o.alpha_min, o.split_ratio, o.creation, bs)


def pb_solve(fluid, opts, tau, phl, rl, ul, phr, rr, ur):
    out = np.zeros(11)
    rc = lib().orc_pb_solve(C.byref(make_fluid(fluid)), C.byref(make_opts(opts)), tau, phl, rl, ul, phr, rr, ur,
                            _dp(out))
    keys = ["p_l", "p_r", "rho_l", "rho_r", "u_l", "u_r", "z", "w", "F0", "F1", "iters"]
    d = dict(zip(keys, out.tolist()))
    d["status"] = rc
    return d


def pb_system(fluid, tau, phl, rl, ul, phr, rr, ur, pls, prs):
    out = np.zeros(7)
    lib().orc_pb_system(C.byref(make_fluid(fluid)), tau, phl, rl, ul, phr, rr, ur, pls, prs, _dp(out))
    return {"G": out[0:2].copy(), "z": out[2], "J": out[3:7].reshape(2, 2).copy()}


def hll(fluid, ph, rl, ml, rr, mr):
    F = np.zeros(2)
    lib().orc_hll(C.byref(make_fluid(fluid)), ph, rl, ml, rr, mr, _dp(F))
    return F


def nopt_star(fluid, ph, rl, ul, rr, ur):
    return lib().orc_nopt_star(C.byref(make_fluid(fluid)), ph, rl, ul, rr, ur)


def creation_solve(fluid, opts, tau, ph, rl, ul, rr, ur):
    out = np.zeros(12)
    rc = lib().orc_creation_solve(C.byref(make_fluid(fluid)), C.byref(make_opts(opts)), tau, ph, rl, ul, rr, ur,
                                  _dp(out))
    keys = ["p_parent_l", "p_created", "p_parent_r", "rho_created", "u_created", "z_l", "z_r", "w_l", "w_r",
            "u_parent_l", "u_parent_r", "iters"]
    d = dict(zip(keys, out.tolist()))
    d["status"] = rc
    return d


def exact_sample(fluid, opts, tau, phl, rl, ul, phr, rr, ur, xi):
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    n = xi.shape[0]
    rho = np.zeros(n)
    u = np.zeros(n)
    ph = np.zeros(n, dtype=np.int32)
    rc = lib().orc_exact_sample(C.byref(make_fluid(fluid)), C.byref(make_opts(opts)), tau, phl, rl, ul, phr, rr,
                                ur, n, _dp(xi), _dp(rho), _dp(u), _ip(ph))
    if rc != 0:
        raise RuntimeError(f"exact solution: status {rc}")
    return rho, u, ph


class Oracle:
    """A batch of instances advanced by the oracle."""

    def __init__(self, batch, options=None, block_solver=None):
        L = lib()
        self.batch = batch
        self.n = batch.n_inst
        self._fl = make_fluid(batch.fluid)
        self._op = make_opts(options or batch.options, block_solver)
        nl = np.ascontiguousarray(batch.n_lattice, dtype=np.int32)
        self.h = L.orc_create(self.n, _ip(nl), _dp(np.ascontiguousarray(batch.x_left)),
                              _dp(np.ascontiguousarray(batch.x_right)), _dp(np.ascontiguousarray(batch.tau)),
                              C.byref(self._fl), C.byref(self._op))
        off = np.ascontiguousarray(batch.cell_offsets, dtype=np.int32)
        ph = np.ascontiguousarray(batch.phase, dtype=np.uint8)
        self.set_rc = L.orc_set_states(self.h, _ip(off), _dp(np.ascontiguousarray(batch.widths)),
                                       _dp(np.ascontiguousarray(batch.rho)), _dp(np.ascontiguousarray(batch.m)),
                                       ph.ctypes.data_as(C.POINTER(C.c_ubyte)), 0.0)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    def run_to(self, t_end, threads=1):
        lib().orc_run_to(self.h, t_end, threads)

    def step(self, n, threads=1):
        lib().orc_step(self.h, n, threads)

    def explicit_run_to(self, t_end, threads=1):
        lib().orc_explicit_run_to(self.h, t_end, threads)

    def states(self):
        L = lib()
        counts = np.zeros(self.n, dtype=np.int32)
        L.orc_n_cells(self.h, _ip(counts))
        tot = int(counts.sum())
        off = np.zeros(self.n + 1, dtype=np.int32)
        w, r, m = np.zeros(tot), np.zeros(tot), np.zeros(tot)
        ph = np.zeros(tot, dtype=np.uint8)
        t = np.zeros(self.n)
        st = np.zeros(self.n, dtype=np.int32)
        L.orc_get_states(self.h, _ip(off), _dp(w), _dp(r), _dp(m), ph.ctypes.data_as(C.POINTER(C.c_ubyte)), _dp(t),
                         _ip(st))
        return {"offsets": off, "widths": w, "rho": r, "m": m, "phase": ph, "t": t, "status": st}

    def pbs(self):
        counts = np.zeros(self.n, dtype=np.int32)
        lib().orc_n_cells(self.h, _ip(counts))
        off = np.zeros(self.n + 1, dtype=np.int32)
        x = np.zeros(int(counts.sum()) + 1)
        lib().orc_get_pbs(self.h, _ip(off), _dp(x))
        return off, x[: off[-1]].copy()

    def stats(self):
        s = np.zeros((self.n, 10), dtype=np.int64)
        lib().orc_get_stats(self.h, s.ctypes.data_as(C.POINTER(C.c_longlong)))
        keys = ["steps", "dts_iters", "dts_max", "newton", "merges", "splits", "creations", "maxiter", "pb_solves"]
        return {k: s[:, i].copy() for i, k in enumerate(keys)}

    def count_ops(self, program) -> dict:
        """Floating-point operations of the program [("step", n) | ("run_to", t_end), ...] run from the
        current states (which are kept): adds, multiplies, divides, square roots, logarithms, exponentials,
        and the cell-steps they served."""
        kinds = np.array([0 if k == "step" else 1 for k, _ in program], dtype=np.int32)
        args = np.array([float(a) for _, a in program], dtype=np.float64)
        c = np.zeros(7, dtype=np.int64)
        rc = lib().orc_count_ops(self.h, len(program), _ip(kinds), _dp(args), c.ctypes.data_as(C.POINTER(C.c_longlong)))
        if rc != 0:
            raise RuntimeError(f"oracle count_ops: status {rc}")
        return dict(zip(["add", "mul", "div", "sqrt", "log", "exp", "cell_steps"], (int(x) for x in c)))

    def tangent(self, program, seed_w=None, seed_rho=None, seed_m=None, seed_tau=None, threads=1):
        """Forward-mode derivative of the program [("step", n) | ("run_to", t_end), ...] from the current
        states. Seeds: arrays [n_dir, total cells] (widths, rho, m) and [n_dir, n_inst] (tau), any None.
        Returns the final states and a dict of derivative arrays [n_dir, final cells]."""
        seeds = [s for s in (seed_w, seed_rho, seed_m, seed_tau) if s is not None]
        n_dir = seeds[0].shape[0]
        conv = [None if s is None else np.ascontiguousarray(s, dtype=np.float64) for s in
                (seed_w, seed_rho, seed_m, seed_tau)]
        ptr = [C.cast(None, C.POINTER(C.c_double)) if s is None else _dp(s) for s in conv]
        kinds = np.array([0 if k == "step" else 1 for k, _ in program], dtype=np.int32)
        args = np.array([float(a) for _, a in program], dtype=np.float64)
        rc = lib().orc_tangent(self.h, n_dir, ptr[0], ptr[1], ptr[2], ptr[3], len(program), _ip(kinds), _dp(args),
                               threads)
        if rc != 0:
            raise RuntimeError(f"oracle tangent: status {rc}")
        st = self.states()
        tot = st["offsets"][-1]
        d = {"widths": np.zeros((n_dir, tot)), "rho": np.zeros((n_dir, tot)), "m": np.zeros((n_dir, tot))}
        for q in range(n_dir):
            dw, dr, dm = np.zeros(tot), np.zeros(tot), np.zeros(tot)
            lib().orc_get_tangent(self.h, q, _dp(dw), _dp(dr), _dp(dm))
            d["widths"][q], d["rho"][q], d["m"][q] = dw, dr, dm
        return st, d

    def implicit_defect(self, i=0):
        return lib().orc_last_implicit_residual(self.h, i)
