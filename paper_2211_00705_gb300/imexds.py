"""Python binding of the imexds C-ABI (include/imexds.h): argument marshalling only.

Every step of the scheme runs in the CUDA library libimexds.so built in this package directory;
importing this module without that library (or without a CUDA device when a call needs one) raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libimexds.so")

STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_NONPHYSICAL", 4: "ERR_PB_NOCONV", 5: "WARN_DTS_MAXITER",
          6: "ERR_VANISH", 7: "ERR_TIMEOUT", 8: "ERR_STATE", 9: "ERR_CAPACITY"}

EXPORTED = ["imexds_create", "imexds_set_states", "imexds_set_states_device", "imexds_cell_counts",
            "imexds_get_states", "imexds_step", "imexds_run_to", "imexds_get_stats", "imexds_destroy",
            "imexds_status_string", "imexds_last_error_string", "imexds_reset", "imexds_set_kernel_timing",
            "imexds_get_kernel_times", "imexds_set_schedule", "imexds_check_log", "imexds_step_uniform_noalloc",
            "imexds_get_group_phase_cycles", "imexds_adjoint", "imexds_set_adjoint_checkpoint",
            "imexds_adjoint_info", "imexds_adjoint_replay", "imexds_check_div", "imexds_check_tol",
            "imexds_get_states_device", "imexds_adjoint_device"]


class ImexdsError(RuntimeError):
    pass


class Eos(C.Structure):
    _fields_ = [("kind", C.c_int), ("a2", C.c_double), ("p0", C.c_double), ("rho0", C.c_double)]


class FluidS(C.Structure):
    _fields_ = [("vapour", Eos), ("liquid", Eos), ("p_sat", C.c_double), ("p_min", C.c_double),
                ("p_tilde", C.c_double)]


class OptionsS(C.Structure):
    _fields_ = [("cfl", C.c_double), ("theta_nb", C.c_double), ("tol_nb", C.c_double), ("tol_k", C.c_double),
                ("res_mode", C.c_int), ("l_max", C.c_int), ("newton_tol", C.c_double),
                ("newton_itmax", C.c_int), ("alpha_min", C.c_double), ("split_ratio", C.c_double),
                ("creation", C.c_int), ("zone_capacity", C.c_int), ("schedule", C.c_int),
                ("group_cells", C.c_int), ("group_threads", C.c_int), ("block_solver", C.c_int)]


class ProblemS(C.Structure):
    _fields_ = [("n_inst", C.c_int32), ("n_lattice", C.POINTER(C.c_int32)), ("x_left", C.POINTER(C.c_double)),
                ("x_right", C.POINTER(C.c_double)), ("tau", C.POINTER(C.c_double)), ("fluid", FluidS)]


_lib = None


def load():
    """Load libimexds.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImexdsError(f"CUDA library missing: {LIB_PATH} (run __graft_entry__.build())")
        L = C.CDLL(LIB_PATH)
        dp, ip, vp = C.POINTER(C.c_double), C.POINTER(C.c_int32), C.c_void_p
        u8p = C.POINTER(C.c_uint8)
        L.imexds_create.argtypes = [C.POINTER(ProblemS), C.POINTER(OptionsS), vp, C.POINTER(vp)]
        L.imexds_set_states.argtypes = [vp, ip, dp, dp, dp, u8p, C.c_double]
        L.imexds_set_states_device.argtypes = [vp, ip, vp, vp, vp, vp, C.c_double]
        L.imexds_cell_counts.argtypes = [vp, ip]
        L.imexds_get_states.argtypes = [vp, ip, dp, dp, dp, u8p, dp, ip]
        L.imexds_step.argtypes = [vp, C.c_int32]
        L.imexds_run_to.argtypes = [vp, C.c_double]
        L.imexds_get_stats.argtypes = [vp, C.POINTER(C.c_int64)]
        L.imexds_destroy.argtypes = [vp]
        L.imexds_reset.argtypes = [vp]
        L.imexds_set_kernel_timing.argtypes = [vp, C.c_int32]
        L.imexds_get_kernel_times.argtypes = [vp, dp, C.POINTER(C.c_int64)]
        L.imexds_set_schedule.argtypes = [vp, C.c_int32]
        L.imexds_get_group_phase_cycles.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.imexds_check_log.argtypes = [C.c_int32, dp, dp, dp]
        L.imexds_check_div.argtypes = [C.c_int32, dp, dp, dp, dp]
        L.imexds_check_tol.argtypes = [C.c_int32, dp, dp, dp, C.POINTER(C.c_uint8), C.POINTER(C.c_uint8)]
        L.imexds_step_uniform_noalloc.argtypes = [C.POINTER(FluidS), C.c_double, C.c_int32, ip, dp, dp, vp, vp, vp,
                                                  vp, vp, vp, vp]
        L.imexds_adjoint.argtypes = [vp, dp, dp, dp, dp, dp, dp, dp, ip]
        L.imexds_adjoint_device.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, ip]
        L.imexds_get_states_device.argtypes = [vp, ip, vp, vp, vp, vp, dp, ip]
        L.imexds_set_adjoint_checkpoint.argtypes = [vp, C.c_int32]
        L.imexds_adjoint_info.argtypes = [vp, dp, dp, C.POINTER(C.c_int64)]
        L.imexds_adjoint_replay.argtypes = [vp, ip, dp, dp, dp, ip]
        L.imexds_status_string.restype = C.c_char_p
        L.imexds_status_string.argtypes = [C.c_int]
        L.imexds_last_error_string.restype = C.c_char_p
        _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        L = load()
        msg = L.imexds_status_string(rc).decode()
        if rc == 2:
            msg += ": " + L.imexds_last_error_string().decode()
        raise ImexdsError(f"imexds status {rc} ({msg})")


def last_error() -> str:
    """Text of the library's last recorded error (imexds_last_error_string)."""
    return load().imexds_last_error_string().decode()


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def make_fluid(f) -> FluidS:
    """From an inputs.Fluid."""
    return FluidS(Eos(0, f.a2_vap, 0.0, 0.0), Eos(1, f.a2_liq, f.p_sat, f.rho0_liq), f.p_sat, f.p_min, f.p_tilde)


def make_options(o, zone_capacity: int = 0, schedule: int = 0, group_cells: int = 0,
                 group_threads: int = 0) -> OptionsS:
    return OptionsS(o.cfl, o.theta_nb, o.tol_nb, o.tol_k, o.res_mode, o.l_max, o.newton_tol, o.newton_itmax,
                    o.alpha_min, o.split_ratio, o.creation, zone_capacity, schedule, group_cells, group_threads,
                    getattr(o, "block_solver", 0))


def step_uniform_noalloc(fluid, cfl, n_lattice, x_left, x_right, rho_in, m_in, phase, rho_out, m_out, dt_out,
                         stream: int = 0):
    """One explicit step of single-phase instances without any GPU allocation by the library (see
    include/imexds.h). rho_in/m_in/phase/rho_out/m_out/dt_out are CUDA tensors (float64, uint8)."""
    nl = np.ascontiguousarray(n_lattice, dtype=np.int32)
    xl = np.ascontiguousarray(x_left, dtype=np.float64)
    xr = np.ascontiguousarray(x_right, dtype=np.float64)
    fl = make_fluid(fluid)
    _check(load().imexds_step_uniform_noalloc(
        C.byref(fl), float(cfl), int(nl.shape[0]), _ip(nl), _dp(xl), _dp(xr), C.c_void_p(rho_in.data_ptr()),
        C.c_void_p(m_in.data_ptr()), C.c_void_p(phase.data_ptr()), C.c_void_p(rho_out.data_ptr()),
        C.c_void_p(m_out.data_ptr()), C.c_void_p(dt_out.data_ptr()), C.c_void_p(stream)))


def check_div(a, b):
    """The library's quotient (Newton-Raphson-refined reciprocal) and CUDA's division at the pairs (a, b)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    fast = np.zeros_like(a)
    ref = np.zeros_like(a)
    _check(load().imexds_check_div(int(a.shape[0]), _dp(a), _dp(b), _dp(fast), _dp(ref)))
    return fast, ref


def check_tol(d, w, lim):
    """The library's bit-pattern stop test |d| < lim max(|w|, 1) and the FP64 comparison (diagnostic)."""
    d, w, lim = (np.ascontiguousarray(v, dtype=np.float64) for v in (d, w, lim))
    fast = np.zeros(d.shape[0], dtype=np.uint8)
    ref = np.zeros(d.shape[0], dtype=np.uint8)
    u8 = C.POINTER(C.c_uint8)
    _check(load().imexds_check_tol(int(d.shape[0]), _dp(d), _dp(w), _dp(lim), fast.ctypes.data_as(u8),
                                   ref.ctypes.data_as(u8)))
    return fast, ref


def check_log(x):
    """Table-driven logarithm of the library and CUDA's log at the points x (diagnostic)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    fast = np.zeros_like(x)
    ref = np.zeros_like(x)
    _check(load().imexds_check_log(int(x.shape[0]), _dp(x), _dp(fast), _dp(ref)))
    return fast, ref


class Imexds:
    """A context of the CUDA library holding a batch of instances (see include/imexds.h)."""

    def __init__(self, n_lattice, x_left, x_right, tau, fluid, options, stream: int = 0, zone_capacity: int = 0,
                 schedule: int = 0, group_cells: int = 0, group_threads: int = 0):
        L = load()
        self._keep = [np.ascontiguousarray(n_lattice, dtype=np.int32), np.ascontiguousarray(x_left, dtype=np.float64),
                      np.ascontiguousarray(x_right, dtype=np.float64), np.ascontiguousarray(tau, dtype=np.float64)]
        nl, xl, xr, tau_ = self._keep
        self.n_inst = int(nl.shape[0])
        prob = ProblemS(self.n_inst, _ip(nl), _dp(xl), _dp(xr), _dp(tau_), make_fluid(fluid))
        opts = make_options(options, zone_capacity, schedule, group_cells, group_threads)
        h = C.c_void_p()
        _check(L.imexds_create(C.byref(prob), C.byref(opts), C.c_void_p(stream), C.byref(h)))
        self.h = h

    @classmethod
    def from_batch(cls, batch, options=None, stream: int = 0, zone_capacity: int = 0, schedule: int = 0,
                   group_cells: int = 0, group_threads: int = 0) -> "Imexds":
        ctx = cls(batch.n_lattice, batch.x_left, batch.x_right, batch.tau, batch.fluid, options or batch.options,
                  stream=stream, zone_capacity=zone_capacity, schedule=schedule, group_cells=group_cells,
                  group_threads=group_threads)
        ctx.set_states(batch.cell_offsets, batch.widths, batch.rho, batch.m, batch.phase)
        return ctx

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            load().imexds_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_states(self, offsets, widths, rho, m, phase, t0: float = 0.0):
        off = np.ascontiguousarray(offsets, dtype=np.int32)
        w = np.ascontiguousarray(widths, dtype=np.float64)
        r = np.ascontiguousarray(rho, dtype=np.float64)
        mm = np.ascontiguousarray(m, dtype=np.float64)
        ph = np.ascontiguousarray(phase, dtype=np.uint8)
        self._check_lists(off, [("widths", w), ("rho", r), ("m", mm), ("phase", ph)])
        _check(load().imexds_set_states(self.h, _ip(off), _dp(w), _dp(r), _dp(mm),
                                        ph.ctypes.data_as(C.POINTER(C.c_uint8)), t0))
        self._n0 = int(off[-1])

    def set_states_device(self, offsets, widths_d, rho_d, m_d, phase_d, t0: float = 0.0):
        """Device-pointer variant: widths_d/rho_d/m_d (float64) and phase_d (uint8) are CUDA tensors."""
        off = np.ascontiguousarray(offsets, dtype=np.int32)
        self._check_lists(off, [("widths_d", widths_d), ("rho_d", rho_d), ("m_d", m_d), ("phase_d", phase_d)])
        _check(load().imexds_set_states_device(self.h, _ip(off), C.c_void_p(widths_d.data_ptr()),
                                               C.c_void_p(rho_d.data_ptr()), C.c_void_p(m_d.data_ptr()),
                                               C.c_void_p(phase_d.data_ptr()), t0))
        self._n0 = int(off[-1])

    def _check_lists(self, off, arrays):
        """The library reads offsets[n_inst] entries of every cell array: refuse shorter (or longer) ones."""
        if off.ndim != 1 or off.shape[0] != self.n_inst + 1:
            raise ValueError(f"offsets has {off.shape[0]} entries, expected n_inst + 1 = {self.n_inst + 1}")
        n = int(off[-1])
        for name, a in arrays:
            if a.shape[0] != n:
                raise ValueError(f"{name} has {a.shape[0]} entries, offsets[-1] is {n}")

    def step(self, n_steps: int):
        _check(load().imexds_step(self.h, int(n_steps)))

    def run_to(self, t_end: float):
        _check(load().imexds_run_to(self.h, float(t_end)))

    def cell_counts(self) -> np.ndarray:
        c = np.zeros(self.n_inst, dtype=np.int32)
        _check(load().imexds_cell_counts(self.h, _ip(c)))
        return c

    def get_states(self) -> dict:
        counts = self.cell_counts()
        tot = int(counts.sum())
        off = np.zeros(self.n_inst + 1, dtype=np.int32)
        w, r, m = np.zeros(tot), np.zeros(tot), np.zeros(tot)
        ph = np.zeros(tot, dtype=np.uint8)
        t = np.zeros(self.n_inst)
        st = np.zeros(self.n_inst, dtype=np.int32)
        _check(load().imexds_get_states(self.h, _ip(off), _dp(w), _dp(r), _dp(m),
                                        ph.ctypes.data_as(C.POINTER(C.c_uint8)), _dp(t), _ip(st)))
        return {"offsets": off, "widths": w, "rho": r, "m": m, "phase": ph, "t": t, "status": st}

    def get_states_device(self, widths_d, rho_d, m_d, phase_d) -> dict:
        """Device-resident get_states: the cell lists are written into the given CUDA tensors (float64 widths,
        rho, m and uint8 phase, each with cell_counts().sum() entries); offsets, t and status come back as host
        arrays."""
        tot = int(self.cell_counts().sum())
        for name, a in (("widths_d", widths_d), ("rho_d", rho_d), ("m_d", m_d), ("phase_d", phase_d)):
            if a.shape[0] != tot:
                raise ValueError(f"{name} has {a.shape[0]} entries, the cell lists {tot}")
        off = np.zeros(self.n_inst + 1, dtype=np.int32)
        t = np.zeros(self.n_inst)
        st = np.zeros(self.n_inst, dtype=np.int32)
        _check(load().imexds_get_states_device(self.h, _ip(off), C.c_void_p(widths_d.data_ptr()),
                                               C.c_void_p(rho_d.data_ptr()), C.c_void_p(m_d.data_ptr()),
                                               C.c_void_p(phase_d.data_ptr()), _dp(t), _ip(st)))
        return {"offsets": off, "t": t, "status": st}

    def reset(self):
        """Restore the states given to the last set_states (device-to-device)."""
        _check(load().imexds_reset(self.h))

    def set_kernel_timing(self, on: bool):
        _check(load().imexds_set_kernel_timing(self.h, 1 if on else 0))

    KERNELS = ["k_pre", "k_plan", "k_sweep", "k_dts", "k_post", "k_group"]

    def set_schedule(self, schedule: int):
        """0 automatic, 1 per-step kernels, 2 instance groups in lockstep, 3 instance groups advancing
        independently."""
        _check(load().imexds_set_schedule(self.h, int(schedule)))

    def kernel_times(self) -> dict:
        ms = np.zeros(6)
        n = np.zeros(6, dtype=np.int64)
        _check(load().imexds_get_kernel_times(self.h, _dp(ms), n.ctypes.data_as(C.POINTER(C.c_int64))))
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(self.KERNELS)}

    PHASES = ["plan", "sweep", "block_solve", "post", "concurrent", "launch"]

    def group_phase_cycles(self) -> dict:
        """SM cycles per phase of the group kernel (timing mode), for the slowest group and summed over groups;
        keys as imexds_get_group_phase_cycles: plan + post + concurrent = launch (lockstep groups)."""
        a = np.zeros(6, dtype=np.int64)
        b = np.zeros(6, dtype=np.int64)
        _check(load().imexds_get_group_phase_cycles(self.h, a.ctypes.data_as(C.POINTER(C.c_int64)),
                                                    b.ctypes.data_as(C.POINTER(C.c_int64))))
        keys = self.PHASES
        return {"slowest": dict(zip(keys, a.tolist())), "sum": dict(zip(keys, b.tolist()))}

    def set_adjoint_checkpoint(self, every: int):
        _check(load().imexds_set_adjoint_checkpoint(self.h, int(every)))

    def adjoint(self, dJ_drho_T, dJ_dm_T, dJ_dw_T=None) -> dict:
        """Gradient of a loss of the final states of the last forward run (see include/imexds.h).
        Inputs follow get_states' cell order; outputs the initial states' order (set_states)."""
        n0 = self._n_initial_cells()
        r = np.ascontiguousarray(dJ_drho_T, dtype=np.float64).ravel()
        m = np.ascontiguousarray(dJ_dm_T, dtype=np.float64).ravel()
        w = None if dJ_dw_T is None else np.ascontiguousarray(dJ_dw_T, dtype=np.float64).ravel()
        nT = int(self.cell_counts().sum())   # the library reads one entry per final cell
        for name, a in (("dJ_drho_T", r), ("dJ_dm_T", m), ("dJ_dw_T", w)):
            if a is not None and a.shape[0] != nT:
                raise ValueError(f"{name} has {a.shape[0]} entries, the final cell lists {nT}")
        g = {"rho": np.zeros(n0), "m": np.zeros(n0), "widths": np.zeros(n0), "tau": np.zeros(self.n_inst),
             "status": np.zeros(self.n_inst, dtype=np.int32)}
        null = C.cast(None, C.POINTER(C.c_double))
        _check(load().imexds_adjoint(self.h, null if w is None else _dp(w), _dp(r), _dp(m), _dp(g["widths"]),
                                     _dp(g["rho"]), _dp(g["m"]), _dp(g["tau"]), _ip(g["status"])))
        return g

    def adjoint_device(self, dJ_drho_T, dJ_dm_T, out_rho, out_m, out_tau, dJ_dw_T=None, out_w=None):
        """Device-resident adjoint: seeds and outputs are CUDA tensors (float64) in the orders of adjoint();
        dJ_dw_T and out_w may be None. Returns the per-instance statuses (host array)."""
        nT = int(self.cell_counts().sum())
        n0 = self._n_initial_cells()
        for name, a, want in (("dJ_drho_T", dJ_drho_T, nT), ("dJ_dm_T", dJ_dm_T, nT), ("dJ_dw_T", dJ_dw_T, nT),
                              ("out_rho", out_rho, n0), ("out_m", out_m, n0), ("out_w", out_w, n0),
                              ("out_tau", out_tau, self.n_inst)):
            if a is not None and a.shape[0] != want:
                raise ValueError(f"{name} has {a.shape[0]} entries, expected {want}")
        st = np.zeros(self.n_inst, dtype=np.int32)

        def ptr(a):
            return C.c_void_p(None if a is None else a.data_ptr())
        _check(load().imexds_adjoint_device(self.h, ptr(dJ_dw_T), ptr(dJ_drho_T), ptr(dJ_dm_T), ptr(out_w),
                                            ptr(out_rho), ptr(out_m), ptr(out_tau), _ip(st)))
        return st

    def adjoint_info(self) -> dict:
        ms, err = np.zeros(1), np.zeros(1)
        cs = np.zeros(1, dtype=np.int64)
        _check(load().imexds_adjoint_info(self.h, _dp(ms), _dp(err), cs.ctypes.data_as(C.POINTER(C.c_int64))))
        return {"kernel_ms": float(ms[0]), "replay_err": float(err[0]), "cell_steps": int(cs[0])}

    def adjoint_replay(self) -> dict:
        """The last adjoint's replayed final cell lists and, per instance, where a replay was stopped."""
        L = load()
        off = np.zeros(self.n_inst + 1, dtype=np.int32)
        site = np.zeros(self.n_inst, dtype=np.int32)
        null = C.cast(None, C.POINTER(C.c_double))
        _check(L.imexds_adjoint_replay(self.h, _ip(off), null, null, null, _ip(site)))
        tot = int(off[-1])
        w, r, m = np.zeros(tot), np.zeros(tot), np.zeros(tot)
        _check(L.imexds_adjoint_replay(self.h, _ip(off), _dp(w), _dp(r), _dp(m), _ip(site)))
        return {"offsets": off, "widths": w, "rho": r, "m": m, "site": site}

    def _n_initial_cells(self) -> int:
        return int(self._n0)

    def stats(self) -> dict:
        s = np.zeros((self.n_inst, 10), dtype=np.int64)
        _check(load().imexds_get_stats(self.h, s.ctypes.data_as(C.POINTER(C.c_int64))))
        keys = ["steps", "dts_iters", "dts_max", "newton", "merges", "splits", "creations", "maxiter", "pb_solves",
                "launches"]
        return {k: s[:, i].copy() for i, k in enumerate(keys)}
