"""torch.autograd.Function over the library: forward = a run of the scheme (imexds_step / imexds_run_to),
backward = the discrete adjoint. Argument marshalling only; both directions run in the CUDA library, and the
per-cell data stays on the device (imexds_set_states_device, imexds_get_states_device, imexds_adjoint_device).

    rho_T, m_T = ImexdsFunction.apply(rho0, m0, tau, spec)

rho0, m0: float64 CUDA tensors of the initial cell states (instances concatenated, cell order of
imexds_set_states); tau: float64 tensor of the kinetic coefficients (one per instance; its values are read to
the host to build the problem). spec: a `RunSpec` with the rest of the problem (lattice, domain, widths, phases,
fluid, options, the program of calls). Outputs: the final cell states (cell order of imexds_get_states) as new
CUDA tensors on the device of rho0. The final cell lists can differ in length from the initial ones (merges,
splits, created cells); spec.last_offsets holds the final offsets after a forward call and spec.last_widths the
final widths (a CUDA tensor). Gradients flow to rho0, m0 and tau; the widths are not inputs here. One library
context is kept per RunSpec and reused while tau is unchanged.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from .imexds import Imexds


@dataclasses.dataclass
class RunSpec:
    n_lattice: np.ndarray
    x_left: np.ndarray
    x_right: np.ndarray
    cell_offsets: np.ndarray
    widths: np.ndarray
    phase: np.ndarray
    fluid: object
    options: object
    program: list                 # [("step", n) | ("run_to", t_end), ...]
    checkpoint_every: int = 64
    last_offsets: np.ndarray | None = None
    last_widths: torch.Tensor | None = None
    # cached between calls: the context, the tau it was built with, the device copies of widths and phases
    _ctx: object = dataclasses.field(default=None, repr=False)
    _tau: np.ndarray | None = dataclasses.field(default=None, repr=False)
    _dev: dict = dataclasses.field(default_factory=dict, repr=False)

    def context(self, tau: np.ndarray) -> Imexds:
        if self._ctx is None or self._tau is None or not np.array_equal(self._tau, tau):
            if self._ctx is not None:
                self._ctx.close()
            self._ctx = Imexds(self.n_lattice, self.x_left, self.x_right, tau, self.fluid, self.options)
            self._ctx.set_adjoint_checkpoint(self.checkpoint_every)
            self._tau = tau.copy()
        return self._ctx

    def device_lists(self, device):
        if device not in self._dev:
            self._dev[device] = (torch.as_tensor(np.ascontiguousarray(self.widths, dtype=np.float64), device=device),
                                 torch.as_tensor(np.ascontiguousarray(self.phase, dtype=np.uint8), device=device))
        return self._dev[device]


class ImexdsFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho0, m0, tau, spec: RunSpec):
        dev = rho0.device
        c = spec.context(tau.detach().cpu().numpy().astype(np.float64))
        w0, ph0 = spec.device_lists(dev)
        c.set_states_device(spec.cell_offsets, w0, rho0.detach().contiguous(), m0.detach().contiguous(), ph0)
        for kind, arg in spec.program:
            if kind == "step":
                c.step(int(arg))
            else:
                c.run_to(float(arg))
        tot = int(c.cell_counts().sum())
        wT = torch.empty(tot, dtype=torch.float64, device=dev)
        rT = torch.empty(tot, dtype=torch.float64, device=dev)
        mT = torch.empty(tot, dtype=torch.float64, device=dev)
        phT = torch.empty(tot, dtype=torch.uint8, device=dev)
        s = c.get_states_device(wT, rT, mT, phT)
        spec.last_offsets = s["offsets"]
        spec.last_widths = wT
        ctx.imexds = c
        ctx.n0 = int(rho0.shape[0])
        ctx.n_inst = int(tau.shape[0])
        return rT, mT

    @staticmethod
    def backward(ctx, g_rho, g_m):
        c = ctx.imexds
        nT = int(c.cell_counts().sum())
        dev = g_rho.device if g_rho is not None else g_m.device
        zero = torch.zeros(nT, dtype=torch.float64, device=dev)
        gr = zero if g_rho is None else g_rho.detach().to(torch.float64).contiguous()
        gm = zero if g_m is None else g_m.detach().to(torch.float64).contiguous()
        out_r = torch.empty(ctx.n0, dtype=torch.float64, device=dev)
        out_m = torch.empty(ctx.n0, dtype=torch.float64, device=dev)
        out_t = torch.empty(ctx.n_inst, dtype=torch.float64, device=dev)
        st = c.adjoint_device(gr, gm, out_r, out_m, out_t)
        ctx.imexds = None
        if (st != 0).any():
            raise RuntimeError(f"adjoint: instances without gradient: {np.nonzero(st)[0].tolist()}")
        return out_r, out_m, out_t, None
