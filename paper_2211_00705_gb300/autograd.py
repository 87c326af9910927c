"""torch.autograd.Function over the library: forward = a run of the scheme (imexds_step / imexds_run_to),
backward = the discrete adjoint (imexds_adjoint). Argument marshalling only; both directions run in the
CUDA library.

    rho_T, m_T = ImexdsFunction.apply(rho0, m0, tau, spec)

rho0, m0: float64 tensors of the initial cell states (instances concatenated, cell order of
imexds_set_states); tau: float64 tensor of the kinetic coefficients (one per instance). spec: a
`RunSpec` with the rest of the problem (lattice, domain, widths, phases, fluid, options, the program of
calls). Outputs: the final cell states (cell order of imexds_get_states) on the device of rho0. The final
cell lists can differ in length from the initial ones (merges, splits); spec.last_offsets holds the
final offsets after a forward call. Gradients flow to rho0, m0 and tau; the widths are not inputs here.
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
    last_widths: np.ndarray | None = None


class ImexdsFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho0, m0, tau, spec: RunSpec):
        c = Imexds(spec.n_lattice, spec.x_left, spec.x_right, tau.detach().cpu().numpy(), spec.fluid, spec.options)
        c.set_adjoint_checkpoint(spec.checkpoint_every)
        c.set_states(spec.cell_offsets, spec.widths, rho0.detach().cpu().numpy(), m0.detach().cpu().numpy(),
                     spec.phase)
        for kind, arg in spec.program:
            if kind == "step":
                c.step(int(arg))
            else:
                c.run_to(float(arg))
        s = c.get_states()
        spec.last_offsets = s["offsets"]
        spec.last_widths = s["widths"]
        ctx.imexds = c
        ctx.dev = rho0.device
        return (torch.from_numpy(s["rho"]).to(rho0.device), torch.from_numpy(s["m"]).to(rho0.device))

    @staticmethod
    def backward(ctx, g_rho, g_m):
        c = ctx.imexds
        gr = np.zeros(0) if g_rho is None else g_rho.detach().cpu().numpy().astype(np.float64)
        gm = np.zeros(0) if g_m is None else g_m.detach().cpu().numpy().astype(np.float64)
        n = int(c.cell_counts().sum())
        if g_rho is None:
            gr = np.zeros(n)
        if g_m is None:
            gm = np.zeros(n)
        g = c.adjoint(gr, gm)
        c.close()
        ctx.imexds = None
        if (g["status"] != 0).any():
            raise RuntimeError(f"adjoint: instances without gradient: {np.nonzero(g['status'])[0].tolist()}")
        dev = ctx.dev
        return (torch.from_numpy(g["rho"]).to(dev), torch.from_numpy(g["m"]).to(dev),
                torch.from_numpy(g["tau"]).to(dev), None)
