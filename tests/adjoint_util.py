"""Helpers of the adjoint tests: the density-misfit loss of the adjoint workload and directional
derivatives from gradients and from the oracle's tangent mode."""
import numpy as np

from paper_2211_00705_gb300 import inputs as I


def misfit(states, target, batch):
    """J_i = 1/2 h sum_j (rho(x_j) - rho_tgt(x_j))^2 over the background centres x_j of instance i
    (piecewise-constant sampling of the cell list). Returns (J per instance, dJ/drho per final cell)."""
    off = states["offsets"]
    rs, idx = I.sample_density(states, off, batch.n_lattice, batch.x_left, batch.x_right)
    h = np.repeat((batch.x_right - batch.x_left) / batch.n_lattice, batch.n_lattice)
    inst = np.repeat(np.arange(batch.n_inst), batch.n_lattice)
    d = rs - target
    J = np.zeros(batch.n_inst)
    np.add.at(J, inst, 0.5 * h * d * d)
    g = np.zeros(int(off[-1]))
    np.add.at(g, idx, h * d)
    return J, g


def target_samples(states, batch):
    rs, _ = I.sample_density(states, states["offsets"], batch.n_lattice, batch.x_left, batch.x_right)
    return rs


def per_instance_dot(offsets, a, b):
    out = np.zeros(len(offsets) - 1)
    for i in range(len(out)):
        s = slice(offsets[i], offsets[i + 1])
        out[i] = float(np.dot(a[s], b[s]))
    return out


def directions(batch, n_rand=3, seed=5):
    """Seed directions: tau of every instance; random density and momentum fields; the pair of widths at
    every phase boundary (+d, -d: the boundary moves by d)."""
    rng = np.random.default_rng(seed)
    M = int(batch.cell_offsets[-1])
    dirs = []
    zero = np.zeros(M)
    dirs.append({"tau": batch.tau.copy(), "rho": zero, "m": zero, "widths": zero})
    for _ in range(n_rand):
        dirs.append({"tau": np.zeros(batch.n_inst), "rho": rng.standard_normal(M) * batch.rho, "m": zero,
                     "widths": zero})
    for _ in range(n_rand):
        dirs.append({"tau": np.zeros(batch.n_inst), "rho": zero,
                     "m": rng.standard_normal(M) * np.maximum(np.abs(batch.m), batch.rho), "widths": zero})
    dw = np.zeros(M)
    flips = np.where(batch.phase[:-1] != batch.phase[1:])[0]
    for f in flips:
        inst = np.searchsorted(batch.cell_offsets, f, side="right") - 1
        if batch.cell_offsets[inst + 1] - 1 == f:
            continue  # instance boundary, not a phase boundary
        d = 1e-3 * min(batch.widths[f], batch.widths[f + 1])
        dw[f], dw[f + 1] = d, -d
    dirs.append({"tau": np.zeros(batch.n_inst), "rho": zero, "m": zero, "widths": dw})
    return dirs


def grad_dot(batch, g, d):
    """Per-instance directional derivative from an adjoint gradient."""
    off = batch.cell_offsets
    return (per_instance_dot(off, g["rho"], d["rho"]) + per_instance_dot(off, g["m"], d["m"])
            + per_instance_dot(off, g["widths"], d["widths"]) + g["tau"] * d["tau"])
