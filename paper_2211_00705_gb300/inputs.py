"""Seeded synthetic inputs for the explicit-implicit splitting scheme (arXiv 2211.00705).

This module only draws numbers and lays out cell lists; it holds none of the scheme's
arithmetic, and both the CUDA path and the CPU oracle take their inputs from it.

Random numbers: splitmix64 (Steele, Lea and Flood 2014) with 53-bit uniforms.
Seed of a workload = 221100705 + workload id; instance i draws from the stream
seed ^ (0x9E3779B97F4A7C15 * (i + 1)).

Kinetic coefficient: tau = c * tau_paper, where tau_paper = (2 pi)^{-1/2} (m / k T0)^{3/2} of Sec. 4
and c is the workload's coefficient (1 where a workload names none). Taken in SI units, the
coefficients 1e-4..1e-2 admit no Riemann solution for most of the drawn states: the vapour side
chokes at a mass flux of about rho_V* a_V while the kinetic relation asks for far more.

Grid layout of one instance (a reading of the "cut cell with volume fraction alpha" of
Sec. 3.1): background cells of width h = (x_R - x_L)/N; the phase boundary sits inside
background cell j at x_{j+1} - alpha h, splitting it into a (1 - alpha) h piece of the left
phase and an alpha h piece of the right phase (the tiny cell). Every other face is a
background-lattice face.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15

# ---------------------------------------------------------------- paper constants (Sec. 4)
BOLTZMANN = 1.380658e-23            # J/K (Eq. eos:isoT_idgas)
WATER_MOLECULE_MASS = (2 * 1.0079 + 15.9994) / 6.02205e26   # kg
T0_PAPER = 363.15                   # K (Table tab:init_dat_4)
P_SAT_PAPER = 70182.360745          # Pa, saturation pressure at T0 (Table tab:init_dat_4)
P_TILDE_PAPER = 70388.660656        # Pa, maximum vapour pressure (Table tab:max_vap_lintait363)
RHO_TILDE_PAPER = 0.419977          # kg/m^3
P_MIN_PAPER = 0.0                   # Pa, minimum liquid pressure
RHO_MIN_PAPER = 965.289008          # kg/m^3


def vapour_a2_paper() -> float:
    """k T0 / m of the ideal-gas vapour (Eq. eos:isoT_idgas)."""
    return BOLTZMANN * T0_PAPER / WATER_MOLECULE_MASS


def tau_paper() -> float:
    """Kinetic coefficient tau = (2 pi)^{-1/2} (m / k T0)^{3/2} (Sec. 4)."""
    return (1.0 / math.sqrt(2.0 * math.pi)) * (WATER_MOLECULE_MASS / (BOLTZMANN * T0_PAPER)) ** 1.5


@dataclasses.dataclass
class Fluid:
    """Two-phase isothermal fluid: vapour p = a_V^2 rho, liquid p = p0 + a_L^2 (rho - rho0)."""

    a2_vap: float
    a2_liq: float
    p_sat: float
    rho0_liq: float
    p_min: float
    p_tilde: float


def workload_fluid(a_vap: float = 415.0, a_liq: float = 1500.0, rho0_liq: float | None = None) -> Fluid:
    """EOS of the synthetic workloads. Without rho0_liq the liquid saturation density is
    rho_min + p_sat / a_L^2 (p = p_min = 0 at rho_min, Table tab:max_vap_lintait363)."""
    if rho0_liq is None:
        rho0_liq = RHO_MIN_PAPER + P_SAT_PAPER / (a_liq * a_liq)
    return Fluid(a2_vap=a_vap * a_vap, a2_liq=a_liq * a_liq, p_sat=P_SAT_PAPER, rho0_liq=rho0_liq,
                 p_min=P_MIN_PAPER, p_tilde=a_vap * a_vap * RHO_TILDE_PAPER)


def paper_fluid(a_liq: float) -> Fluid:
    """EOS of the paper's cavitation/nucleation tests at T0 = 363.15 K for a given liquid sound speed
    (the paper does not print it)."""
    return Fluid(a2_vap=vapour_a2_paper(), a2_liq=a_liq * a_liq, p_sat=P_SAT_PAPER,
                 rho0_liq=RHO_MIN_PAPER + P_SAT_PAPER / (a_liq * a_liq), p_min=P_MIN_PAPER,
                 p_tilde=P_TILDE_PAPER)


@dataclasses.dataclass
class Options:
    cfl: float = 0.5
    theta_nb: float = 0.9
    tol_nb: float = 1e-3
    tol_k: float = 1e-1
    res_mode: int = 0          # 0: residual as printed (1/s); 1: residual times dt
    l_max: int = 10000
    newton_tol: float = 1e-12
    newton_itmax: int = 50
    alpha_min: float = 1e-8
    split_ratio: float = 2.0
    creation: int = 0
    block_solver: int = 0      # 0: dual time stepping on each implicit block (Alg. 2); 1: Newton on its system


def scaled_options(**kw) -> Options:
    """Dimensionless residual (res * dt) with tolerances 1e-3 * 3e-6 and 1e-1 * 3e-6."""
    o = Options(res_mode=1, tol_nb=3e-9, tol_k=3e-7)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


@dataclasses.dataclass
class Batch:
    """Cell lists of a batch of instances, concatenated (phase 0 vapour, 1 liquid)."""

    n_lattice: np.ndarray    # int32 [n_inst]
    x_left: np.ndarray       # float64 [n_inst]
    x_right: np.ndarray      # float64 [n_inst]
    tau: np.ndarray          # float64 [n_inst]
    cell_offsets: np.ndarray # int32 [n_inst + 1]
    widths: np.ndarray       # float64 [n_cells]
    rho: np.ndarray          # float64 [n_cells]
    m: np.ndarray            # float64 [n_cells]
    phase: np.ndarray        # uint8 [n_cells]
    fluid: Fluid
    options: Options
    t_end: float = 0.0       # > 0: run to t_end
    n_steps: int = 0         # > 0: fixed number of steps
    name: str = ""

    @property
    def n_inst(self) -> int:
        return int(self.n_lattice.shape[0])

    def subset(self, idx) -> "Batch":
        idx = np.asarray(idx, dtype=np.int64)
        offs = self.cell_offsets
        parts = [np.arange(offs[i], offs[i + 1]) for i in idx]
        cells = np.concatenate(parts) if parts else np.zeros(0, np.int64)
        counts = np.array([offs[i + 1] - offs[i] for i in idx], dtype=np.int64)
        new_off = np.zeros(len(idx) + 1, dtype=np.int32)
        new_off[1:] = np.cumsum(counts)
        return dataclasses.replace(
            self, n_lattice=self.n_lattice[idx].copy(), x_left=self.x_left[idx].copy(),
            x_right=self.x_right[idx].copy(), tau=self.tau[idx].copy(), cell_offsets=new_off,
            widths=self.widths[cells].copy(), rho=self.rho[cells].copy(), m=self.m[cells].copy(),
            phase=self.phase[cells].copy())


# ---------------------------------------------------------------- splitmix64 streams
class SplitMix64:
    """Vectorised splitmix64: one independent stream per lane."""

    def __init__(self, seeds):
        self.state = np.asarray(seeds, dtype=np.uint64).copy()

    def next_u64(self) -> np.ndarray:
        with np.errstate(over="ignore"):
            self.state = self.state + np.uint64(GOLDEN)
            z = self.state.copy()
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            return z ^ (z >> np.uint64(31))

    def uniform(self) -> np.ndarray:
        """53-bit uniforms in [0, 1)."""
        return (self.next_u64() >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def instance_seeds(workload_id: int, n: int) -> np.ndarray:
    seed = 221100705 + workload_id
    i = np.arange(1, n + 1, dtype=object)
    return np.array([(seed ^ ((GOLDEN * int(k)) & MASK64)) & MASK64 for k in i], dtype=np.uint64)


def _riemann_cells(N, j, alpha, rho_l, u_l, ph_l, rho_r, u_r, ph_r):
    """Cell list of one Riemann instance on [0, 1]: lattice cells 0..j-1 left phase, the cut
    background cell j as (1-alpha) h | alpha h, lattice cells j+1..N-1 right phase."""
    h = 1.0 / N
    M = N + 1
    widths = np.full(M, h)
    widths[j] = (1.0 - alpha) * h
    widths[j + 1] = alpha * h
    rho = np.empty(M)
    m = np.empty(M)
    ph = np.empty(M, dtype=np.uint8)
    rho[: j + 1] = rho_l
    m[: j + 1] = rho_l * u_l
    ph[: j + 1] = ph_l
    rho[j + 1:] = rho_r
    m[j + 1:] = rho_r * u_r
    ph[j + 1:] = ph_r
    return widths, rho, m, ph


def _assemble(cells, n_lattice, tau, fluid, options, **kw) -> Batch:
    n = len(cells)
    counts = np.array([len(c[0]) for c in cells], dtype=np.int64)
    offs = np.zeros(n + 1, dtype=np.int32)
    offs[1:] = np.cumsum(counts)
    return Batch(n_lattice=np.asarray(n_lattice, dtype=np.int32), x_left=np.zeros(n), x_right=np.ones(n),
                 tau=np.asarray(tau, dtype=np.float64), cell_offsets=offs,
                 widths=np.concatenate([c[0] for c in cells]), rho=np.concatenate([c[1] for c in cells]),
                 m=np.concatenate([c[2] for c in cells]), phase=np.concatenate([c[3] for c in cells]),
                 fluid=fluid, options=options, **kw)


def riemann_batch(workload_id: int, n_inst: int, n_range=(100, 100), alpha_range=(1e-3, 1e-3),
                  coef_range=(1e-3, 1e-3), rho_liq=(950.0, 1000.0), rho_vap=(0.5, 1.0), u_range=(-50.0, 50.0),
                  pb_range=(0.35, 0.65), fluid: Fluid | None = None, options: Options | None = None,
                  t_end: float = 2e-4, n_steps: int = 0, name: str = "") -> Batch:
    """Liquid | vapour Riemann instances (workloads 0, 1 and 3): per instance draw N uniform-integer in
    n_range, the cut cell j = floor(U[pb_range] N), alpha log-uniform in alpha_range, the kinetic
    coefficient c log-uniform in coef_range (tau = c * tau_paper), one liquid and one vapour state
    (rho uniform, u uniform)."""
    fluid = fluid or workload_fluid()
    options = options or Options()
    rng = SplitMix64(instance_seeds(workload_id, n_inst))
    uN, uj, ua, ut, url, uul, urv, uuv = (rng.uniform() for _ in range(8))
    N = n_range[0] + np.floor(uN * (n_range[1] - n_range[0] + 1)).astype(np.int64)
    N = np.minimum(N, n_range[1])
    j = np.floor((pb_range[0] + uj * (pb_range[1] - pb_range[0])) * N).astype(np.int64)
    la0, la1 = math.log(alpha_range[0]), math.log(alpha_range[1])
    alpha = np.exp(la0 + ua * (la1 - la0))
    lt0, lt1 = math.log(coef_range[0]), math.log(coef_range[1])
    tau = np.exp(lt0 + ut * (lt1 - lt0)) * tau_paper()
    rl = rho_liq[0] + url * (rho_liq[1] - rho_liq[0])
    ul = u_range[0] + uul * (u_range[1] - u_range[0])
    rv = rho_vap[0] + urv * (rho_vap[1] - rho_vap[0])
    uv = u_range[0] + uuv * (u_range[1] - u_range[0])
    cells = [_riemann_cells(int(N[i]), int(j[i]), float(alpha[i]), rl[i], ul[i], 1, rv[i], uv[i], 0)
             for i in range(n_inst)]
    return _assemble(cells, N, tau, fluid, options, t_end=t_end, n_steps=n_steps, name=name)


def riemann_set(n_lattice, alpha: float, rho_liq: float, u_liq: float, rho_vap: float, u_vap: float, tau: float,
                options: Options | None = None, fluid: Fluid | None = None, t_end: float = 2e-4, n_steps: int = 0,
                name: str = "") -> Batch:
    """Fixed liquid | vapour Riemann data at several lattice sizes, one instance per entry of n_lattice: the
    boundary in background cell N // 2 with the tiny vapour piece alpha h (the layout of riemann_batch), the
    same states and kinetic coefficient tau in every instance (the pseudo-time-step study of Sec. 4.1)."""
    fluid = fluid or workload_fluid()
    options = options or Options()
    ns = [int(N) for N in n_lattice]
    cells = [_riemann_cells(N, N // 2, alpha, rho_liq, u_liq, 1, rho_vap, u_vap, 0) for N in ns]
    return _assemble(cells, np.array(ns), np.full(len(ns), float(tau)), fluid, options, t_end=t_end,
                     n_steps=n_steps, name=name)


def jitter_states(batch: Batch, workload_id: int, eps: float = 1e-3) -> Batch:
    """Per-cell jitter of the states: rho (1 + eps U[-1,1]), m + eps rho U[-1,1] (1 m/s). The discrete
    scheme is not differentiable where the CFL maximum is attained by several cells at once (piecewise
    constant data); the jitter makes it unique, so gradient checks compare derivatives, not one-sided
    slopes. Streams: one splitmix64 lane per cell, seeded from (1000 + workload_id, cell index)."""
    n = int(batch.cell_offsets[-1])
    rng = SplitMix64(instance_seeds(1000 + workload_id, n))
    a, b = rng.uniform(), rng.uniform()
    return dataclasses.replace(batch, rho=batch.rho * (1.0 + eps * (2.0 * a - 1.0)),
                               m=batch.m + eps * batch.rho * (2.0 * b - 1.0))


def adjoint_batch(n_inst: int = 1024, n_lattice: int = 500, n_steps: int = 2000, tol_scale: float = 1e-4,
                  jitter: float = 1e-3, workload_id: int = 3) -> Batch:
    """The adjoint workload: Riemann instances as in workload 3 (N cells, alpha = 1e-3, tau = 1e-3 tau_paper,
    states as workload 0) with jittered states and dual-time tolerances tightened by tol_scale, so that
    the forward run is the converged implicit scheme that the adjoint differentiates."""
    b = riemann_batch(workload_id, n_inst, n_range=(n_lattice, n_lattice), alpha_range=(1e-3, 1e-3),
                      coef_range=(1e-3, 1e-3),
                      options=scaled_options(tol_nb=3e-9 * tol_scale, tol_k=3e-7 * tol_scale), t_end=0.0,
                      n_steps=n_steps, name=f"{n_inst} Riemann instances, N={n_lattice}, {n_steps} steps, adjoint")
    return jitter_states(b, workload_id, jitter) if jitter > 0 else b


def sample_density(batch_or_states, offsets, n_lattice, x_left, x_right):
    """rho at the background cell centres x_j of every instance (piecewise-constant sampling of the cell
    list) and, per sample, the index of the cell that holds it. Returns (rho_samples, cell_index) with
    one entry per background cell, instances concatenated."""
    w, r = batch_or_states["widths"], batch_or_states["rho"]
    out_r, out_i = [], []
    for i in range(len(n_lattice)):
        a, b = int(offsets[i]), int(offsets[i + 1])
        N = int(n_lattice[i])
        h = (x_right[i] - x_left[i]) / N
        xc = x_left[i] + (np.arange(N) + 0.5) * h
        edges = x_left[i] + np.concatenate([[0.0], np.cumsum(w[a:b])])
        k = np.clip(np.searchsorted(edges, xc, side="right") - 1, 0, b - a - 1)
        out_r.append(r[a + k])
        out_i.append(a + k)
    return np.concatenate(out_r), np.concatenate(out_i)


def workload(wid: int, scale: float = 1.0) -> Batch:
    """The five synthetic workloads. scale < 1 shrinks instance counts (not sizes) for tests."""
    if wid == 0:
        return riemann_batch(0, 1, n_range=(100, 100), alpha_range=(1e-3, 1e-3), coef_range=(1e-3, 1e-3),
                             options=Options(), t_end=2e-4,
                             name="single Riemann instance, N=100, alpha=1e-3, tau=1e-3, t_end=2e-4 s")
    if wid == 1:
        n = max(1, int(round(4096 * scale)))
        return riemann_batch(1, n, n_range=(200, 2000), alpha_range=(1e-6, 1e-1), coef_range=(1e-4, 1e-2),
                             options=scaled_options(), t_end=2e-4,
                             name=f"{n} Riemann instances, N in [200,2000], alpha in [1e-6,1e-1], t_end=2e-4 s")
    if wid == 3:
        n = max(1, int(round(1024 * scale)))
        return riemann_batch(3, n, n_range=(500, 500), alpha_range=(1e-3, 1e-3), coef_range=(1e-3, 1e-3),
                             options=scaled_options(), t_end=0.0, n_steps=2000,
                             name=f"{n} Riemann instances, N=500, 2000 steps")
    if wid == 4:
        n = max(1, int(round(16384 * scale)))
        return cavitation_batch(4, n, name=f"{n} cavitation instances, N in [64,4096], 5000 steps")
    if wid == 2:
        return bubbles_domain(2, n_cells=1 << 24, n_bubbles=1024,
                              name="one domain of 2^24 cells with 1024 vapour bubbles, 1000 steps")
    raise ValueError(wid)


def cavitation_batch(workload_id: int, n_inst: int, n_range=(64, 4096), v_range=(10.0, 200.0),
                     n_steps: int = 5000, name: str = "") -> Batch:
    """Pure liquid at rest density rho0 = 1000 (read as the saturation density) with u = -V left of face
    floor(N/2) and +V right of it, V uniform in v_range (workload 4, phase creation)."""
    fluid = workload_fluid(rho0_liq=1000.0)
    rng = SplitMix64(instance_seeds(workload_id, n_inst))
    uN, uV = rng.uniform(), rng.uniform()
    N = np.minimum(n_range[0] + np.floor(uN * (n_range[1] - n_range[0] + 1)).astype(np.int64), n_range[1])
    V = v_range[0] + uV * (v_range[1] - v_range[0])
    cells = []
    for i in range(n_inst):
        n = int(N[i])
        h = 1.0 / n
        widths = np.full(n, h)
        rho = np.full(n, 1000.0)
        u = np.where(np.arange(n) < n // 2, -V[i], V[i])
        cells.append((widths, rho, rho * u, np.ones(n, dtype=np.uint8)))
    return _assemble(cells, N, np.full(n_inst, tau_paper()), fluid, scaled_options(creation=1), n_steps=n_steps,
                     name=name)


def nucleation_batch(workload_id: int, n_inst: int, n_range=(64, 1024), v_range=(14.0, 16.0), n_steps: int = 500,
                     p_vap: float = 70000.0, name: str = "") -> Batch:
    """Pure vapour at pressure p_vap (below p_sat, as in the paper's nucleation test, Sec. 4.3) with
    u = +V left of face floor(N/2) and -V right of it (compression), V uniform in v_range: the same-phase
    star pressure at the centre exceeds the maximum vapour pressure and a liquid cell nucleates there
    (App. B, the mirror of workload 4). With the workload fluid (a_V = 415 m/s, p_tilde = 72.3 kPa) the
    threshold lies near V = 13.5 m/s; V in [14, 16] nucleates exactly one droplet that persists (faster
    collisions supersaturate the post-shock vapour and nucleate several droplets, whose vapour gaps then
    vanish, a case the method does not treat)."""
    fluid = workload_fluid(rho0_liq=1000.0)
    rng = SplitMix64(instance_seeds(workload_id, n_inst))
    uN, uV = rng.uniform(), rng.uniform()
    N = np.minimum(n_range[0] + np.floor(uN * (n_range[1] - n_range[0] + 1)).astype(np.int64), n_range[1])
    V = v_range[0] + uV * (v_range[1] - v_range[0])
    rho_v = p_vap / fluid.a2_vap
    cells = []
    for i in range(n_inst):
        n = int(N[i])
        h = 1.0 / n
        u = np.where(np.arange(n) < n // 2, V[i], -V[i])
        rho = np.full(n, rho_v)
        cells.append((np.full(n, h), rho, rho * u, np.zeros(n, dtype=np.uint8)))
    return _assemble(cells, N, np.full(n_inst, tau_paper()), fluid, scaled_options(creation=1), n_steps=n_steps,
                     name=name or f"{n_inst} nucleation instances, N in {list(n_range)}, {n_steps} steps")


def slab_creation_batch(workload_id: int = 6, n_inst: int = 8, n_lattice: int = 64, slab_range=(4, 5),
                        alpha_cav=(0.08, 0.2), alpha_nuc=(1e-4, 1e-2), v_cav=(20.0, 60.0), v_nuc=(14.0, 16.0),
                        n_steps: int = 40, name: str = "") -> Batch:
    """A slab of S lattice cells (S uniform-integer in slab_range) of one phase between two regions of the
    other, every cell left of the slab's centre face moving at -V and every cell right of it at +V: even
    instances hold a liquid slab in vapour pulled apart (V in v_cav: cavitation at the centre face), odd
    instances a vapour slab in liquid compressed (u = +V left, -V right, V in v_nuc: nucleation). Both
    boundaries sit inside the slab's end lattice cells with the tiny piece (fraction alpha, log-uniform in
    alpha_cav or alpha_nuc) outside the slab, so the slab's inner cells lie in no implicit neighbourhood and the
    centre face is a face between two explicit cells; the two boundary neighbourhoods are fewer than four lattice
    cells apart. A pulled-apart slab's boundaries move outwards into the tiny pieces: alpha_cav and v_cav keep
    those pieces above half their width in the first step (no merge), so the centre face cavitates in step 1.
    Both phases at saturation (liquid rho0 = 1000 read as the saturation density)."""
    fluid = workload_fluid(rho0_liq=1000.0)
    rng = SplitMix64(instance_seeds(workload_id, n_inst))
    uS, uV, ua1, ua2 = rng.uniform(), rng.uniform(), rng.uniform(), rng.uniform()
    rho_v = fluid.p_sat / fluid.a2_vap
    cells = []
    for i in range(n_inst):
        n = n_lattice
        h = 1.0 / n
        S = min(slab_range[0] + int(uS[i] * (slab_range[1] - slab_range[0] + 1)), slab_range[1])
        nuc = (i % 2) == 1
        lo, hi = (v_nuc if nuc else v_cav)
        V = lo + uV[i] * (hi - lo)
        ar = alpha_nuc if nuc else alpha_cav
        la0, la1 = math.log(ar[0]), math.log(ar[1])
        a1 = math.exp(la0 + ua1[i] * (la1 - la0))
        a2 = math.exp(la0 + ua2[i] * (la1 - la0))
        slab_ph, out_ph = (0, 1) if nuc else (1, 0)
        rho_of = {0: rho_v, 1: 1000.0}
        s0 = n // 2 - S // 2
        c = s0 + S // 2                       # centre face (lattice face index)
        w, ph, x0 = [], [], []
        for j in range(s0):
            w.append(h); ph.append(out_ph); x0.append(j * h)
        w += [a1 * h, (1.0 - a1) * h]; ph += [out_ph, slab_ph]; x0 += [s0 * h, (s0 + a1) * h]
        for j in range(s0 + 1, s0 + S - 1):
            w.append(h); ph.append(slab_ph); x0.append(j * h)
        j = s0 + S - 1
        w += [(1.0 - a2) * h, a2 * h]; ph += [slab_ph, out_ph]; x0 += [j * h, (j + 1 - a2) * h]
        for j in range(s0 + S, n):
            w.append(h); ph.append(out_ph); x0.append(j * h)
        w, ph, x0 = np.array(w), np.array(ph, np.uint8), np.array(x0)
        rho = np.array([rho_of[int(p)] for p in ph])
        left = x0 < c * h - 0.5 * h * 1e-9
        u = np.where(left, V if nuc else -V, -V if nuc else V)
        cells.append((w, rho, rho * u, ph))
    return _assemble(cells, [n_lattice] * n_inst, np.full(n_inst, tau_paper()), fluid, scaled_options(creation=1),
                     n_steps=n_steps, name=name or f"{n_inst} slab creation instances, N={n_lattice}, {n_steps} steps")


def bubbles_domain(workload_id: int, n_cells: int = 1 << 24, n_bubbles: int = 1024, width_range=(2, 20),
                   alpha_range=(1e-6, 1e-1), n_steps: int = 1000, gap: int = 4, name: str = "") -> Batch:
    """One liquid domain on [0, 1] (rho = rho0 = 1000, u = 0) with vapour bubbles (workload 2). A bubble of
    W background cells starting at cell s has its two phase boundaries inside cells s and s+W-1, each cut
    so that the tiny piece (fraction alpha, log-uniform) lies inside the bubble. Vapour density
    p_sat/a_V^2 (1 + 0.01 U[-1,1]). Bubbles closer than `gap` cells to another are redrawn."""
    fluid = workload_fluid(rho0_liq=1000.0)
    rng = SplitMix64(instance_seeds(workload_id, 1))
    starts, widths_b = [], []
    occupied = np.zeros(n_cells + 2 * gap + 64, dtype=bool)
    while len(starts) < n_bubbles:
        W = width_range[0] + int(rng.uniform()[0] * (width_range[1] - width_range[0] + 1))
        W = min(W, width_range[1])
        s = 8 + int(rng.uniform()[0] * (n_cells - 16 - W))
        lo, hi = s - gap, s + W + gap
        if occupied[lo:hi].any():
            continue
        occupied[s:s + W] = True
        starts.append(s)
        widths_b.append(W)
    order = np.argsort(starts)
    starts = np.array(starts)[order]
    widths_b = np.array(widths_b)[order]
    la0, la1 = math.log(alpha_range[0]), math.log(alpha_range[1])
    rho_v0 = fluid.p_sat / fluid.a2_vap
    h = 1.0 / n_cells
    w_list, r_list, m_list, p_list = [], [], [], []
    prev = 0
    for s, W in zip(starts, widths_b):
        a1 = math.exp(la0 + rng.uniform()[0] * (la1 - la0))
        a2 = math.exp(la0 + rng.uniform()[0] * (la1 - la0))
        rv = rho_v0 * (1.0 + 0.01 * (2.0 * rng.uniform()[0] - 1.0))
        nl = s - prev   # liquid lattice cells before the bubble
        w_list.append(np.full(nl, h)); r_list.append(np.full(nl, 1000.0)); p_list.append(np.ones(nl, np.uint8))
        # cut cell s: liquid (1 - a1) h | vapour a1 h ; bubble interior ; cut cell s+W-1: vapour a2 h | liquid (1-a2) h
        bw = [(1.0 - a1) * h, a1 * h] + [h] * (W - 2) + [a2 * h, (1.0 - a2) * h]
        br = [1000.0, rv] + [rv] * (W - 2) + [rv, 1000.0]
        bp = [1, 0] + [0] * (W - 2) + [0, 1]
        w_list.append(np.array(bw)); r_list.append(np.array(br)); p_list.append(np.array(bp, np.uint8))
        prev = s + W
    nl = n_cells - prev
    w_list.append(np.full(nl, h)); r_list.append(np.full(nl, 1000.0)); p_list.append(np.ones(nl, np.uint8))
    widths = np.concatenate(w_list)
    rho = np.concatenate(r_list)
    cells = [(widths, rho, np.zeros_like(rho), np.concatenate(p_list))]
    return _assemble(cells, [n_cells], [tau_paper()], fluid, scaled_options(), n_steps=n_steps, name=name)
