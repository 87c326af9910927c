"""Seeded input generator: the splitmix64 reference outputs, workload shapes and layouts."""
import numpy as np

from paper_2211_00705_gb300 import inputs as I


def test_splitmix64_reference_outputs():
    """Published reference outputs of splitmix64 (Steele, Lea and Flood 2014) for seed 1234567."""
    r = I.SplitMix64([1234567])
    assert [int(r.next_u64()[0]) for _ in range(5)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
        16408922859458223821]


def test_riemann_layout_is_on_the_lattice():
    b = I.workload(1, scale=64 / 4096)
    for k in range(b.n_inst):
        a0, a1 = b.cell_offsets[k], b.cell_offsets[k + 1]
        N = b.n_lattice[k]
        assert a1 - a0 == N + 1
        assert abs(b.widths[a0:a1].sum() - 1.0) < 1e-12
        ph = b.phase[a0:a1]
        flips = np.where(ph[:-1] != ph[1:])[0]
        assert len(flips) == 1
        j = flips[0]
        alpha = b.widths[a0 + j + 1] * N
        assert 1e-6 * (1 - 1e-12) <= alpha <= 1e-1 * (1 + 1e-12)
        assert 200 <= N <= 2000
        assert b.tau[k] / I.tau_paper() >= 1e-4 * (1 - 1e-12) and b.tau[k] / I.tau_paper() <= 1e-2 * (1 + 1e-12)


def test_workloads_are_deterministic():
    a = I.workload(0)
    b = I.workload(0)
    np.testing.assert_array_equal(a.rho, b.rho)
    np.testing.assert_array_equal(a.m, b.m)


def test_cavitation_workload_shape():
    b = I.workload(4, scale=16 / 16384)
    for k in range(b.n_inst):
        a0, a1 = b.cell_offsets[k], b.cell_offsets[k + 1]
        u = b.m[a0:a1] / b.rho[a0:a1]
        n = b.n_lattice[k]
        assert (u[: n // 2] < 0).all() and (u[n // 2:] > 0).all()
        assert 10 <= u[-1] <= 200
        assert (b.phase[a0:a1] == 1).all()


def test_bench_workload_at_full_size():
    """The 4096-instance workload as generated: N uniform in [200, 2000] (sum ~ 4096 * 1100 cells), one
    liquid | vapour boundary per instance with liquid rho in [950, 1000], vapour rho in [0.5, 1] and u in
    [-50, 50] on both sides, widths summing to the domain, run to t_end = 2e-4 s."""
    b = I.workload(1)
    assert b.n_inst == 4096 and b.t_end == 2e-4
    assert (b.n_lattice >= 200).all() and (b.n_lattice <= 2000).all()
    assert 0.97 * 4096 * 1100 <= b.n_lattice.sum() <= 1.03 * 4096 * 1100
    np.testing.assert_array_equal(np.diff(b.cell_offsets), b.n_lattice + 1)
    inst = np.repeat(np.arange(b.n_inst), np.diff(b.cell_offsets))
    np.testing.assert_allclose(np.bincount(inst, weights=b.widths), 1.0, rtol=0, atol=1e-12)
    flips = np.nonzero((b.phase[:-1] != b.phase[1:]) & (inst[:-1] == inst[1:]))[0]
    assert len(flips) == b.n_inst
    assert (b.phase[flips] == 1).all() and (b.phase[flips + 1] == 0).all()   # liquid left, vapour right
    liq, vap = b.phase == 1, b.phase == 0
    assert (b.rho[liq] >= 950).all() and (b.rho[liq] <= 1000).all()
    assert (b.rho[vap] >= 0.5).all() and (b.rho[vap] <= 1.0).all()
    u = b.m / b.rho
    assert (np.abs(u) <= 50 * (1 + 1e-12)).all()


def test_fixed_step_and_adjoint_workloads():
    """1024 instances of N = 500, alpha = 1e-3, 2000 steps; the adjoint workload adds a per-cell jitter of at
    most 1e-3 and tightens the dual-time tolerances by 1e-4."""
    b = I.workload(3)
    assert b.n_inst == 1024 and (b.n_lattice == 500).all() and b.n_steps == 2000
    a = I.adjoint_batch(n_inst=8, n_lattice=500, n_steps=2000)
    base = I.workload(3, scale=8 / 1024)
    np.testing.assert_array_equal(a.widths, base.widths)
    assert np.max(np.abs(a.rho / base.rho - 1.0)) <= 1e-3
    assert np.max(np.abs(a.m - base.m) / base.rho) <= 1e-3
    assert a.options.tol_nb == base.options.tol_nb * 1e-4 and a.options.tol_k == base.options.tol_k * 1e-4


def test_bubble_domain_layout():
    """The bubble domain at reduced size: 2 boundaries per bubble, bubble spans of 2..20 lattice cells at
    least 4 liquid cells apart, tiny vapour pieces of fraction in [1e-6, 1e-1] at both ends of a bubble,
    liquid at rest at rho = 1000, vapour within 1 % of the saturation density."""
    n_cells, n_b = 4096, 64
    b = I.bubbles_domain(2, n_cells=n_cells, n_bubbles=n_b)
    h = 1.0 / n_cells
    assert b.n_inst == 1 and abs(b.widths.sum() - 1.0) < 1e-12
    ph = b.phase.astype(int)
    starts = np.nonzero(np.diff(ph) == -1)[0] + 1   # first vapour cell of each bubble
    ends = np.nonzero(np.diff(ph) == 1)[0]          # last vapour cell
    assert len(starts) == len(ends) == n_b
    x = np.concatenate([[0.0], np.cumsum(b.widths)])
    for s, e in zip(starts, ends):
        a1, a2 = b.widths[s] / h, b.widths[e] / h
        assert 1e-6 * (1 - 1e-9) <= a1 <= 1e-1 * (1 + 1e-9) and 1e-6 * (1 - 1e-9) <= a2 <= 1e-1 * (1 + 1e-9)
        span = (x[e + 1] - x[s]) / h + (1 - a1) + (1 - a2)   # lattice cells holding the bubble
        assert 2 - 1e-6 <= span <= 20 + 1e-6
    gaps = (x[starts[1:]] - x[ends[:-1] + 1]) / h       # liquid between consecutive bubbles
    assert gaps.min() >= 4 + 1 - 1e-6                    # the cut cells' liquid parts plus >= 4 lattice cells
    liq = b.phase == 1
    assert (b.rho[liq] == 1000.0).all() and (b.m == 0.0).all()
    rho_sat_v = b.fluid.p_sat / b.fluid.a2_vap
    assert np.max(np.abs(b.rho[~liq] / rho_sat_v - 1.0)) <= 0.01 * (1 + 1e-12)


def test_slab_creation_layout():
    """The slab instances: a valid cell list (faces on the lattice except the two boundaries), the slab's
    inner cells of width h, phases alternating out | slab | out, one velocity jump at the centre face."""
    b = I.slab_creation_batch(n_inst=6)
    for i in range(b.n_inst):
        s = slice(b.cell_offsets[i], b.cell_offsets[i + 1])
        w, ph, u = b.widths[s], b.phase[s], b.m[s] / b.rho[s]
        assert abs(w.sum() - 1.0) < 1e-12
        flips = np.nonzero(np.diff(ph.astype(int)))[0]
        assert len(flips) == 2
        slab = ph[flips[0] + 1]
        assert slab == (0 if i % 2 else 1)
        inner = w[flips[0] + 2:flips[1]]
        assert len(inner) >= 2 and np.allclose(inner, 1.0 / b.n_lattice[i])
        assert np.count_nonzero(np.abs(np.diff(u)) > 1e-9) == 1


def test_riemann_set_matches_single_riemann_instances():
    """riemann_set (fixed states at several N, the pseudo-time-step study's data) is the concatenation of the
    one-instance riemann_batch draws with those states, the boundary at the lattice midpoint and tau fixed."""
    Ns, alpha, tau = (100, 200, 400), 1e-4, 1e-2 * I.tau_paper()
    s = I.riemann_set(Ns, alpha, 972.0, -6.0, 0.40, 4.0, tau, t_end=2e-4)
    parts = []
    for N in Ns:
        b = I.riemann_batch(0, 1, n_range=(N, N), alpha_range=(alpha, alpha), coef_range=(1, 1),
                            rho_liq=(972.0, 972.0), rho_vap=(0.40, 0.40), u_range=(0, 0), pb_range=(0.5, 0.5))
        b.m[:] = np.where(b.phase == 1, b.rho * -6.0, b.rho * 4.0)
        parts.append(b)
    np.testing.assert_array_equal(s.n_lattice, Ns)
    np.testing.assert_array_equal(s.tau, np.full(3, tau))
    for f in ("rho", "m", "phase"):
        np.testing.assert_array_equal(getattr(s, f), np.concatenate([getattr(b, f) for b in parts]))
    # riemann_batch draws alpha log-uniformly, exp(log alpha) here: the tiny widths agree to rounding
    np.testing.assert_allclose(s.widths, np.concatenate([b.widths for b in parts]), rtol=1e-14, atol=0)
    np.testing.assert_array_equal(np.diff(s.cell_offsets), [N + 1 for N in Ns])
    assert s.t_end == 2e-4
