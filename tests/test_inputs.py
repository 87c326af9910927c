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
