"""Pins of the CPU oracle against values the paper prints and facts the mathematics fixes.

These tests check the oracle itself (no GPU): the printed exact star states of the cavitation and
nucleation tests (Sec. 4.2/4.3), the printed saturation table, closed forms, special cases,
symmetry and finite-difference checks of the phase-boundary Jacobian.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import pyoracle as P
from paper_2211_00705_gb300 import inputs as I

with open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")) as _f:
    GOLD = json.load(_f)


def _liquid_rho(fl, p):
    return fl.rho0_liq + (p - fl.p_sat) / fl.a2_liq


def _fit_liquid_sound_speed():
    """The paper does not print the liquid sound speed; fit it to the printed exact u_L*^- of the
    cavitation test by bisection (u_L* decreases monotonically in a_L on [1400, 1600])."""
    g = GOLD["cavitation"]
    target = g["exact_u_liquid_star_left"]
    opts = I.Options()

    def u_star(a):
        fl = I.paper_fluid(a)
        r0 = _liquid_rho(fl, g["p_liquid"])
        r = P.creation_solve(fl, opts, I.tau_paper(), 1, r0, g["u_left"], r0, g["u_right"])
        assert r["status"] == 0
        return r["u_parent_l"]

    lo, hi = 1400.0, 1600.0
    flo = u_star(lo) - target
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        fm = u_star(mid) - target
        if (fm > 0) == (flo > 0):
            lo, flo = mid, fm
        else:
            hi = mid
    return 0.5 * (lo + hi)


@pytest.fixture(scope="module")
def a_liq():
    return _fit_liquid_sound_speed()


def test_vapour_constant_matches_printed_saturation_table():
    """k T0 / m from the constants of Eq. eos:isoT_idgas equals p_tilde / rho_tilde of the printed
    Table tab:max_vap_lintait363 (an ideal gas obeys p = (kT0/m) rho at every point)."""
    t = GOLD["saturation_table"]
    assert I.vapour_a2_paper() == pytest.approx(t["p_tilde"] / t["rho_tilde"], rel=2e-6)


def test_cavitation_exact_star_states(a_liq):
    """Single-phase liquid data with phase creation (App. B) against the printed exact solution of
    Sec. 4.2 (Tables tab:sol_dat_4_p/tab:sol_dat_4_u and the interface speeds in the text). One
    number (u_L*^-) was used to fit the unprinted liquid sound speed; the others are independent."""
    g = GOLD["cavitation"]
    assert 1450.0 < a_liq < 1510.0
    fl = I.paper_fluid(a_liq)
    r0 = _liquid_rho(fl, g["p_liquid"])
    r = P.creation_solve(fl, I.Options(), I.tau_paper(), 1, r0, g["u_left"], r0, g["u_right"])
    assert r["status"] == 0
    assert r["p_parent_l"] == pytest.approx(g["exact_p_liquid_star"], rel=5e-9)
    assert r["p_parent_r"] == pytest.approx(g["exact_p_liquid_star"], rel=5e-9)
    assert r["p_created"] == pytest.approx(g["exact_p_vapour_star"], rel=5e-9)
    assert abs(r["u_created"]) < 1e-9
    assert r["u_parent_r"] == pytest.approx(-g["exact_u_liquid_star_left"], abs=1e-6)
    assert r["w_r"] == pytest.approx(g["w_right"], abs=6e-7)
    assert r["w_l"] == pytest.approx(-g["w_right"], abs=6e-7)
    # created cell (w_r - w_l) dt with dt = C h / S_max, S_max = |u| + a_L of the initial data
    dt = g["cfl"] * g["h0"] / (abs(g["u_right"]) + a_liq)
    assert (r["w_r"] - r["w_l"]) * dt == pytest.approx(g["h_vapour_created"], rel=2e-4)


def test_nucleation_exact_star_states(a_liq):
    """Single-phase vapour data with liquid creation against the printed exact solution of Sec. 4.3
    (Tables tab:sol_dat_3_p/tab:sol_dat_3_u)."""
    g = GOLD["nucleation"]
    fl = I.paper_fluid(a_liq)
    rv = g["p_vapour"] / fl.a2_vap
    r = P.creation_solve(fl, I.Options(), I.tau_paper(), 0, rv, g["u_left"], rv, g["u_right"])
    assert r["status"] == 0
    assert r["p_parent_l"] == pytest.approx(g["exact_p_vapour_star"], rel=1e-10)
    assert r["p_created"] == pytest.approx(g["exact_p_liquid_star"], rel=1e-10)
    assert r["u_parent_l"] == pytest.approx(g["exact_u_vapour_star_left"], abs=1e-6)
    assert abs(r["u_created"]) < 1e-9
    assert r["w_r"] == pytest.approx(g["w_right"], abs=6e-7)


def test_two_phase_boundary_reproduces_the_printed_right_boundary(a_liq):
    """The right phase boundary of the printed cavitation solution, posed as a two-phase Riemann
    problem (vapour star | liquid star), is its own solution: the App. A solver returns the printed
    star pressures and boundary speed with both outer waves of zero strength."""
    g = GOLD["cavitation"]
    fl = I.paper_fluid(a_liq)
    rv = g["exact_p_vapour_star"] / fl.a2_vap
    rl = _liquid_rho(fl, g["exact_p_liquid_star"])
    r = P.pb_solve(fl, I.Options(), I.tau_paper(), 0, rv, 0.0, 1, rl, -g["exact_u_liquid_star_left"])
    assert r["status"] == 0
    assert r["p_l"] == pytest.approx(g["exact_p_vapour_star"], rel=1e-8)
    assert r["p_r"] == pytest.approx(g["exact_p_liquid_star"], rel=1e-8)
    assert r["w"] == pytest.approx(g["w_right"], abs=2e-6)


def _random_pb_cases(n=60, seed=7):
    rng = np.random.default_rng(seed)
    fl = I.workload_fluid()
    cases = []
    for _ in range(n):
        rl = rng.uniform(950, 1000)
        rv = rng.uniform(0.5, 1.0)
        ul, uv = rng.uniform(-50, 50, 2)
        tau = I.tau_paper() * 10 ** rng.uniform(-4, -2)
        cases.append((fl, tau, rl, ul, rv, uv))
    return cases


def test_pb_solution_satisfies_jump_conditions_and_entropy():
    """At the converged boundary state: mass and momentum jump conditions (Eq. jc:isoT), the kinetic
    relation (Eq. isoT:kin_rel1 with e_kin relative to the boundary) and the entropy inequality
    rho (u - w) [[g + e_kin]] <= 0 (Eq. isoT:entropy_ineq_1d)."""
    for fl, tau, rl, ul, rv, uv in _random_pb_cases():
        r = P.pb_solve(fl, I.Options(), tau, 1, rl, ul, 0, rv, uv)
        assert r["status"] == 0
        w, z = r["w"], r["z"]
        mass_l = r["rho_l"] * (r["u_l"] - w)
        mass_r = r["rho_r"] * (r["u_r"] - w)
        # liquid side: u_l* - w is a difference of O(10 m/s) numbers; allow rho_L * 1e-12 m/s
        assert mass_l == pytest.approx(-z, rel=1e-9, abs=1e-9)
        assert mass_r == pytest.approx(-z, rel=1e-9, abs=1e-9)
        mom_l = mass_l * r["u_l"] + r["p_l"]
        mom_r = mass_r * r["u_r"] + r["p_r"]
        assert mom_l == pytest.approx(mom_r, rel=1e-11)
        gl = fl.a2_liq * math.log(r["rho_l"] / fl.rho0_liq)
        gv = fl.a2_vap * math.log(r["rho_r"] / (fl.p_sat / fl.a2_vap))
        jump = (gv + 0.5 * (r["u_r"] - w) ** 2) - (gl + 0.5 * (r["u_l"] - w) ** 2)
        assert z == pytest.approx(tau * r["p_r"] * jump, rel=1e-6, abs=1e-12)
        assert -z * jump <= 1e-12
        # the flux through the moving face is the same from either side (Eq. pb_flux:pt)
        assert r["F0"] == pytest.approx(-z)
        assert r["F1"] == pytest.approx(mom_r, rel=1e-11)


def test_pb_mirror_symmetry():
    """x -> -x: swapping the sides and reversing velocities mirrors the solution: star pressures swap,
    w and the mass flux z change sign, the momentum flux is unchanged."""
    for fl, tau, rl, ul, rv, uv in _random_pb_cases(30, seed=11):
        a = P.pb_solve(fl, I.Options(), tau, 1, rl, ul, 0, rv, uv)
        b = P.pb_solve(fl, I.Options(), tau, 0, rv, -uv, 1, rl, -ul)
        assert a["status"] == 0 and b["status"] == 0
        assert b["p_l"] == pytest.approx(a["p_r"], rel=1e-11)
        assert b["p_r"] == pytest.approx(a["p_l"], rel=1e-11)
        assert b["w"] == pytest.approx(-a["w"], rel=1e-9, abs=1e-12)
        assert b["z"] == pytest.approx(-a["z"], rel=1e-8, abs=1e-14)
        assert b["F1"] == pytest.approx(a["F1"], rel=1e-11)


def test_pb_without_transfer_is_a_contact():
    """tau = 0 gives z = 0, hence [[p]] = 0 and [[u]] = 0 across the boundary (App. A, no phase
    transition)."""
    for fl, _, rl, ul, rv, uv in _random_pb_cases(20, seed=3):
        r = P.pb_solve(fl, I.Options(), 0.0, 1, rl, ul, 0, rv, uv)
        assert r["status"] == 0
        assert r["z"] == 0.0
        assert r["p_l"] == pytest.approx(r["p_r"], rel=1e-12)
        assert r["u_l"] == pytest.approx(r["u_r"], rel=1e-9, abs=1e-9)
        assert r["w"] == pytest.approx(r["u_r"], rel=1e-9, abs=1e-9)


def test_pb_jacobian_matches_finite_differences():
    """The analytic Jacobian of Eq. jacobian:ex_sys against central differences of G."""
    rng = np.random.default_rng(5)
    fl = I.workload_fluid()
    for _ in range(30):
        rl, rv = rng.uniform(955, 995), rng.uniform(0.5, 1.0)
        ul, uv = rng.uniform(-30, 30, 2)
        tau = I.tau_paper() * 10 ** rng.uniform(-3, 0)
        pl, pr = rng.uniform(2e4, 2e5, 2)
        J = P.pb_system(fl, tau, 1, rl, ul, 0, rv, uv, pl, pr)["J"]
        for j, (dl, dr) in enumerate([(1.0, 0.0), (0.0, 1.0)]):
            eps = 1e-4 * (pl if j == 0 else pr)
            gp = P.pb_system(fl, tau, 1, rl, ul, 0, rv, uv, pl + eps * dl, pr + eps * dr)["G"]
            gm = P.pb_system(fl, tau, 1, rl, ul, 0, rv, uv, pl - eps * dl, pr - eps * dr)["G"]
            fd = (gp - gm) / (2 * eps)
            np.testing.assert_allclose(J[:, j], fd, rtol=2e-6, atol=1e-12)


def test_wave_functions_by_quadrature():
    """With tau = 0 the boundary reduces to the classical two-wave problem; the velocity jump of a
    rarefaction equals the printed integral of v/a dp (App. A), evaluated here by quadrature."""
    fl = I.workload_fluid()
    rl, ul, rv, uv = 980.0, -20.0, 0.8, 20.0   # expansion: both outer waves are rarefactions
    r = P.pb_solve(fl, I.Options(), 0.0, 1, rl, ul, 0, rv, uv)
    assert r["status"] == 0
    pl0 = fl.p_sat + fl.a2_liq * (rl - fl.rho0_liq)
    ps = r["p_l"]
    assert ps < pl0
    zeta = np.linspace(pl0, ps, 200001)
    v = 1.0 / (fl.rho0_liq + (zeta - fl.p_sat) / fl.a2_liq)
    integral = np.trapezoid(v / math.sqrt(fl.a2_liq), zeta)
    assert (ul - r["u_l"]) == pytest.approx(integral, rel=1e-8)


def test_hll_consistency_and_upwind_limits():
    """HLL: F(U, U) = F(U); supersonic states take the upwind physical flux (Toro)."""
    fl = I.workload_fluid()
    rng = np.random.default_rng(1)
    for ph, a2 in ((0, fl.a2_vap), (1, fl.a2_liq)):
        for _ in range(20):
            r = rng.uniform(0.5, 1.0) if ph == 0 else rng.uniform(950, 1000)
            u = rng.uniform(-50, 50)
            p = a2 * r if ph == 0 else fl.p_sat + a2 * (r - fl.rho0_liq)
            F = P.hll(fl, ph, r, r * u, r, r * u)
            np.testing.assert_allclose(F, [r * u, r * u * u + p], rtol=1e-14, atol=1e-12)
    a = math.sqrt(fl.a2_vap)
    r1, u1, r2, u2 = 0.7, a + 100.0, 0.9, a + 150.0
    F = P.hll(fl, 0, r1, r1 * u1, r2, r2 * u2)
    np.testing.assert_allclose(F, [r1 * u1, r1 * u1 * u1 + fl.a2_vap * r1], rtol=1e-15)
    F = P.hll(fl, 0, r1, -r1 * u1, r2, -r2 * u2)
    np.testing.assert_allclose(F, [-r2 * u2, r2 * u2 * u2 + fl.a2_vap * r2], rtol=1e-15)


def test_hll_state_is_the_fan_average_of_the_exact_two_rarefaction_solution():
    """Integral consistency of HLL (Toro): when S_L, S_R bound every wave, the HLL intermediate state
    U* = U_L + (F_HLL - F_L)/S_L is the exact average of the Riemann solution over [S_L t, S_R t]. For two
    rarefactions in one phase (dp/drho = a^2 constant in both EOS of Sec. 2) the fan heads move at exactly
    u_l - a and u_r + a, the Davis estimates of reading R6. The exact solution (Riemann invariants
    u +- a ln rho; star state rho* = sqrt(rho_l rho_r) exp((u_l - u_r)/2a)) is integrated piecewise by
    quadrature and compared with U* from the oracle's flux, from both sides."""
    from scipy.integrate import quad
    fl = I.workload_fluid()
    rng = np.random.default_rng(5)
    for ph, a2 in ((0, fl.a2_vap), (1, fl.a2_liq)):
        a = math.sqrt(a2)
        p = (lambda r: a2 * r) if ph == 0 else (lambda r: fl.p_sat + a2 * (r - fl.rho0_liq))
        for _ in range(6):
            rl = rng.uniform(0.5, 1.0) if ph == 0 else rng.uniform(950, 1000)
            rr = rl * math.exp(rng.uniform(-0.01, 0.01))
            ul = rng.uniform(-40, 40)
            ur = ul + a * (abs(math.log(rl / rr)) + rng.uniform(0.01, 0.05))   # both waves rarefactions
            rs = math.sqrt(rl * rr) * math.exp((ul - ur) / (2 * a))
            us = ul + a * math.log(rl / rs)
            assert rs < min(rl, rr)

            def U(xi):
                if xi < ul - a:
                    return rl, rl * ul
                if xi < us - a:
                    u = xi + a
                    r = rl * math.exp((ul - u) / a)
                    return r, r * u
                if xi < us + a:
                    return rs, rs * us
                if xi < ur + a:
                    u = xi - a
                    r = rr * math.exp((u - ur) / a)
                    return r, r * u
                return rr, rr * ur

            SL, SR = ul - a, ur + a
            pts = [SL, us - a, us + a, SR]
            avg = [sum(quad(lambda x, k=k: U(x)[k], pts[i], pts[i + 1], epsabs=0, epsrel=1e-12, limit=200)[0]
                       for i in range(3)) / (SR - SL) for k in (0, 1)]
            F = np.array(P.hll(fl, ph, rl, rl * ul, rr, rr * ur))
            FL = np.array([rl * ul, rl * ul * ul + p(rl)])
            FR = np.array([rr * ur, rr * ur * ur + p(rr)])
            from_left = np.array([rl, rl * ul]) + (F - FL) / SL
            from_right = np.array([rr, rr * ur]) + (F - FR) / SR
            scale = np.array([rl, rl * a])
            np.testing.assert_allclose(from_left / scale, np.array(avg) / scale, rtol=0, atol=1e-11)
            np.testing.assert_allclose(from_right / scale, np.array(avg) / scale, rtol=0, atol=1e-11)


def test_nopt_star_pressure_by_brute_force():
    """Same-phase star pressure without transition: root of f(p; W_l) + f(p; W_r) + du found by a
    dense scan of the sign change, including shock-shock, shock-rarefaction and two-rarefaction data."""
    fl = I.workload_fluid(rho0_liq=1000.0)
    a = math.sqrt(fl.a2_liq)

    def f(p, r):
        pK = fl.p_sat + fl.a2_liq * (r - 1000.0)
        rs = 1000.0 + (p - fl.p_sat) / fl.a2_liq
        if p > pK:
            return math.sqrt((p - pK) * (1 / r - 1 / rs))
        return a * math.log(rs / r)

    for (rl, ul, rr, ur) in [(1000.0, -10.0, 1000.0, 10.0), (1000.0, 10.0, 1000.0, -10.0),
                             (1001.0, 5.0, 999.5, 3.0), (1000.2, -1.0, 1000.0, 30.0)]:
        ps = P.nopt_star(fl, 1, rl, ul, rr, ur)
        grid = np.linspace(ps - 2e4, ps + 2e4, 4001)
        phi = np.array([f(p, rl) + f(p, rr) + (ur - ul) for p in grid])
        k = np.where(np.diff(np.sign(phi)) != 0)[0]
        assert len(k) == 1
        assert abs(grid[k[0]] - ps) <= 10.0 + 1e-9 * abs(ps)
        assert abs(f(ps, rl) + f(ps, rr) + (ur - ul)) < 1e-9


def test_creation_mirror_and_conservation():
    """Cavitation data mirrored in x gives the mirrored cavity; the created cell's mass and momentum
    equal what the two boundaries withdraw from the neighbours (App. B fluxes with each boundary's
    own mass flux)."""
    fl = I.workload_fluid(rho0_liq=1000.0)
    for V in (10.0, 80.0, 200.0):
        r = P.creation_solve(fl, I.Options(), I.tau_paper(), 1, 1000.0, -V, 1000.2, V * 0.9)
        m = P.creation_solve(fl, I.Options(), I.tau_paper(), 1, 1000.2, -V * 0.9, 1000.0, V)
        assert r["status"] == 0 and m["status"] == 0
        assert m["p_created"] == pytest.approx(r["p_created"], rel=1e-11)
        assert m["w_l"] == pytest.approx(-r["w_r"], rel=1e-10)
        assert m["u_created"] == pytest.approx(-r["u_created"], rel=1e-6, abs=1e-9)
        # mass: rho_C (w_r - w_l) = z_r - z_l ; momentum: rho_C u_C (w_r - w_l) = (z_r - z_l) u_C
        assert r["rho_created"] * (r["w_r"] - r["w_l"]) == pytest.approx(r["z_r"] - r["z_l"], rel=1e-10)
