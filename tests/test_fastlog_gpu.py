"""The table-driven logarithm of the boundary solves against CUDA's log (ulp distance) and against
numpy's log (relative error), including arguments next to 1 where ln x is small."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ulps(a, b):
    ai = a.view(np.int64)
    bi = b.view(np.int64)
    return np.abs(ai - bi)


def test_fast_log_accuracy():
    from paper_2211_00705_gb300.imexds import check_log
    rng = np.random.default_rng(3)
    x = np.concatenate([np.exp(rng.uniform(-20, 20, 200000)), 1 + rng.uniform(-1e-3, 1e-3, 50000),
                        1 + rng.uniform(-1e-12, 1e-12, 1000), [1.0, 2.0, 0.5, np.sqrt(2), 1 / np.sqrt(2)]])
    x = x[x > 0]
    fast, ref = check_log(x)
    assert np.max(_ulps(fast, ref)) <= 4
    rel = np.abs(fast - np.log(x)) / np.maximum(np.abs(np.log(x)), 1e-300)
    assert np.max(rel[np.abs(np.log(x)) > 0]) < 1e-15
    assert fast[-5] == 0.0


def test_newton_raphson_quotient_against_division():
    """a * rcp_nr(b) against CUDA's correctly rounded division over the ranges the kernels use (densities
    1e-3..1e4, momenta and wave-speed spans of either sign): within 2 ulp."""
    import numpy as np
    from paper_2211_00705_gb300.imexds import check_div
    rng = np.random.default_rng(0)
    n = 1 << 20
    b = 10.0 ** rng.uniform(-3, 4, n)
    a = rng.standard_normal(n) * 10.0 ** rng.uniform(-3, 6, n)
    fast, ref = check_div(a, b)
    ulp = np.spacing(np.abs(ref))
    assert np.max(np.abs(fast - ref) / ulp) <= 2.0


def test_refined_reciprocal_against_division():
    """rcp_nr(b) alone (a = 1) against CUDA's correctly rounded 1 / b, within 1 ulp, over every binade the
    kernels use and mantissas spread over [1, 2), including the ends of the binade."""
    import numpy as np
    from paper_2211_00705_gb300.imexds import check_div
    rng = np.random.default_rng(5)
    n = 1 << 20
    mant = np.concatenate([rng.uniform(1.0, 2.0, n), 1.0 + np.arange(1, 2049) * 2.0 ** -52,
                           2.0 - np.arange(1, 2049) * 2.0 ** -52])
    b = np.ldexp(mant, rng.integers(-12, 40, mant.shape[0]))
    fast, ref = check_div(np.ones_like(b), b)
    assert np.max(np.abs(fast - ref) / np.spacing(np.abs(ref))) <= 1.0


def test_bit_pattern_stop_test_against_the_fp64_comparison():
    """The dual-time stop test |d| < lim max(|w|, 1), decided on bit patterns in integer instructions, gives
    the FP64 comparison's answer: random magnitudes over 600 decades, either sign, the boundary values
    (products rounded onto the limit, w = +-1, zeros of either sign, subnormals, infinities)."""
    from paper_2211_00705_gb300.imexds import check_tol
    rng = np.random.default_rng(11)
    n = 1 << 20
    w = rng.choice([-1.0, 1.0], n) * 10.0 ** rng.uniform(-300, 300, n)
    lim = 10.0 ** rng.uniform(-300, 0, n)
    m = np.maximum(np.abs(w), 1.0)
    d = rng.choice([-1.0, 1.0], n) * lim * m * rng.choice([0.5, 1.0, 2.0, 1.0 - 2.0 ** -52, 1.0 + 2.0 ** -52], n)
    tiny = np.array([0.0, -0.0, 5e-324, -5e-324, 2.2250738585072014e-308, np.inf, -np.inf, 1.0, -1.0])
    dd = np.concatenate([d, np.repeat(tiny, len(tiny)), tiny, np.full(len(tiny), 3e-9)])
    ww = np.concatenate([w, np.tile(tiny, len(tiny)), np.ones(len(tiny)), tiny])
    ll = np.concatenate([lim, np.full(len(tiny) ** 2, 3e-13), np.full(len(tiny), 5e-324), np.full(len(tiny), 3e-9)])
    fast, ref = check_tol(dd, ww, ll)
    assert 0.2 < ref.mean() < 0.8  # both outcomes are well represented
    np.testing.assert_array_equal(fast, ref)
