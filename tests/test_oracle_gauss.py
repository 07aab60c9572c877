"""Pins for the Gaussian-fit noise mode of the oracle (oracle/sc_oracle.py,
reading 7b), checked against things other than the oracle itself: a histogram
worked out by hand, an independent binning (np.histogram on the bin edges), a
general least-squares solver (scipy.optimize.least_squares) and a brute-force
grid over the fit's objective, exact Gaussian counts, exact invariances, the
known behaviour on Gaussian noise with and without an emission tail, and
planted mistakes that must each trip a pin.
"""
import numpy as np
import pytest
from scipy.optimize import least_squares

import oracle.sc_oracle as O

XI = (np.arange(256) + 0.5) / 128.0 - 1.0  # bin centres, stated once more for the independent solvers


def objective(h, tau):
    """min over A of sum (h - A g)^2, by a 1-parameter linear least squares."""
    g = np.exp(-XI ** 2 / (2.0 * tau * tau))
    a = np.linalg.lstsq(g[:, None], np.asarray(h, dtype=np.float64), rcond=None)[0][0]
    return float(np.sum((h - a * g) ** 2))


def test_histogram_worked_by_hand():
    """Nine values: sorted -3, -1, -1, -1, 1, 1, 1, 3, 50. Median 1; |v - 1| =
    4, 2, 2, 2, 0, 0, 0, 2, 49, median 2, so sigma_M = 2 * 1.4826 = 2.9652 and
    k = 128 / 14.826 = 8.63348 bins per unit. Bins: -3 -> floor(-25.9) + 128 =
    102, -1 -> floor(-8.63) + 128 = 119, 1 -> 8 + 128 = 136, 3 -> 25 + 128 =
    153; 50 -> 431.7, outside the 256 bins."""
    v = np.array([-3, -1, -1, -1, 1, 1, 1, 3, 50], dtype=np.float64)
    s_mad = O.noise(v, "mad")
    assert s_mad == pytest.approx(2.9652, rel=1e-15)
    assert float(O.gauss_scale(s_mad)) == pytest.approx(8.63348, rel=1e-6)
    h = O.gauss_histogram(v, s_mad)
    expect = np.zeros(256, dtype=np.int64)
    expect[102], expect[119], expect[136], expect[153] = 1, 3, 3, 1
    np.testing.assert_array_equal(h, expect)


@pytest.mark.parametrize("seed", [0, 1])
def test_histogram_matches_np_histogram(seed):
    """np.histogram (binary search over the 257 edges (j - 128) / k) agrees
    wherever a value is not within float32 rounding of an edge."""
    rng = np.random.default_rng(seed)
    v = (rng.standard_normal(200_000) * rng.uniform(0.5, 4.0)).astype(np.float32).astype(np.float64)
    s_mad = O.noise(v, "mad")
    k = float(O.gauss_scale(s_mad))
    q = v * k
    keep = np.abs(q - np.round(q)) > 1e-4  # drop values next to an edge
    edges = (np.arange(257) - 128) / k
    ref, _ = np.histogram(v[keep], bins=edges)
    np.testing.assert_array_equal(O.gauss_histogram(v[keep], s_mad), ref)


@pytest.mark.parametrize("tau0,amp", [(0.1, 1.0), (0.2, 3.5e4), (0.35, 17.0), (0.6, 2.0e6)])
def test_fit_recovers_exact_gaussian_counts(tau0, amp):
    """Counts that are exactly A exp(-xi^2 / (2 tau0^2)): the residual is zero
    at tau0, so tau0 is the least-squares answer."""
    h = amp * np.exp(-XI ** 2 / (2.0 * tau0 * tau0))
    assert O.gauss_fit(h) == pytest.approx(tau0, rel=1e-12)


@pytest.mark.parametrize("seed,tau0", [(0, 0.2), (1, 0.12), (2, 0.3), (3, 0.5)])
def test_fit_matches_general_least_squares(seed, tau0):
    """Poisson counts around a Gaussian: the same minimum as a Levenberg-Marquardt
    fit of both parameters, and no point of a 4000-step grid over the bracket
    has a lower objective."""
    rng = np.random.default_rng(seed)
    lam = 4000.0 * np.exp(-XI ** 2 / (2.0 * tau0 * tau0)) + 3.0
    h = rng.poisson(lam).astype(np.float64)
    tau = O.gauss_fit(h)
    r = least_squares(lambda p: h - p[0] * np.exp(-XI ** 2 / (2.0 * p[1] * p[1])), x0=[h.max(), 0.25],
                      method="lm", xtol=1e-15, ftol=1e-15, gtol=1e-15)
    assert tau == pytest.approx(abs(r.x[1]), rel=1e-8)
    grid = np.linspace(0.05, 0.8, 4000)
    assert objective(h, tau) <= min(objective(h, t) for t in grid) * (1.0 + 1e-12)


def test_gaussian_noise_and_emission_tail():
    """Gaussian noise: within 0.5 % of the true sigma (2e6 values). With 2 %
    of the voxels turned into bright positive emission the fit stays within
    0.5 % while the standard deviation grows by more than 40 %."""
    rng = np.random.default_rng(5)
    v = (rng.standard_normal(2_000_000) * 1.7).astype(np.float32).astype(np.float64)
    assert O.noise(v, "gauss") == pytest.approx(1.7, rel=5e-3)
    v[:40_000] = np.abs(v[:40_000]) * 6.0 + 5.0
    assert O.noise(v, "gauss") == pytest.approx(1.7, rel=5e-3)
    assert O.noise(v, "std") > 1.4 * 1.7


def test_invariances():
    """Doubling the data doubles the noise exactly (k halves exactly, the same
    bins fill); mirroring the data mirrors the histogram, and the fit, which
    sees only xi^2, gives the same noise up to the order of its sums."""
    rng = np.random.default_rng(7)
    v = (rng.standard_normal(100_001) * 0.37 + 0.02).astype(np.float32).astype(np.float64)
    g = O.noise(v, "gauss")
    assert O.noise(2.0 * v, "gauss") == 2.0 * g
    s_mad = O.noise(v, "mad")
    q = v.astype(np.float32) * O.gauss_scale(s_mad)
    assert not np.any(q == np.floor(q))  # no value on an edge: floor(-q) = -floor(q) - 1
    np.testing.assert_array_equal(O.gauss_histogram(-v, s_mad), O.gauss_histogram(v, s_mad)[::-1])
    assert O.noise(-v, "gauss") == pytest.approx(g, rel=1e-12)


def test_degenerate():
    """sigma_M = 0 gives 0; data whose bulk lies far from 0 leave the histogram
    (centred at 0) empty, the bracket does not straddle a root, and the noise
    falls back to sigma_M."""
    assert O.noise(np.full(11, 3.25), "gauss") == 0.0
    rng = np.random.default_rng(3)
    v = (rng.standard_normal(5000) + 100.0).astype(np.float32).astype(np.float64)
    assert O.gauss_fit(O.gauss_histogram(v, O.noise(v, "mad"))) is None
    assert O.noise(v, "gauss") == O.noise(v, "mad")


PINS = [test_histogram_worked_by_hand, lambda: test_histogram_matches_np_histogram(0),
        lambda: test_fit_recovers_exact_gaussian_counts(0.2, 3.5e4),
        lambda: test_fit_matches_general_least_squares(0, 0.2), test_gaussian_noise_and_emission_tail,
        test_invariances, test_degenerate]


def _mut_centres_no_half(orig):
    return lambda: np.arange(256) / 128.0 - 1.0


def _mut_tau_not_squared(orig):
    def f(h):
        t = orig(h)
        return None if t is None else t * t / 0.2
    return f


def _mut_range_4(orig):
    return lambda s: np.float32(128.0 / (4.0 * s))


def _mut_no_profile(orig):
    def f(h):  # fits the shape with A fixed at 1
        x2 = XI ** 2
        lo, hi = O.GAUSS_TAU_BRACKET
        d = lambda t: float(np.sum((np.asarray(h) - np.exp(-x2 / (2 * t * t))) * x2 * np.exp(-x2 / (2 * t * t))))
        if not (d(lo) > 0 > d(hi)):
            return None
        for _ in range(80):
            mid = 0.5 * (lo + hi)
            lo, hi = (mid, hi) if d(mid) > 0 else (lo, mid)
        return 0.5 * (lo + hi)
    return f


def _mut_floor_as_trunc(orig):
    def f(v, s_mad):
        k = O.gauss_scale(s_mad)
        q = np.trunc(np.asarray(v, dtype=np.float32) * k)
        q = q[(q >= -128) & (q < 128)]
        return np.bincount(q.astype(np.int64) + 128, minlength=256).astype(np.int64)
    return f


MUTATIONS = [("gauss_bin_centres", _mut_centres_no_half), ("gauss_fit", _mut_tau_not_squared),
             ("gauss_scale", _mut_range_4), ("gauss_fit", _mut_no_profile),
             ("gauss_histogram", _mut_floor_as_trunc)]


@pytest.mark.parametrize("name,mut", MUTATIONS, ids=[f"{n}-{m.__name__}" for n, m in MUTATIONS])
def test_planted_mistake_is_caught(monkeypatch, name, mut):
    monkeypatch.setattr(O, name, mut(getattr(O, name)))
    caught = []
    for pin in PINS:
        try:
            pin()
        except (AssertionError, ValueError, IndexError, TypeError):
            caught.append(pin)
    assert caught, f"planted mistake in {name} ({mut.__name__}) passed every pin"
