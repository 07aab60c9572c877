"""Pins for the sampled-Gaussian spatial kernel of the oracle (reading 1b:
the Gaussian of a given FWHM sampled at integer offsets within +-4 sigma, in
units of 1/1024 of the central sample, rounded, over the taps' sum).

Checked against what the mathematics and an independent library fix: the
Gaussian's second and fourth moments (sigma^2, 3 sigma^4), scipy.ndimage's
own sampled Gaussian filter, a direct 3-D convolution written with loops, the
closed form of a smoothed impulse, conservation of an interior source, a
constant interior, and a brute-force S+C on tiny cubes. The last test plants
plausible mistakes and checks that each trips at least one pin.
"""
import math

import numpy as np
import pytest

import oracle.sc_oracle as O

FWHM_C = math.sqrt(8.0 * math.log(2.0))
FWHMS = (2.0, 2.5, 3.0, 4.0, 5.0, 6.0, 7.3, 10.0, 15.0, 20.0)


def sigma_of(fwhm):
    return fwhm / FWHM_C


def bf_smooth_sampled(x, fwhm, wz):
    """Direct 3-D convolution with explicit loops over the composed kernel."""
    x = np.asarray(x, dtype=np.float64)
    nz, ny, nx = x.shape
    t = [int(v) for v in O.gauss_taps(fwhm)] if fwhm > 0 else [1]
    tot = float(sum(t))
    h = (len(t) - 1) // 2
    kxy = {d: t[d + h] / tot for d in range(-h, h + 1)}
    r = (wz - 1) // 2 if wz > 1 else 0
    out = np.zeros_like(x)
    for z in range(nz):
        for y in range(ny):
            for xx in range(nx):
                acc = 0.0
                for dz in range(-r, r + 1):
                    if not 0 <= z + dz < nz:
                        continue
                    for dy, wy in kxy.items():
                        if not 0 <= y + dy < ny:
                            continue
                        for dx, wx in kxy.items():
                            if 0 <= xx + dx < nx:
                                acc += wy * wx * x[z + dz, y + dy, xx + dx] / (2 * r + 1)
                out[z, y, xx] = acc
    return out


def bf_median(vals):
    s = sorted(vals)
    n = len(s)
    return 0.5 * (s[(n - 1) // 2] + s[n // 2])


def bf_sc_sampled(cube, kernels, t, n_repl):
    c = np.asarray(cube, dtype=np.float64)
    fin = np.isfinite(c)
    vals = [float(v) for v in c[fin]]
    med = bf_median(vals)
    s0 = 1.4826 * bf_median([abs(v - med) for v in vals])
    mask = np.zeros(c.shape, dtype=bool)
    sig = []
    for fs, wz in kernels:
        x = np.zeros_like(c)
        for idx in np.ndindex(c.shape):
            if fin[idx]:
                x[idx] = ((1.0 if c[idx] >= 0 else -1.0) * n_repl * s0) if (mask[idx] and n_repl > 0) else c[idx]
        s = bf_smooth_sampled(x, fs, wz)
        v = [float(s[i]) for i in np.ndindex(c.shape) if fin[i]]
        m = bf_median(v)
        sk = 1.4826 * bf_median([abs(a - m) for a in v])
        if sk > 0:
            for idx in np.ndindex(c.shape):
                if fin[idx] and abs(s[idx]) > t * sk:
                    mask[idx] = True
        sig.append(sk)
    return mask.astype(np.uint8), sig, s0


# ----------------------------------------------------------------------------
# Pins

def pin_taps_structure():
    """Support +-floor(4 sigma), symmetric, central tap 1024, falling outward."""
    for f in FWHMS:
        t = O.gauss_taps(f)
        h = int(math.floor(4.0 * sigma_of(f)))
        assert t.size == 2 * h + 1, f
        assert np.array_equal(t, t[::-1]), f
        assert t[h] == 1024, f
        assert np.all(np.diff(t[h:]) <= 0) and np.all(t >= 0), f
    assert O.gauss_taps(0.0).tolist() == [1024]
    # FWHM 2 px: sigma^2 = 1 / (2 ln 2), so the samples are powers of two
    assert O.gauss_taps(2.0).tolist() == [2, 64, 512, 1024, 512, 64, 2]


def pin_moments():
    """Unit sum; the Gaussian's second moment sigma^2 and fourth 3 sigma^4 (up to
    the rounding of the taps and the cut at 4 sigma)."""
    for f in FWHMS:
        s = sigma_of(f)
        k = O.kernel_1d(f, "sampled")
        h = (k.size - 1) // 2
        i = np.arange(-h, h + 1)
        assert abs(k.sum() - 1.0) < 1e-14
        assert abs((i * i * k).sum() / (s * s) - 1.0) < 1e-2, f
        assert abs((i ** 4 * k).sum() / (3.0 * s ** 4) - 1.0) < 4e-2, f


def pin_vs_scipy():
    """scipy.ndimage's sampled Gaussian (truncate = 4) on an impulse, 1-D and
    through the x and y passes of smooth: within 1e-3 of the peak."""
    ndimage = pytest.importorskip("scipy.ndimage")
    for f in FWHMS:
        s = sigma_of(f)
        k = O.kernel_1d(f, "sampled")
        h = (k.size - 1) // 2
        x = np.zeros(201)
        x[100] = 1.0
        g = ndimage.gaussian_filter1d(x, s, truncate=4.0, mode="constant")
        assert np.abs(g[100 - h:101 + h] - k).max() < 1e-3 * k.max(), f
        assert max(g[:100 - h].max(), g[101 + h:].max()) < 1e-3 * k.max(), f
    for f in (3.0, 6.0, 10.0):
        s = sigma_of(f)
        x = np.zeros((3, 61, 61))
        x[1, 30, 30] = 1.0
        got = O.smooth(x, f, 1, "sampled")
        ref = ndimage.gaussian_filter(x, (0.0, s, s), truncate=4.0, mode="constant")
        assert np.abs(got - ref).max() < 2e-3 * got.max(), f


def pin_smooth_bruteforce():
    rng = np.random.default_rng(31)
    for shape, fs, wz in [((5, 7, 8), 3.0, 3), ((4, 9, 13), 6.0, 1), ((7, 6, 5), 2.5, 7), ((3, 12, 4), 5.0, 15),
                          ((6, 5, 6), 0.0, 5)]:
        x = rng.standard_normal(shape)
        np.testing.assert_allclose(O.smooth(x, fs, wz, "sampled"), bf_smooth_sampled(x, fs, wz), rtol=0, atol=1e-12)


def pin_impulse_constant_and_edges():
    for f in (3.0, 6.0, 10.0):
        t = O.gauss_taps(f)
        for wz in (1, 7):
            x = np.zeros((21, 81, 81))
            x[10, 40, 40] = 1.0
            s = O.smooth(x, f, wz, "sampled")
            assert abs(s[10, 40, 40] - (1024.0 / t.sum()) ** 2 / wz) < 1e-15
            assert abs(s.sum() - 1.0) < 1e-12  # unit-sum kernel conserves an interior source
            assert s.max() == s[10, 40, 40]
    x = np.full((20, 50, 50), 2.5)
    s = O.smooth(x, 10.0, 7, "sampled")
    np.testing.assert_allclose(s[3:-3, 16:-16, 16:-16], 2.5, rtol=0, atol=1e-12)
    assert s[0, 0, 0] < 2.5  # zero padding, no renormalisation at the edges


def pin_sc_bruteforce():
    kernels = [(0.0, 0), (3.0, 0), (3.0, 3), (2.5, 1)]
    for seed in range(3):
        rng = np.random.default_rng(40 + seed)
        c = rng.standard_normal((5, 7, 6))
        c[tuple(int(rng.integers(0, n)) for n in c.shape)] += 7.0
        c[rng.random(c.shape) < 0.08] = np.nan
        c = c.astype(np.float32)
        for n_repl, t in ((2.0, 2.0), (0.0, 2.5)):
            m, sig, s0 = O.sc_filter(c, kernels, t, "mad", n_repl, spatial="sampled")
            bm, bsig, bs0 = bf_sc_sampled(c, kernels, t, n_repl)
            assert abs(s0 - bs0) < 1e-12
            np.testing.assert_allclose(sig, bsig, rtol=1e-12, atol=0)
            assert np.array_equal(m, bm), (seed, n_repl)


def pin_smoothed_at():
    rng = np.random.default_rng(33)
    x = rng.standard_normal((12, 30, 25))
    pts = np.stack([rng.integers(0, n, 40) for n in x.shape], axis=1)
    for fs, wz in ((3.0, 3), (6.0, 1), (10.0, 7)):
        ref = O.smooth(x, fs, wz, "sampled")
        got = O.smoothed_at(x, fs, wz, pts, "sampled")
        np.testing.assert_allclose(got, ref[tuple(pts.T)], rtol=0, atol=1e-12)


def pin_cascade_untouched():
    """The default spatial kernel is still the cascade, and the two differ."""
    x = np.zeros((3, 41, 41))
    x[1, 20, 20] = 1.0
    a = O.smooth(x, 6.0, 1)
    assert abs(a[1, 20, 20] - (19.0 / 125.0) ** 2) < 1e-15
    assert not np.allclose(a, O.smooth(x, 6.0, 1, "sampled"))


PINS = [pin_taps_structure, pin_moments, pin_vs_scipy, pin_smooth_bruteforce, pin_impulse_constant_and_edges,
        pin_sc_bruteforce, pin_smoothed_at, pin_cascade_untouched]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    pin()


# ----------------------------------------------------------------------------
# Planted mistakes

def _mut_taps_cut_3_sigma(orig):
    def f(fwhm):
        t = orig(fwhm)
        h = (t.size - 1) // 2
        c = int(math.floor(3.0 * fwhm / FWHM_C)) if fwhm > 0 else 0
        return t[h - c:h + c + 1] if c < h else t
    return f


def _mut_taps_sigma_half_fwhm(orig):
    def f(fwhm):
        return orig(fwhm * FWHM_C / 2.0)
    return f


def _mut_taps_no_half(orig):
    def f(fwhm):
        if not fwhm > 0:
            return orig(fwhm)
        s = fwhm / FWHM_C
        h = int(math.floor(4.0 * s))
        i = np.arange(-h, h + 1, dtype=np.float64)
        return np.rint(1024 * np.exp(-i * i / (s * s))).astype(np.int64)
    return f


def _mut_kernel_unnormalised(orig):
    def f(fwhm, spatial="cascade"):
        if spatial == "sampled":
            return O.gauss_taps(fwhm).astype(np.float64) / 1024.0
        return orig(fwhm, spatial)
    return f


def _mut_smooth_sampled_no_y(orig):
    def f(x, fwhm, wz, spatial="cascade"):
        if spatial != "sampled" or not fwhm > 0:
            return orig(x, fwhm, wz, spatial)
        k = O.kernel_1d(fwhm, "sampled")
        s = O.fir_along(np.asarray(x, dtype=np.float64), k, axis=2)
        return O.box_mean(s, wz, axis=0) if wz > 1 else s
    return f


def _mut_fir_off_by_one(orig):
    def f(x, k, axis):
        return np.roll(orig(x, k, axis), 1, axis=axis)
    return f


def _mut_fir_edge_renormalised(orig):
    def f(x, k, axis):
        ones = np.ones_like(x)
        return orig(x, k, axis) / orig(ones, k, axis)
    return f


MUTATIONS = [
    ("gauss_taps", _mut_taps_cut_3_sigma), ("gauss_taps", _mut_taps_sigma_half_fwhm),
    ("gauss_taps", _mut_taps_no_half), ("kernel_1d", _mut_kernel_unnormalised),
    ("smooth", _mut_smooth_sampled_no_y), ("fir_along", _mut_fir_off_by_one),
    ("fir_along", _mut_fir_edge_renormalised),
]


@pytest.mark.parametrize("name,mut", MUTATIONS, ids=[f"{n}-{m.__name__}" for n, m in MUTATIONS])
def test_planted_mistake_is_caught(monkeypatch, name, mut):
    monkeypatch.setattr(O, name, mut(getattr(O, name)))
    caught = []
    for pin in PINS:
        try:
            pin()
        except (AssertionError, ValueError, IndexError):
            caught.append(pin.__name__)
    assert caught, f"planted mistake in {name} ({mut.__name__}) passed every pin"
