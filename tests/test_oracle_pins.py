"""Pins for the CPU oracle (oracle/sc_oracle.py), checked against things other
than the oracle itself: hand-derived closed forms (tests/golden), brute force
in pure Python on tiny cubes, the standard library and independent numpy
routines, and invariants that the mathematics fixes. The last test plants
plausible mistakes in the oracle and checks that every one of them trips at
least one pin.
"""
import json
import math
import os
import statistics

import numpy as np
import pytest

import oracle.sc_oracle as O

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))
FWHM_C = math.sqrt(8.0 * math.log(2.0))


# ----------------------------------------------------------------------------
# Brute-force references, written independently of the oracle's code.

def bf_widths(fwhm):
    """Among all 3-box cascades of odd widths that differ by at most 2, the one
    whose variance sum((w^2-1)/12) is closest to sigma^2 (the property the
    Kovesi construction is built to satisfy)."""
    if fwhm <= 0:
        return ()
    s2 = (fwhm / FWHM_C) ** 2
    best = None
    for wl in range(1, 80, 2):
        for m in range(0, 4):
            ws = tuple(sorted([wl] * m + [wl + 2] * (3 - m)))
            var = sum((w * w - 1) / 12.0 for w in ws)
            key = abs(var - s2)
            if best is None or key < best[0] - 1e-12:
                best = (key, ws)
    return best[1]


def bf_kernel(widths):
    """Composed 1-D kernel as {offset: weight} by enumerating every tap combination."""
    k = {0: 1.0}
    for w in widths:
        r = (w - 1) // 2
        nk = {}
        for off, val in k.items():
            for d in range(-r, r + 1):
                nk[off + d] = nk.get(off + d, 0.0) + val / w
        k = nk
    return k


def bf_smooth(x, fwhm, wz):
    """Direct 3-D convolution with explicit loops; x is a nested-list-like array."""
    x = np.asarray(x, dtype=np.float64)
    nz, ny, nx = x.shape
    kxy = bf_kernel(bf_widths(fwhm))
    r = (wz - 1) // 2 if wz > 1 else 0
    kz = {d: 1.0 / (2 * r + 1) for d in range(-r, r + 1)}
    out = np.zeros_like(x)
    for z in range(nz):
        for y in range(ny):
            for xx in range(nx):
                acc = 0.0
                for dz, wzv in kz.items():
                    if not 0 <= z + dz < nz:
                        continue
                    for dy, wy in kxy.items():
                        if not 0 <= y + dy < ny:
                            continue
                        for dx, wx in kxy.items():
                            if 0 <= xx + dx < nx:
                                acc += wzv * wy * wx * x[z + dz, y + dy, xx + dx]
                out[z, y, xx] = acc
    return out


def bf_median(vals):
    s = sorted(vals)
    n = len(s)
    return 0.5 * (s[(n - 1) // 2] + s[n // 2])


def bf_noise(vals, mode):
    if mode == "mad":
        m = bf_median(vals)
        return 1.4826 * bf_median([abs(v - m) for v in vals])
    return statistics.stdev(vals)


def bf_sc(cube, kernels, t, mode, n_repl):
    c = np.asarray(cube, dtype=np.float64)
    fin = np.isfinite(c)
    sigma0 = bf_noise([float(v) for v in c[fin]], mode)
    mask = np.zeros(c.shape, dtype=bool)
    sigmas = []
    for fs, wz in kernels:
        x = np.zeros_like(c)
        for idx in np.ndindex(c.shape):
            if not fin[idx]:
                continue
            if mask[idx] and n_repl > 0:
                x[idx] = (1.0 if c[idx] >= 0 else -1.0) * n_repl * sigma0
            else:
                x[idx] = c[idx]
        s = bf_smooth(x, fs, wz)
        vals = [float(s[i]) for i in np.ndindex(c.shape) if fin[i]]
        sk = bf_noise(vals, mode)
        if sk > 0:
            for idx in np.ndindex(c.shape):
                if fin[idx] and abs(s[idx]) > t * sk:
                    mask[idx] = True
        sigmas.append(sk)
    return mask.astype(np.uint8), sigmas, sigma0


def tiny_cube(seed, shape=(5, 6, 7), nan_frac=0.08, bright=3):
    rng = np.random.default_rng(seed)
    c = rng.standard_normal(shape)
    for _ in range(bright):
        idx = tuple(int(rng.integers(0, n)) for n in shape)
        c[idx] += float(rng.choice([-1, 1])) * rng.uniform(4, 9)
    c[rng.random(shape) < nan_frac] = np.nan
    return c.astype(np.float32)


# ----------------------------------------------------------------------------
# Pins, as plain functions so that the mutation test can rerun them.

def pin_widths_golden():
    for f, row in GOLDEN["cascade_widths"].items():
        assert tuple(O.cascade_widths(float(f))) == tuple(row["widths"]), f


def pin_widths_bruteforce():
    for f in np.linspace(0.3, 30.0, 167):
        assert tuple(O.cascade_widths(float(f))) == bf_widths(float(f)), f
    assert O.cascade_widths(0.0) == ()


def pin_effective_fwhm():
    for f, v in GOLDEN["effective_fwhm"].items():
        if f == "derivation":
            continue
        var = sum((w * w - 1) / 12.0 for w in O.cascade_widths(float(f)))
        assert abs(FWHM_C * math.sqrt(var) - v) < 1e-3


def pin_box_vs_numpy_convolve():
    rng = np.random.default_rng(1)
    for w in (1, 3, 5, 7, 9, 15, 31):
        for n in (1, 4, 17, 40):
            x = rng.standard_normal((3, n))
            got = O.box_mean(x, w, axis=1)
            ref = np.stack([np.convolve(row, np.full(w, 1.0 / w))[(w - 1) // 2:(w - 1) // 2 + n] for row in x])
            np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)


def pin_smooth_bruteforce():
    rng = np.random.default_rng(2)
    for shape, fs, wz in [((6, 7, 8), 3.0, 3), ((9, 5, 12), 6.0, 7), ((12, 12, 12), 5.0, 15),
                          ((4, 11, 3), 10.0, 1), ((7, 3, 9), 0.0, 5), ((5, 5, 5), 2.2, 31)]:
        x = rng.standard_normal(shape)
        np.testing.assert_allclose(O.smooth(x, fs, wz), bf_smooth(x, fs, wz), rtol=0, atol=1e-12)


def pin_impulse_closed_form():
    for f, row in GOLDEN["central_coefficient_1d"].items():
        cnum, cden = row["value"]
        for wz in (1, 3, 7, 15):
            x = np.zeros((41, 41, 41))
            x[20, 20, 20] = 1.0
            s = O.smooth(x, float(f), wz)
            assert abs(s[20, 20, 20] - (cnum / cden) ** 2 / wz) < 1e-14
            assert abs(s.sum() - 1.0) < 1e-12  # unit-sum kernel conserves an interior source
            assert s.max() == s[20, 20, 20]


def pin_constant_interior():
    x = np.full((40, 40, 40), 2.5)
    s = O.smooth(x, 10.0, 15)
    np.testing.assert_allclose(s[7:-7, 11:-11, 11:-11], 2.5, rtol=0, atol=1e-12)
    assert s[0, 0, 0] < 2.5  # zero padding, no renormalisation at the edges


def pin_kernel_1d():
    for f in (3.0, 5.0, 6.0, 10.0, 4.4):
        k = O.kernel_1d(f)
        ref = bf_kernel(bf_widths(f))
        assert k.size == len(ref)
        h = (k.size - 1) // 2
        for off, v in ref.items():
            assert abs(k[off + h] - v) < 1e-15


def pin_median_sorted():
    rng = np.random.default_rng(3)
    cases = [[1.0], [2.0, 1.0], [3.0, 1.0, 2.0], [0.0, -0.0, 0.0, 1.0], [5.0] * 7, [1.0, 1.0, 2.0, 2.0],
             list(rng.standard_normal(101)), list(rng.standard_normal(100)), list(rng.integers(-3, 3, 64) * 1.0),
             [1e-40, -1e-40, 3e-39, 0.0, 2e-45]]
    for v in cases:
        assert O.median(np.array(v)) == bf_median(v)
        assert O.median(np.array(v)) == statistics.median(v)


def pin_noise():
    g = GOLDEN["mad_example"]
    assert abs(O.noise(np.array(g["values"], dtype=float), "mad") - g["sigma"]) < 1e-12
    rng = np.random.default_rng(4)
    for n in (2, 3, 10, 51):
        v = list(rng.standard_normal(n) * 3 + 1)
        assert abs(O.noise(np.array(v), "mad") - bf_noise(v, "mad")) < 1e-12
        assert abs(O.noise(np.array(v), "std") - statistics.stdev(v)) < 1e-12
    big = rng.standard_normal(400_000)
    assert abs(O.noise(big, "mad") - 1.0) < 4.0 / math.sqrt(big.size)  # 1.4826 MAD of N(0,1) -> 1
    assert abs(O.noise(big, "std") - 1.0) < 4.0 / math.sqrt(big.size)


def pin_sc_bruteforce():
    kernels = [(0.0, 0), (0.0, 3), (3.0, 0), (3.0, 3)]
    for seed in range(4):
        c = tiny_cube(seed)
        for mode, n_repl, t in (("mad", 2.0, 2.5), ("mad", 0.0, 2.5), ("std", 1.5, 2.0), ("mad", 1.0, 1.5)):
            m, sig, s0 = O.sc_filter(c, kernels, t, mode, n_repl)
            bm, bsig, bs0 = bf_sc(c, kernels, t, mode, n_repl)
            assert abs(s0 - bs0) < 1e-12
            np.testing.assert_allclose(sig, bsig, rtol=1e-12, atol=0)
            assert np.array_equal(m, bm), (seed, mode, n_repl)


def pin_threshold_finder():
    rng = np.random.default_rng(5)
    c = rng.standard_normal((8, 9, 10)).astype(np.float32)
    c[0, 0, :4] = np.nan
    m, sig, s0 = O.sc_filter(c, [(0.0, 0)], 2.0, "mad", 2.0)
    fin = np.isfinite(c)
    vals = [float(v) for v in c[fin]]
    s_ref = 1.4826 * statistics.median([abs(v - statistics.median(vals)) for v in vals])
    assert abs(s0 - s_ref) < 1e-12 and abs(sig[0] - s_ref) < 1e-12
    assert np.array_equal(m.astype(bool), fin & (np.abs(c.astype(np.float64)) > 2.0 * s_ref))


def pin_invariants():
    c = tiny_cube(11, shape=(10, 12, 11), nan_frac=0.05, bright=6)
    ks = [(0.0, 0), (0.0, 3), (3.0, 0), (3.0, 3), (5.0, 7)]
    # replacement off: mask is an OR of independent clips, so order does not matter
    m1, s1, _ = O.sc_filter(c, ks, 2.5, "mad", 0.0)
    m2, s2, _ = O.sc_filter(c, ks[::-1], 2.5, "mad", 0.0)
    assert np.array_equal(m1, m2) and np.allclose(s1, s2[::-1], rtol=0, atol=0)
    # replacement off: mask shrinks as the threshold grows
    prev = None
    for t in (1.0, 1.5, 2.0, 3.0, 5.0, 1e9):
        m, _, _ = O.sc_filter(c, ks, t, "mad", 0.0)
        if prev is not None:
            assert not np.any(m & ~prev)
        prev = m
    assert not prev.any()  # t -> infinity gives an empty mask
    # NaN voxels never enter the mask; the smoothed cube is NaN exactly there
    m, _, _, ss = O.sc_filter(c, ks, 1.0, "mad", 2.0, return_smoothed=True)
    fin = np.isfinite(c)
    assert not m[~fin].any()
    for s in ss:
        assert np.array_equal(np.isfinite(s), fin)


def pin_replacement_identity():
    # Voxels the first pair detects all hold +-V exactly; with n*sigma0 = V the
    # replacement changes nothing, so the result equals replacement off.
    rng = np.random.default_rng(7)
    c = np.clip(rng.standard_normal((9, 10, 11)), -3, 3)
    pos = [(1, 2, 3), (4, 5, 6), (7, 1, 9), (2, 8, 2), (5, 5, 5)]
    v = 12.0
    for i, p in enumerate(pos):
        c[p] = v if i % 2 == 0 else -v
    c = c.astype(np.float32)
    vals = [float(x) for x in c.ravel()]
    med = statistics.median(vals)
    s0 = 1.4826 * statistics.median([abs(x - med) for x in vals])
    ks = [(0.0, 0), (3.0, 3), (5.0, 7)]
    t = 5.0
    m_off, sig_off, _ = O.sc_filter(c, ks, t, "mad", 0.0)
    m_id, sig_id, _ = O.sc_filter(c, ks, t, "mad", v / s0)
    assert np.array_equal(m_off, m_id)
    np.testing.assert_allclose(sig_id, sig_off, rtol=1e-12)
    # and a different replacement value does change the smoothed statistics
    _, sig_2, _ = O.sc_filter(c, ks, t, "mad", 2.0)
    assert not np.allclose(sig_2[1:], sig_off[1:], rtol=1e-9)


def pin_smoothed_at():
    rng = np.random.default_rng(8)
    x = rng.standard_normal((20, 30, 25))
    pts = np.stack([rng.integers(0, n, 40) for n in x.shape], axis=1)
    for fs, wz in ((0.0, 1), (3.0, 3), (6.0, 15), (10.0, 7)):
        ref = O.smooth(x, fs, wz)
        got = O.smoothed_at(x, fs, wz, pts)
        np.testing.assert_allclose(got, ref[tuple(pts.T)], rtol=0, atol=1e-12)


PINS = [pin_widths_golden, pin_widths_bruteforce, pin_effective_fwhm, pin_box_vs_numpy_convolve,
        pin_smooth_bruteforce, pin_impulse_closed_form, pin_constant_interior, pin_kernel_1d,
        pin_median_sorted, pin_noise, pin_sc_bruteforce, pin_threshold_finder, pin_invariants,
        pin_replacement_identity, pin_smoothed_at]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    pin()


# ----------------------------------------------------------------------------
# Planted mistakes: each must make at least one pin fail.

def _mut_box_offcentre(orig):
    def f(x, w, axis):
        out = orig(x, w, axis)
        return np.roll(out, 1, axis=axis) if w > 1 else out
    return f


def _mut_widths_m_plus(orig):
    def f(fwhm, n=3):
        w = orig(fwhm, n)
        return tuple(sorted(w[1:] + (w[0] + 2,))) if len(w) == 3 and w[0] != w[-1] else w
    return f


def _mut_replace_sign(orig):
    def f(c, mask, finite, value):
        x = orig(c, mask, finite, value)
        return np.where(mask & finite & (value > 0), -x, x)
    return f


def _mut_mad_about_zero(orig):
    def f(v, mode="mad"):
        if mode == "mad":
            return O.MAD_TO_SIGMA * O.median(np.abs(np.asarray(v, dtype=np.float64)))
        return orig(v, mode)
    return f


def _mut_median_lower(orig):
    def f(v):
        v = np.sort(np.asarray(v, dtype=np.float64))
        return float(v[(v.size - 1) // 2])
    return f


def _mut_smooth_no_y(orig):
    def f(x, fwhm, wz, spatial="cascade"):
        if spatial != "cascade":
            return orig(x, fwhm, wz, spatial)
        s = np.asarray(x, dtype=np.float64)
        for w in O.cascade_widths(fwhm):
            s = O.box_mean(s, w, axis=2)
        for w in O.cascade_widths(fwhm):
            s = O.box_mean(s, w, axis=2)
        return O.box_mean(s, wz, axis=0) if wz > 1 else s
    return f


def _mut_smooth_z_narrow(orig):
    def f(x, fwhm, wz, spatial="cascade"):
        return orig(x, fwhm, wz - 2 if wz > 3 else wz, spatial)
    return f


def _mut_sc_sigmak_replacement(orig):
    # replacement value taken from the previous pair's sigma instead of sigma_0
    def f(cube, kernels, threshold, noise_mode="mad", replacement=2.0, mask=None, return_smoothed=False,
          spatial="cascade"):
        c = np.asarray(cube, dtype=np.float64)
        fin = np.isfinite(c)
        s0 = O.noise(c[fin], noise_mode)
        m = np.zeros(c.shape, dtype=bool)
        last = s0
        sig, ss = [], []
        for fs, wz in kernels:
            s = O.smoothed(c, m, fs, wz, replacement * last if replacement > 0 else 0.0, spatial)
            ok = np.isfinite(s)
            sk = O.noise(s[ok], noise_mode)
            m |= ok & (np.abs(s) > threshold * sk)
            sig.append(sk)
            ss.append(s)
            last = sk
        out = (m.astype(np.uint8), sig, s0)
        return out + (ss,) if return_smoothed else out
    return f


def _mut_no_reblank(orig):
    def f(c, mask, fwhm, wz, value, spatial="cascade"):
        c = np.asarray(c, dtype=np.float64)
        fin = np.isfinite(c)
        return O.smooth(O.replaced_input(c, mask, fin, value), fwhm, wz, spatial)
    return f


def _mut_smooth_truncate_each_pass(orig):
    # zero padding applied again after every boxcar (intermediates cut at the edge)
    def f(x, fwhm, wz, spatial="cascade"):
        if spatial != "cascade":
            return orig(x, fwhm, wz, spatial)
        s = np.asarray(x, dtype=np.float64)
        for w in O.cascade_widths(fwhm):
            s = O.box_mean(s, w, axis=2)
        for w in O.cascade_widths(fwhm):
            s = O.box_mean(s, w, axis=1)
        return O.box_mean(s, wz, axis=0) if wz > 1 else s
    return f


def _mut_clip_positive_only(orig):
    # only positive excursions enter the mask (the paper keeps both signs)
    def f(cube, kernels, threshold, noise_mode="mad", replacement=2.0, mask=None, return_smoothed=False,
          spatial="cascade"):
        c = np.asarray(cube, dtype=np.float64)
        fin = np.isfinite(c)
        s0 = O.noise(c[fin], noise_mode)
        m = np.zeros(c.shape, dtype=bool)
        sig, ss = [], []
        for fs, wz in kernels:
            s = O.smoothed(c, m, fs, wz, replacement * s0 if replacement > 0 else 0.0, spatial)
            ok = np.isfinite(s)
            sk = O.noise(s[ok], noise_mode)
            if sk > 0:
                m |= ok & (np.nan_to_num(s) > threshold * sk)
            sig.append(sk)
            ss.append(s)
        out = (m.astype(np.uint8), sig, s0)
        return out + (ss,) if return_smoothed else out
    return f


def _mut_std_biased(orig):
    def f(v, mode="mad"):
        if mode == "std":
            v = np.asarray(v, dtype=np.float64)
            return math.sqrt(float(((v - v.mean()) ** 2).sum()) / v.size)
        return orig(v, mode)
    return f


def _mut_kernel1d_flip(orig):
    def f(fwhm, spatial="cascade"):
        k = orig(fwhm, spatial)
        return np.roll(k, 1)
    return f


def _mut_smoothed_at_transposed(orig):
    def f(x, fwhm, wz, points, spatial="cascade"):
        return orig(np.swapaxes(x, 0, 2).copy() if x.shape[0] == x.shape[2] else x[::-1], fwhm, wz, points, spatial)
    return f


MUTATIONS = [
    ("box_mean", _mut_box_offcentre), ("cascade_widths", _mut_widths_m_plus),
    ("replaced_input", _mut_replace_sign), ("noise", _mut_mad_about_zero), ("median", _mut_median_lower),
    ("smooth", _mut_smooth_no_y), ("smooth", _mut_smooth_z_narrow), ("sc_filter", _mut_sc_sigmak_replacement),
    ("smoothed", _mut_no_reblank), ("noise", _mut_std_biased), ("kernel_1d", _mut_kernel1d_flip),
    ("smoothed_at", _mut_smoothed_at_transposed), ("smooth", _mut_smooth_truncate_each_pass),
    ("sc_filter", _mut_clip_positive_only),
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
