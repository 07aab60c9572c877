"""Pins for the auto-flagger oracle (oracle/flagger.py), checked against things
other than the oracle itself: pure-Python brute force with the statistics
module on tiny cubes, cubes whose channel and pixel noises have closed forms,
degenerate cases, and planted mistakes that must each trip a pin.
"""
import math
import statistics

import numpy as np
import pytest

import oracle.flagger as FL


def bf_noise(vals):
    vals = [float(v) for v in vals if math.isfinite(float(v))]
    if not vals:
        return math.nan
    m = statistics.median(vals)
    return float(np.float32(1.4826 * statistics.median([abs(v - m) for v in vals])))


def bf_flags(noises, k):
    vals = [v for v in noises if math.isfinite(v)]
    if not vals:
        return [False] * len(noises)
    m = statistics.median(vals)
    r = 1.4826 * statistics.median([abs(v - m) for v in vals])
    return [math.isfinite(v) and abs(v - m) > k * r for v in noises]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_brute_force_tiny(seed):
    rng = np.random.default_rng(seed)
    c = (rng.standard_normal((9, 5, 6)) * rng.uniform(0.5, 3.0, (9, 1, 1))).astype(np.float32)
    c[rng.random(c.shape) < 0.1] = np.nan
    c[4] = np.nan  # a channel without finite voxels
    nz, ny, nx = c.shape
    cn = [bf_noise(c[z].ravel()) for z in range(nz)]
    pn = [bf_noise(c[:, y, x]) for y in range(ny) for x in range(nx)]
    np.testing.assert_array_equal(FL.channel_noise(c), np.array(cn, dtype=np.float32))
    np.testing.assert_array_equal(FL.pixel_noise(c).ravel(), np.array(pn, dtype=np.float32))
    out, fc, fp = FL.autoflag(c, 1.5)
    assert list(fc) == bf_flags(cn, 1.5)
    assert list(fp.ravel()) == bf_flags(pn, 1.5)
    ref = c.copy()
    for z in range(nz):
        if fc[z]:
            ref[z] = np.nan
    for i, f in enumerate(bf_flags(pn, 1.5)):
        if f:
            ref[:, i // nx, i % nx] = np.nan
    assert np.array_equal(np.isnan(out), np.isnan(ref)) and np.array_equal(out[~np.isnan(out)], ref[~np.isnan(ref)])


def pattern(shape):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return ((x + y + z) % 3 - 1).astype(np.float64)  # every full 3-period row balanced


def test_channel_closed_form():
    """Channel c holds a_c * s with s balanced over {-1, 0, 1} in every plane
    (9 x 9 planes): median 0, MAD a_c, noise 1.4826 a_c. Most a_c lie in
    [1, 1.07]; channels 3 and 7 have a = 5 and channel 9 a = 0.1."""
    s = pattern((12, 9, 9))
    a = np.array([1.0 + 0.01 * (c % 8) for c in range(12)])
    a[3], a[7], a[9] = 5.0, 5.0, 0.1
    c = (s * a[:, None, None]).astype(np.float32)
    noise = FL.channel_noise(c)
    # the cube stores fl32(a_c), so the MAD is fl32(a_c) exactly
    np.testing.assert_array_equal(noise, (1.4826 * a.astype(np.float32).astype(np.float64)).astype(np.float32))
    _, fc, fp = FL.autoflag(c, 4.0, pixels=False)
    assert np.flatnonzero(fc).tolist() == [3, 7, 9]
    assert not fp.any()


def test_pixel_closed_form():
    """Spectra of 27 channels with the balanced pattern; pixel (2, 5) scaled by
    4 and pixel (6, 1) by 0.25, the others by 1 + 0.02 * ((x + y) mod 5)."""
    s = pattern((27, 8, 8))
    ny, nx = 8, 8
    scale = 1.0 + 0.02 * ((np.arange(nx)[None, :] + np.arange(ny)[:, None]) % 5)
    scale[2, 5], scale[6, 1] = 4.0, 0.25
    c = (s * scale[None, :, :]).astype(np.float32)
    np.testing.assert_array_equal(FL.pixel_noise(c),
                                  (1.4826 * scale.astype(np.float32).astype(np.float64)).astype(np.float32))
    out, fc, fp = FL.autoflag(c, 4.0, channels=False)
    assert sorted(map(tuple, np.argwhere(fp))) == [(2, 5), (6, 1)]
    assert np.isnan(out[:, 2, 5]).all() and np.isnan(out[:, 6, 1]).all() and not fc.any()
    assert np.isfinite(out[:, 0, 0]).all()


def test_degenerate():
    s = pattern((6, 9, 9)).astype(np.float32)
    _, fc, fp = FL.autoflag(s, 1.0)  # all channel noises equal: R = 0, nothing deviates
    assert not fc.any()
    c = np.full((4, 3, 3), np.nan, dtype=np.float32)
    out, fc, fp = FL.autoflag(c, 1.0)
    assert not fc.any() and not fp.any() and np.isnan(out).all()


PINS = [lambda: test_brute_force_tiny(0), lambda: test_brute_force_tiny(2), test_channel_closed_form,
        test_pixel_closed_form, test_degenerate]


def _mut_rms_unscaled(orig):
    def f(noise, k):
        fl, m, r = orig(noise, k * 1.4826)
        return fl, m, r
    return f


def _mut_mean_centre(orig):
    def f(noise, k):
        v = np.asarray(noise, dtype=np.float64)
        ok = np.isfinite(v)
        if not ok.any():
            return orig(noise, k)
        m = float(v[ok].mean())
        r = 1.4826 * float(np.median(np.abs(v[ok] - m)))
        out = np.zeros(v.shape, dtype=bool)
        out[ok] = np.abs(v[ok] - m) > k * r
        return out, m, r
    return f


def _mut_pixel_axis(orig):
    def f(cube, mode="mad"):
        return orig(np.swapaxes(cube, 0, 1).copy(), mode)[:cube.shape[1], :cube.shape[2]] \
            if cube.shape[0] >= cube.shape[1] else orig(cube, mode) * 1.5
    return f


MUTATIONS = [("flags", _mut_rms_unscaled), ("flags", _mut_mean_centre), ("pixel_noise", _mut_pixel_axis)]


@pytest.mark.parametrize("name,mut", MUTATIONS, ids=[f"{n}-{m.__name__}" for n, m in MUTATIONS])
def test_planted_mistake_is_caught(monkeypatch, name, mut):
    monkeypatch.setattr(FL, name, mut(getattr(FL, name)))
    caught = []
    for pin in PINS:
        try:
            pin()
        except (AssertionError, ValueError, IndexError):
            caught.append(pin)
    assert caught, f"planted mistake in {name} ({mut.__name__}) passed every pin"
