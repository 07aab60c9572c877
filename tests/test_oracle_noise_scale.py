"""Pins for the local noise normalisation oracle (oracle/noise_scale.py),
checked against things other than the oracle itself: brute force in pure
Python (per-voxel loops, the statistics module's median and stdev) on tiny
cubes, hand-derived closed forms, the S+C noise of the whole cube, degenerate
cases and a statistical check on a cube with two noise levels. The last test
plants plausible mistakes in the oracle and checks that each trips a pin.
"""
import math
import statistics

import numpy as np
import pytest

import oracle.noise_scale as NS
import oracle.sc_oracle as O


def bf_noise_scale(c, window, grid, mode):
    """Per-voxel brute force of the readings: the voxel's cell, the cell's
    centre, the clipped window around it, the statistic from the statistics
    module, then the division."""
    nz, ny, nx = c.shape
    out = np.full(c.shape, np.nan)
    rads = [(w - 1) // 2 for w in window]  # x, y, z

    def centre(i, g, n):
        start = (i // g) * g
        extent = min(g, n - start)
        return start + (extent - 1) // 2

    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                cx, cy, cz = centre(x, grid[0], nx), centre(y, grid[1], ny), centre(z, grid[2], nz)
                vals = []
                for zz in range(max(0, cz - rads[2]), min(nz, cz + rads[2] + 1)):
                    for yy in range(max(0, cy - rads[1]), min(ny, cy + rads[1] + 1)):
                        for xx in range(max(0, cx - rads[0]), min(nx, cx + rads[0] + 1)):
                            v = float(c[zz, yy, xx])
                            if math.isfinite(v):
                                vals.append(v)
                if not vals or not math.isfinite(float(c[z, y, x])):
                    continue
                if mode == "mad":
                    m = statistics.median(vals)
                    s = 1.4826 * statistics.median([abs(v - m) for v in vals])
                else:
                    s = statistics.stdev(vals) if len(vals) > 1 else 0.0
                if s > 0:
                    out[z, y, x] = float(c[z, y, x]) / s
    return out


def tiny_cube(shape, seed, nan_frac=0.1):
    rng = np.random.default_rng(seed)
    c = rng.standard_normal(shape).astype(np.float32)
    c[rng.random(shape) < nan_frac] = np.nan
    return c


@pytest.mark.parametrize("window,grid", [((3, 3, 3), (2, 2, 2)), ((3, 3, 3), (1, 1, 1)), ((5, 3, 1), (2, 3, 2)),
                                         ((1, 5, 3), (4, 4, 4)), ((7, 7, 7), (3, 2, 5))])
@pytest.mark.parametrize("mode", ["mad", "std"])
def test_brute_force_tiny(window, grid, mode):
    c = tiny_cube((5, 6, 7), seed=11 + sum(window) + sum(grid))
    got, _ = NS.noise_scale(c, window, grid, mode)
    ref = bf_noise_scale(c, window, grid, mode)
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    ok = ~np.isnan(ref)
    np.testing.assert_allclose(got[ok], ref[ok], rtol=1e-12, atol=0)


def pattern_cube(a_left, a_right, split_x, shape=(9, 9, 12)):
    """a * s with s = ((x + y + z) mod 3) - 1: every full 3 x 3 x 3 block holds
    nine each of -a, 0, +a."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    s = ((x + y + z) % 3 - 1).astype(np.float64)
    a = np.where(x < split_x, a_left, a_right)
    return (a * s).astype(np.float32), s


def test_closed_form_pattern_mad():
    """3 x 3 x 3 windows on 3 x 3 x 3 cells never straddle x = 6. In every
    window: median 0; |x - 0| is 0 nine times and a eighteen times, so MAD = a
    and sigma = 1.4826 a; the normalised value is s / 1.4826 whatever a is."""
    c, s = pattern_cube(2.0, 5.0, 6)
    got, sig = NS.noise_scale(c, (3, 3, 3), (3, 3, 3), "mad")
    np.testing.assert_allclose(got, s / 1.4826, rtol=1e-15, atol=1e-15)
    np.testing.assert_allclose(sig[:, :, :2], 1.4826 * 2.0, rtol=1e-15)
    np.testing.assert_allclose(sig[:, :, 2:], 1.4826 * 5.0, rtol=1e-15)


def test_closed_form_pattern_std():
    """Same windows: mean 0 and sum of squares 18 a^2 over 27 values, so
    sigma = a * sqrt(18 / 26)."""
    c, s = pattern_cube(2.0, 5.0, 6)
    got, _ = NS.noise_scale(c, (3, 3, 3), (3, 3, 3), "std")
    np.testing.assert_allclose(got, s / math.sqrt(18.0 / 26.0), rtol=1e-14, atol=1e-15)


def test_whole_cube_window_is_the_cube_noise():
    """A window covering the cube from one cell: every voxel is divided by the
    S+C noise of the whole cube."""
    c = tiny_cube((6, 5, 9), seed=3)
    got, sig = NS.noise_scale(c, (17, 11, 13), (9, 5, 6), "mad")
    s0 = O.noise(c[np.isfinite(c)].astype(np.float64), "mad")
    assert sig.shape == (1, 1, 1) and sig[0, 0, 0] == s0
    ok = np.isfinite(c)
    np.testing.assert_allclose(got[ok], c[ok].astype(np.float64) / s0, rtol=1e-15)
    assert np.isnan(got[~ok]).all()


def test_degenerate_windows_blank():
    c = np.full((4, 5, 6), 3.0, dtype=np.float32)  # noise 0 everywhere
    got, sig = NS.noise_scale(c, (3, 3, 3), (2, 2, 2), "mad")
    assert np.isnan(got).all() and (sig == 0).all()
    c = tiny_cube((4, 5, 6), seed=4, nan_frac=0.0)
    got, _ = NS.noise_scale(c, (1, 1, 1), (1, 1, 1), "mad")  # one-voxel windows: MAD 0
    assert np.isnan(got).all()
    c[:2, :, :3] = np.nan  # one cell of (3, 5, 2) without finite voxels, windows confined to it
    got, sig = NS.noise_scale(c, (3, 1, 1), (3, 5, 2), "mad")
    assert np.isnan(sig[0, 0, 0]) and np.isnan(got[:2, :, :3]).all()
    assert np.isfinite(got[2:, :, :]).all()


def test_cell_layout():
    assert NS.cells(10, 4) == [(0, 4, 1), (4, 8, 5), (8, 10, 8)]
    assert NS.cells(5, 1) == [(i, i + 1, i) for i in range(5)]
    assert NS.cells(7, 7) == [(0, 7, 3)]
    assert NS.window_slice(1, 5, 10) == slice(0, 4)
    assert NS.window_slice(8, 5, 10) == slice(6, 10)
    with pytest.raises(ValueError):
        NS.window_slice(3, 4, 10)


def test_two_noise_levels_are_equalised():
    """White noise with sigma 1 below z = 32 and 4 above: away from the step,
    the normalised cube has unit noise on both sides (statistical)."""
    rng = np.random.default_rng(7)
    c = rng.standard_normal((64, 40, 40)).astype(np.float32)
    c[32:] *= 4.0
    got, _ = NS.noise_scale(c, (15, 15, 15), (8, 8, 8), "mad")
    lo, hi = got[:20].ravel(), got[44:].ravel()
    assert abs(np.std(lo) - 1.0) < 0.05 and abs(np.std(hi) - 1.0) < 0.05
    raw = c[44:].ravel()
    assert abs(np.std(raw) - 4.0) < 0.2  # the input really had two levels


# ----------------------------------------------------------------------------
# Planted mistakes.

PINS = [
    lambda: test_brute_force_tiny((3, 3, 3), (2, 2, 2), "mad"),
    lambda: test_brute_force_tiny((5, 3, 1), (2, 3, 2), "std"),
    test_closed_form_pattern_mad, test_closed_form_pattern_std, test_whole_cube_window_is_the_cube_noise,
    test_degenerate_windows_blank, test_cell_layout, test_two_noise_levels_are_equalised,
]


def _mut_centre_at_start(orig):
    def f(n, g):
        return [(a, b, a) for a, b, _ in orig(n, g)]
    return f


def _mut_window_one_wider_below(orig):
    def f(centre, w, n):
        s = orig(centre, w, n)
        r = (w - 1) // 2
        return slice(max(centre - r - (1 if s.start > 0 else 0), 0), s.stop)
    return f


def _mut_mad_not_scaled(orig):
    def f(cube, window, grid, mode="mad"):
        return orig(cube, window, grid, mode) / (1.4826 if mode == "mad" else 1.0)
    return f


def _mut_grid_axes_swapped(orig):
    def f(cube, window, grid, mode="mad"):
        return orig(cube, window, (grid[2], grid[1], grid[0]), mode)
    return f


MUTATIONS = [("cells", _mut_centre_at_start), ("window_slice", _mut_window_one_wider_below),
             ("noise_grid", _mut_mad_not_scaled), ("noise_grid", _mut_grid_axes_swapped)]


@pytest.mark.parametrize("name,mut", MUTATIONS, ids=[f"{n}-{m.__name__}" for n, m in MUTATIONS])
def test_planted_mistake_is_caught(monkeypatch, name, mut):
    monkeypatch.setattr(NS, name, mut(getattr(NS, name)))
    caught = []
    for pin in PINS:
        try:
            pin()
        except (AssertionError, ValueError, IndexError):
            caught.append(pin)
    assert caught, f"planted mistake in {name} ({mut.__name__}) passed every pin"
