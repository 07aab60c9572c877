"""Local noise normalisation (sc_noise_scale) through the C ABI against the
FP64 oracle (oracle/noise_scale.py).

Tolerances from the arithmetic: a cell's noise is an exact order statistic
of MAD keys rounded to float, as in the S+C noise (within 2^-24 relative of
the oracle's double), or a double-precision sum, so sigma is checked to 1e-6
relative (the S+C sigma bound); a voxel is cube * fl32(1 / sigma), within
2^-23 relative of cube / sigma for the library's sigma, hence within
2^-23 + 2^-24 of the oracle's value. NaN positions must agree exactly.
"""
import numpy as np
import pytest
import torch

import oracle.noise_scale as NS
import oracle.sc_oracle as O
from gauss_common import close_to_any, gauss_refs
from synth.cubes import SMALL, CubeSpec, make_cube

pytestmark = pytest.mark.gpu

SIG_RTOL = 1e-6
OUT_RTOL = 2.0 ** -23 + 2.0 ** -24


@pytest.fixture(scope="module")
def ctx():
    from paper_2106_15789_gb300 import Context

    c = Context(0, 1 << 22)
    yield c
    c.close()


def check(ctx, cube_np, window, grid, mode, in_place=False):
    cube = torch.from_numpy(cube_np).cuda()
    out = cube if in_place else None
    got, sig = ctx.noise_scale(cube, window, grid, mode, out=out, want_sigma=True)
    ref, sig_ref = NS.noise_scale(cube_np, window, grid, mode)
    assert sig.shape == sig_ref.shape
    assert np.array_equal(np.isnan(sig), np.isnan(sig_ref))
    ok = np.isfinite(sig_ref)
    np.testing.assert_allclose(sig[ok], sig_ref[ok], rtol=SIG_RTOL, atol=0)
    g = got.cpu().numpy().astype(np.float64)
    assert np.array_equal(np.isnan(g), np.isnan(ref))
    f = ~np.isnan(ref)
    np.testing.assert_allclose(g[f], ref[f], rtol=OUT_RTOL, atol=0)
    return g, sig


@pytest.mark.parametrize("mode", ["mad", "std"])
def test_small_cube_window31(ctx, mode):
    """The paper's 31-voxel windows on the small cube (several tiles, NaN corner)."""
    check(ctx, make_cube(SMALL).numpy(), (31, 31, 31), (16, 16, 16), mode)


@pytest.mark.parametrize("mode", ["mad", "std"])
@pytest.mark.parametrize("shape,window,grid", [((33, 45, 67), (7, 5, 9), (4, 3, 5)),
                                               ((17, 9, 130), (31, 3, 1), (16, 1, 2)),
                                               ((40, 20, 20), (3, 41, 61), (7, 40, 25))])
def test_ragged(ctx, mode, shape, window, grid):
    rng = np.random.default_rng(sum(shape))
    c = (rng.standard_normal(shape) * (1.0 + np.arange(shape[0])[:, None, None] / 10.0)).astype(np.float32)
    c[rng.random(shape) < 0.05] = np.nan
    check(ctx, c, window, grid, mode)


@pytest.mark.parametrize("mode", ["mad", "std"])
def test_literal_running_window(ctx, mode):
    """grid (1, 1, 1): every voxel has its own window."""
    rng = np.random.default_rng(3)
    c = rng.standard_normal((10, 9, 11)).astype(np.float32)
    c[rng.random(c.shape) < 0.1] = np.nan
    check(ctx, c, (3, 5, 3), (1, 1, 1), mode)


def test_duplicates_and_in_place(ctx):
    """Many equal values (ties at the median and MAD ranks), computed in place."""
    rng = np.random.default_rng(9)
    c = (np.round(rng.standard_normal((24, 30, 36)) * 3.0) / 3.0).astype(np.float32)
    c[:5, :7, :9] = np.nan
    check(ctx, c, (9, 9, 9), (6, 6, 6), "mad", in_place=True)


def test_crowded_bins(ctx):
    """Values from {-1, 0, 1}: a third of every window shares one key, more
    than the candidate buffer holds, so the selections run over all keys;
    median 0 and MAD 1 in every window."""
    rng = np.random.default_rng(21)
    c = rng.integers(-1, 2, size=(40, 40, 40)).astype(np.float32)
    g, sig = check(ctx, c, (31, 31, 31), (16, 16, 16), "mad")
    np.testing.assert_allclose(sig, 1.4826, rtol=1e-15)


def test_degenerate(ctx):
    c = np.full((8, 9, 10), 2.5, dtype=np.float32)
    g, sig = check(ctx, c, (3, 3, 3), (4, 4, 4), "mad")
    assert np.isnan(g).all() and (sig == 0).all()
    c = make_cube(CubeSpec(nx=20, ny=20, nz=20, seed=4, n_gal=0)).numpy()
    c[:10, :, :10] = np.nan  # cells whose windows hold no finite voxel
    check(ctx, c, (5, 1, 5), (10, 20, 10), "mad")


def check_gauss(ctx, c, window, grid):
    """Gaussian-fit mode: every cell's noise against the oracle at the MAD
    noises that rounding allows (tests/gauss_common.py), window by window;
    the output is the cube times the float reciprocal of the library's own
    cell noise."""
    cube = torch.from_numpy(c).cuda()
    got, sig = ctx.noise_scale(cube, window, grid, "gauss", want_sigma=True)
    nz, ny, nx = c.shape
    (wx, wy, wz), (gx, gy, gz) = window, grid
    for k, (_, _, zc) in enumerate(NS.cells(nz, gz)):
        for j, (_, _, yc) in enumerate(NS.cells(ny, gy)):
            for i, (_, _, xc) in enumerate(NS.cells(nx, gx)):
                v = c[NS.window_slice(zc, wz, nz), NS.window_slice(yc, wy, ny), NS.window_slice(xc, wx, nx)]
                refs = gauss_refs(v.ravel())
                assert close_to_any(sig[k, j, i], refs), ((k, j, i), sig[k, j, i], refs)
    per = sig[np.arange(nz)[:, None, None] // gz, np.arange(ny)[None, :, None] // gy,
              np.arange(nx)[None, None, :] // gx]
    good = np.isfinite(per) & (per > 0) & np.isfinite(c)
    g = got.cpu().numpy().astype(np.float64)
    assert np.array_equal(np.isnan(g), ~good)
    np.testing.assert_allclose(g[good], c[good].astype(np.float64) / per[good], rtol=OUT_RTOL, atol=0)
    return sig


def test_gauss_small_cube_window31(ctx):
    check_gauss(ctx, make_cube(SMALL).numpy(), (31, 31, 31), (16, 16, 16))


@pytest.mark.parametrize("shape,window,grid", [((33, 45, 67), (7, 5, 9), (4, 3, 5)),
                                               ((40, 20, 20), (3, 41, 61), (7, 40, 25))])
def test_gauss_ragged(ctx, shape, window, grid):
    rng = np.random.default_rng(sum(shape) + 5)
    c = (rng.standard_normal(shape) * (1.0 + np.arange(shape[0])[:, None, None] / 10.0)).astype(np.float32)
    c[rng.random(shape) < 0.05] = np.nan
    check_gauss(ctx, c, window, grid)


def test_gauss_emission_and_offset(ctx):
    """Bright positive emission in one corner of the windows, and a cell far
    from 0 (the fit falls back to the MAD noise there)."""
    rng = np.random.default_rng(17)
    c = rng.standard_normal((24, 32, 32)).astype(np.float32)
    src = rng.random(c.shape) < 0.04
    c[src] = np.abs(c[src]) * 5.0 + 5.0
    c[:8, :16, :16] += 400.0
    check_gauss(ctx, c, (15, 15, 9), (16, 16, 8))


def test_arguments(ctx):
    from paper_2106_15789_gb300 import sc

    c = torch.zeros((8, 8, 8), device="cuda")
    for window, grid, mode, code in (((4, 3, 3), (2, 2, 2), "mad", sc.SC_ERR_ARG),
                                     ((3, 3, 3), (0, 2, 2), "mad", sc.SC_ERR_ARG),
                                     ((3, 3, 3), (2, 2, 2), 7, sc.SC_ERR_ARG)):
        with pytest.raises(sc.ScError) as e:
            ctx.noise_scale(c, window, grid, mode)
        assert e.value.code == code
    big = torch.zeros((64, 64, 64), device="cuda")
    with pytest.raises(sc.ScError) as e:
        ctx.noise_scale(big, (63, 63, 63), (32, 32, 32))
    assert e.value.code == sc.SC_ERR_UNSUPPORTED


def test_sampled_cells_medium(ctx):
    """A 256^3 cube with a channel ripple: 24 sampled cells' noise and voxels
    against the oracle, computed cell by cell."""
    from paper_2106_15789_gb300 import Context

    spec = CubeSpec(nx=256, ny=256, nz=256, seed=12, n_gal=40, ripple=0.3, nan_border=4)
    cube = make_cube(spec, device="cuda")
    big = Context(0, cube.numel())
    try:
        out, sig = big.noise_scale(cube, (31, 31, 31), (16, 16, 16), "mad", want_sigma=True)
    finally:
        big.close()
    c = cube.cpu().numpy()
    o = out.cpu().numpy()
    rng = np.random.default_rng(1)
    cz, cy, cx = NS.cells(256, 16), NS.cells(256, 16), NS.cells(256, 16)
    for _ in range(24):
        k, j, i = (int(v) for v in rng.integers(0, 16, 3))
        w = c[NS.window_slice(cz[k][2], 31, 256), NS.window_slice(cy[j][2], 31, 256), NS.window_slice(cx[i][2], 31, 256)]
        w = w[np.isfinite(w)].astype(np.float64)
        s_ref = O.noise(w, "mad")
        assert abs(sig[k, j, i] - s_ref) <= SIG_RTOL * s_ref
        blk = c[cz[k][0]:cz[k][1], cy[j][0]:cy[j][1], cx[i][0]:cx[i][1]].astype(np.float64)
        got = o[cz[k][0]:cz[k][1], cy[j][0]:cy[j][1], cx[i][0]:cx[i][1]].astype(np.float64)
        f = np.isfinite(blk)
        assert np.array_equal(np.isnan(got), ~f)
        np.testing.assert_allclose(got[f], blk[f] / s_ref, rtol=OUT_RTOL + SIG_RTOL, atol=0)
