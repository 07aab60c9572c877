"""Auto-flagger (sc_autoflag) through the C ABI against the oracle
(oracle/flagger.py).

The noises are float32 on both sides; the GPU's MAD keys round |x - m|
correctly (odd counts) or faithfully (even counts) in single precision, so a
noise may differ from the oracle's by one float ulp: noises are checked to
2^-22 relative. Flags must agree except where |noise - M| lies within 1e-5
relative of k R (where that ulp can decide); the blanked cube must follow
the library's own flags exactly.
"""
import numpy as np
import pytest
import torch

import oracle.flagger as FL
from gauss_common import close_to_any, gauss_refs
from synth.cubes import SMALL, CubeSpec, make_cube

pytestmark = pytest.mark.gpu

NOISE_RTOL = 2.0 ** -22
BAND = 1e-5


@pytest.fixture(scope="module")
def ctx():
    from paper_2106_15789_gb300 import Context

    c = Context(0, 1 << 20)
    yield c
    c.close()


def flags_agree(got, ref, noise, k):
    m_f, m, r = FL.flags(noise, k)
    diff = np.flatnonzero(got.ravel() != ref.ravel())
    v = np.asarray(noise, dtype=np.float64).ravel()
    for i in diff:
        assert abs(abs(v[i] - m) - k * r) <= BAND * max(k * r, 1e-30), (i, v[i], m, r)


def check(ctx, c, k, channels=True, pixels=True, mode="mad", in_place=False):
    cube = torch.from_numpy(c).cuda()
    out, fc, fp, cn, pn = ctx.autoflag(cube, k, channels, pixels, mode, out=cube if in_place else None)
    _, rc, rp = FL.autoflag(c, k, channels, pixels, mode)
    if channels:
        ref_n = FL.channel_noise(c, mode)
        assert np.array_equal(np.isnan(cn), np.isnan(ref_n))
        ok = np.isfinite(ref_n)
        np.testing.assert_allclose(cn[ok], ref_n[ok], rtol=NOISE_RTOL, atol=0)
        flags_agree(fc, rc, ref_n, k)
    if pixels:
        ref_p = FL.pixel_noise(c, mode)
        assert np.array_equal(np.isnan(pn), np.isnan(ref_p))
        ok = np.isfinite(ref_p)
        np.testing.assert_allclose(pn[ok], ref_p[ok], rtol=NOISE_RTOL, atol=0)
        flags_agree(fp, rp, ref_p, k)
    # the blanking follows the library's flags exactly
    o = out.cpu().numpy()
    exp = c.copy()
    exp[fc] = np.nan
    exp[:, fp] = np.nan
    assert np.array_equal(np.isnan(o), np.isnan(exp))
    f = ~np.isnan(exp)
    assert np.array_equal(o[f], exp[f])
    return fc, fp


def rfi_cube(shape, seed):
    """Noise with channel-to-channel and pixel-to-pixel RMS variations, three
    loud channels (RFI) and a few noisy pixels (residual continuum)."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    c = rng.standard_normal(shape) * (1.0 + 0.03 * rng.standard_normal((nz, 1, 1)))
    c *= 1.0 + 0.03 * rng.standard_normal((1, ny, nx))
    for z in rng.choice(nz, 3, replace=False):
        c[z] *= 6.0
    for _ in range(4):
        c[:, rng.integers(ny), rng.integers(nx)] *= 5.0
    c = c.astype(np.float32)
    c[rng.random(shape) < 0.02] = np.nan
    return c


@pytest.mark.parametrize("mode", ["mad", "std"])
@pytest.mark.parametrize("shape", [(64, 40, 48), (130, 37, 33), (300, 20, 70), (1030, 9, 11)])
def test_rfi_cubes(ctx, mode, shape):
    fc, fp = check(ctx, rfi_cube(shape, sum(shape)), 4.0, mode=mode)
    if mode == "mad":
        assert fc.sum() >= 3 and fp.sum() >= 1


@pytest.mark.parametrize("shape", [(64, 40, 48), (300, 20, 21), (1030, 5, 6)])
def test_gauss_mode(ctx, shape):
    """Gaussian-fit channel and pixel noises against the oracle at the MAD
    noises that rounding allows (tests/gauss_common.py); flags equal to the
    oracle's except within 1e-4 of k R (a noise may move by ~1e-6 with the MAD
    noise's rounding); the blanking follows the library's flags exactly."""
    c = rfi_cube(shape, sum(shape) + 1)
    cube = torch.from_numpy(c).cuda()
    out, fc, fp, cn, pn = ctx.autoflag(cube, 4.0, True, True, "gauss")
    _, rc, rp = FL.autoflag(c, 4.0, True, True, "gauss")
    nz, ny, nx = shape
    for z in range(nz):
        refs = gauss_refs(c[z].ravel())
        assert close_to_any(float(cn[z]), refs, 2.0 ** -22), (z, cn[z], refs)
    for y in range(ny):
        for x in range(nx):
            refs = gauss_refs(c[:, y, x])
            assert close_to_any(float(pn[y, x]), refs, 2.0 ** -22), ((y, x), pn[y, x], refs)
    for got, ref, noise in ((fc, rc, FL.channel_noise(c, "gauss")), (fp, rp, FL.pixel_noise(c, "gauss"))):
        _, m, r = FL.flags(noise, 4.0)
        v = np.asarray(noise, dtype=np.float64).ravel()
        for i in np.flatnonzero(got.ravel() != ref.ravel()):
            assert abs(abs(v[i] - m) - 4.0 * r) <= 1e-4 * 4.0 * r, (i, v[i], m, r)
    assert fc.sum() >= 3
    o = out.cpu().numpy()
    exp = c.copy()
    exp[fc] = np.nan
    exp[:, fp] = np.nan
    assert np.array_equal(np.isnan(o), np.isnan(exp))


def test_small_cube_each_kind_and_in_place(ctx):
    c = make_cube(SMALL).numpy()
    check(ctx, c, 3.0, channels=True, pixels=False)
    check(ctx, c, 3.0, channels=False, pixels=True)
    check(ctx, c, 3.0, in_place=True)


def test_degenerate(ctx):
    c = np.full((6, 5, 7), 1.5, dtype=np.float32)  # every noise 0: R = 0, nothing deviates
    fc, fp = check(ctx, c, 2.0)
    assert not fc.any() and not fp.any()
    c = rfi_cube((20, 8, 9), 3)
    c[5] = np.nan        # a channel without finite voxels
    c[:, 2, 3] = np.nan  # a pixel without finite voxels
    check(ctx, c, 3.0)


def test_arguments(ctx):
    from paper_2106_15789_gb300 import sc

    c = torch.zeros((8, 8, 8), device="cuda")
    with pytest.raises(sc.ScError) as e:
        ctx.autoflag(c, -1.0)
    assert e.value.code == sc.SC_ERR_ARG
    with pytest.raises(sc.ScError) as e:
        ctx.autoflag(c, 3.0, noise_mode=7)
    assert e.value.code == sc.SC_ERR_ARG
    big = torch.zeros((1600, 2, 2), device="cuda")
    with pytest.raises(sc.ScError) as e:
        ctx.autoflag(big, 3.0, channels=False, pixels=True)
    assert e.value.code == sc.SC_ERR_UNSUPPORTED
