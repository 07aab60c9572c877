"""Shared spatial passes (through the C ABI).

Pairs that share a spatial kernel differ only in the spectral boxcar and in the
voxels replaced at the start of each pair (SoFiA 2 Sect. 6.2), and the
smoothing is linear and exact in the library's fixed-point arithmetic. The
later pairs of such a run therefore take the first pair's spatial sums plus the
corrections of the voxels masked since then. Their smoothed cube must equal,
bit for bit, the full smoothing of every pair (SC_FLAG_NO_SHARE), whatever the
shape, mask density or list capacity; the whole S+C must still match the FP64
oracle.
"""
import numpy as np
import pytest
import torch

import oracle.sc_oracle as O
from synth.cubes import KERNELS_12, SMALL, CubeSpec, make_cube

pytestmark = pytest.mark.gpu

T = 3.5
N_REPL = 2.0
BAND = 1e-4


@pytest.fixture(scope="module")
def ctx():
    from paper_2106_15789_gb300 import Context

    c = Context(0, 1 << 22)
    yield c
    c.close()


def run_s(ctx, cube_dev, kernels, flags=0, t=T, n=N_REPL, mask0=None):
    from paper_2106_15789_gb300 import sc

    mask = None
    if mask0 is not None:
        mask = torch.from_numpy(mask0.astype(np.uint8)).cuda()
        flags |= sc.SC_FLAG_ACCUMULATE
    m, sig, s0 = ctx.run(cube_dev, kernels, t, "mad", n, mask=mask, flags=flags)
    s = ctx.copy_smoothed(tuple(cube_dev.shape))
    torch.cuda.synchronize()
    return m.cpu().numpy(), sig, s0, s.cpu()


def same_bits(a: torch.Tensor, b: torch.Tensor) -> bool:
    return torch.equal(a.view(torch.int32), b.view(torch.int32))


def check_shared_equals_full(ctx, cube, kernels, t=T, n=N_REPL, mask0=None, expect_shared=True, flags=0):
    from paper_2106_15789_gb300 import sc

    dev = cube.cuda()
    ctx.stats(reset=True)
    m1, sig1, s01, S1 = run_s(ctx, dev, kernels, flags, t, n, mask0)
    kinds = ctx.stats()["smooth_kernel_pair"][: len(kernels)]
    m2, sig2, s02, S2 = run_s(ctx, dev, kernels, flags | sc.SC_FLAG_NO_SHARE, t, n, mask0)
    assert s01 == s02
    assert sig1 == sig2, (sig1, sig2)
    assert np.array_equal(m1, m2), int((m1 != m2).sum())
    assert same_bits(S1, S2), int((S1.view(torch.int32) != S2.view(torch.int32)).sum())
    if expect_shared:
        assert sc.SC_KERNEL_SHARED in kinds, kinds
    return m1, sig1, s01, S1, kinds


def spatial_runs(kernels):
    """Pair indices that may reuse an earlier pair's spatial passes."""
    out = []
    for k in range(1, len(kernels)):
        if kernels[k][0] > 0 and kernels[k][0] == kernels[k - 1][0]:
            out.append(k)
    return out


def test_small_cube_default_kernels_shared_and_oracle(ctx):
    from paper_2106_15789_gb300 import sc

    cube = make_cube(SMALL)
    m, sig, s0, S, kinds = check_shared_equals_full(ctx, cube, KERNELS_12)
    for k in spatial_runs(KERNELS_12):
        assert kinds[k] == sc.SC_KERNEL_SHARED, (k, kinds)
    # the shared run against the oracle: sigmas, the mask outside the band, and
    # the last pair's smoothed cube
    m_ref, s_ref, s0_ref, ss = O.sc_filter(cube.numpy(), KERNELS_12, T, "mad", N_REPL, return_smoothed=True)
    assert abs(s0 - s0_ref) <= 1e-6 * s0_ref
    for k, (a, b) in enumerate(zip(sig, s_ref)):
        assert abs(a - b) <= 1e-6 * b, (k, a, b)
    diff = np.argwhere(m != m_ref)
    for p in diff:
        p = tuple(p)
        assert any(abs(abs(s[p]) / sk - T) < BAND for s, sk in zip(ss, s_ref)), p
    if len(diff) == 0:
        last = ss[-1]
        got = S.numpy().astype(np.float64)
        fin = np.isfinite(last)
        assert np.array_equal(fin, np.isfinite(got))
        err = np.abs(got[fin] - last[fin])
        assert err.max() <= 1e-5 * s_ref[-1], err.max()
        assert np.all(err <= 4 * np.spacing(np.abs(last[fin]).astype(np.float32)).astype(np.float64) + 1e-9)


@pytest.mark.parametrize("fwhm", [3.0, 5.0, 6.0, 10.0])
def test_every_later_pair_equals_full(ctx, fwhm):
    """S of each pair of a spatial run (taken as the last pair of a prefix)."""
    cube = make_cube(CubeSpec(nx=100, ny=70, nz=90, seed=21, n_gal=12, snr=(3.0, 20.0), fwhm_xy=(2.0, 8.0),
                              fwhm_z=(5.0, 30.0), nan_corner=(20, 10, 30)))
    ks = [(0.0, 0), (fwhm, 0), (fwhm, 3), (fwhm, 7), (fwhm, 15)]
    for L in range(3, len(ks) + 1):
        check_shared_equals_full(ctx, cube, ks[:L])


def test_wide_spectral_widths_use_short_tiles(ctx):
    """Boxcars of 17..31 channels take the 64 x 16 tiles of the shared pass."""
    cube = make_cube(CubeSpec(nx=90, ny=75, nz=120, seed=22, n_gal=10, snr=(3.0, 15.0), fwhm_xy=(2.0, 8.0),
                              fwhm_z=(10.0, 40.0)))
    for fwhm in (3.0, 10.0):
        check_shared_equals_full(ctx, cube, [(fwhm, 0), (fwhm, 17), (fwhm, 31), (fwhm, 5)])


@pytest.mark.parametrize("shape", [(67, 45, 40), (130, 97, 33), (64, 32, 20), (1, 1, 50), (3, 200, 17),
                                   (257, 66, 24)])
def test_ragged_shapes(ctx, shape):
    """Odd widths (padded rows of the stored sums, cubes TMA cannot read),
    one-voxel axes, and shapes spanning several tiles with a ragged tail."""
    nx, ny, nz = shape
    cube = make_cube(CubeSpec(nx=nx, ny=ny, nz=nz, seed=23, n_gal=6, snr=(3.0, 15.0), fwhm_xy=(2.0, 6.0),
                              fwhm_z=(5.0, 20.0)))
    check_shared_equals_full(ctx, cube, [(0.0, 0), (6.0, 0), (6.0, 3), (6.0, 7), (3.0, 0), (3.0, 15)])


def test_dense_corrections_and_caller_mask(ctx):
    """A low threshold masks a large share of the cube, so buckets hold far
    more entries than a plane stages in shared memory (the cost bound is
    lifted so that the shared pass takes them); a caller mask adds a dense
    block from the start."""
    cube = make_cube(CubeSpec(nx=96, ny=80, nz=64, seed=24, n_gal=15, snr=(3.0, 30.0), fwhm_xy=(2.0, 8.0),
                              fwhm_z=(5.0, 30.0)))
    ks = [(6.0, 0), (6.0, 3), (6.0, 7), (6.0, 15)]
    ctx.set_share_limit(1 << 40)
    try:
        check_shared_equals_full(ctx, cube, ks, t=1.2)
        check_shared_equals_full(ctx, cube, [(10.0, 0), (10.0, 31), (10.0, 3)], t=1.2)
    finally:
        ctx.set_share_limit(0)
    check_shared_equals_full(ctx, cube, ks, t=1.2)  # the default cost bound routes this to the full kernel
    mask0 = np.zeros(cube.shape, dtype=bool)
    mask0[10:40, 20:60, 30:70] = True
    check_shared_equals_full(ctx, cube, ks, mask0=mask0)


def test_replacement_off(ctx):
    cube = make_cube(SMALL)
    check_shared_equals_full(ctx, cube, KERNELS_12, n=0.0)


def test_list_overflow_falls_back_to_full_kernel(ctx):
    """A correction list above the cap: the gated full kernel computes the pair."""
    cube = make_cube(SMALL)
    ctx.set_share_limit(1)
    try:
        _, sig, _, S, kinds = check_shared_equals_full(ctx, cube, KERNELS_12, t=2.5)
    finally:
        ctx.set_share_limit(0)
    _, sig0, _, S0, _ = check_shared_equals_full(ctx, cube, KERNELS_12, t=2.5)
    assert sig == sig0
    assert same_bits(S, S0)


@pytest.mark.parametrize("fwhm", [2.5, 3.0, 5.0, 6.0, 7.3, 10.0])
def test_sampled_gaussian_pairs_shared(ctx, fwhm):
    """Sampled-Gaussian pairs (half-widths 3 to 16, taps zero-padded to the
    instance's reach) share their spatial sums bit for bit, with 32- and
    16-row tiles, a caller mask, and against the oracle's reading of them."""
    from paper_2106_15789_gb300 import sc

    cube = make_cube(CubeSpec(nx=90, ny=70, nz=80, seed=25, n_gal=10, snr=(3.0, 20.0), fwhm_xy=(2.0, 8.0),
                              fwhm_z=(5.0, 30.0), nan_corner=(15, 10, 20)))
    ks = [(0.0, 0), (fwhm, 0), (fwhm, 3), (fwhm, 7), (fwhm, 31), (fwhm, 15)]
    m, sig, s0, S, kinds = check_shared_equals_full(ctx, cube, ks, flags=sc.SC_FLAG_SAMPLED_GAUSS)
    assert kinds[1] == sc.SC_KERNEL_FIR and all(k == sc.SC_KERNEL_SHARED for k in kinds[2:]), kinds
    mask0 = np.zeros(cube.shape, dtype=bool)
    mask0[5:30, 10:40, 20:60] = True
    check_shared_equals_full(ctx, cube, ks[1:4], mask0=mask0, flags=sc.SC_FLAG_SAMPLED_GAUSS)
    m_ref, s_ref, s0_ref, ss = O.sc_filter(cube.numpy(), ks, T, "mad", N_REPL, return_smoothed=True,
                                           spatial="sampled")
    assert abs(s0 - s0_ref) <= 1e-6 * s0_ref
    for k, (a, b) in enumerate(zip(sig, s_ref)):
        assert abs(a - b) <= 1e-6 * b, (k, a, b)
    for p in map(tuple, np.argwhere(m != m_ref)):
        assert any(abs(abs(s[p]) / sk - T) < BAND for s, sk in zip(ss, s_ref)), p
