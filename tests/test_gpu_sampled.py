"""The sampled-Gaussian spatial kernel (SC_FLAG_SAMPLED_GAUSS) through the C
ABI against the oracle's reading of it (the Gaussian of a given FWHM sampled
within +-4 sigma with integer taps, over their sum).

Smoothing: element by element within the parity tolerance (1e-5 sigma) and
within a few float ulps plus the fixed-point quantum, with and without a
replacement mask, on the small cube and on ragged shapes. S+C: sigmas within
1e-6 relative, mask bit-exact outside the threshold band; the first pair of a
spatial kernel runs the warp-specialised FIR kernel, the later ones share its
spatial sums (half-widths up to 16). A kernel too wide for the smoothing
kernels is refused.
"""
import numpy as np
import pytest
import torch

import oracle.sc_oracle as O
from synth.cubes import KERNELS_12, SMALL, CubeSpec, make_cube

pytestmark = pytest.mark.gpu

T = 3.5
N_REPL = 2.0
SIG_RTOL = 1e-6
S_TOL = 1e-5
BAND = 1e-4


@pytest.fixture(scope="module")
def ctx():
    from paper_2106_15789_gb300 import Context

    c = Context(0, 1 << 22)
    yield c
    c.close()


def check_smooth(ctx, cube, kernel, mask=None, value=0.0):
    from paper_2106_15789_gb300 import sc

    c_np = cube.numpy().astype(np.float64)
    m_t = torch.from_numpy(mask.astype(np.uint8)).cuda() if mask is not None else None
    got = ctx.smooth(cube.cuda(), kernel, mask=m_t, replacement_value=value, flags=sc.SC_FLAG_SAMPLED_GAUSS)
    got = got.cpu().numpy().astype(np.float64)
    ref = O.smoothed(c_np, mask if mask is not None else np.zeros(c_np.shape, bool), kernel[0], kernel[1], value,
                     "sampled")
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    fin = np.isfinite(ref)
    if not fin.any():
        return
    sig = O.noise(ref[fin], "mad")
    err = np.abs(got[fin] - ref[fin])
    if sig > 0:
        assert err.max() <= S_TOL * sig, (kernel, err.max(), sig)
    # exact fixed-point arithmetic: a few float ulps plus the quantum 2^-f of
    # the inputs, f = 62 - e - bitlen(T^2 max(wz, 31) - 1) with max|X| < 2^e and
    # T the taps' sum (the library's scale rule); T^2 reaches 2^29 here, so f
    # can sit below 30
    t_sum = int(O.gauss_taps(kernel[0]).sum()) if kernel[0] > 0 else 1
    mx = max(float(np.nanmax(np.abs(c_np))), value)
    e = int(np.frexp(np.float32(mx))[1])
    f = 62 - e - int(t_sum * t_sum * max(kernel[1], 31) - 1).bit_length()
    bound = 4.0 * np.spacing(np.abs(ref[fin]).astype(np.float32)).astype(np.float64) + 2.0 ** -f
    worst = int(np.argmax(err / bound))
    assert err[worst] <= bound[worst], (kernel, got[fin][worst], ref[fin][worst], err[worst])


@pytest.mark.parametrize("kernel", [(2.5, 1), (3.0, 0), (3.0, 3), (5.0, 3), (6.0, 7), (10.0, 15), (6.0, 31),
                                    (15.0, 3), (23.0, 1), (0.3, 3)])
def test_smooth_matches_oracle(ctx, kernel):
    cube = make_cube(SMALL)
    c_np = cube.numpy()
    rng = np.random.default_rng(15)
    mask = (rng.random(c_np.shape) < 0.03) | (np.abs(np.nan_to_num(c_np)) > 3.0)
    value = float(np.float32(2.1))
    check_smooth(ctx, cube, kernel)
    check_smooth(ctx, cube, kernel, mask, value)


@pytest.mark.parametrize("shape", [(67, 45, 40), (1, 1, 50), (3, 200, 17), (130, 97, 33), (5, 9, 7)])
def test_ragged_shapes(ctx, shape):
    nx, ny, nz = shape
    cube = make_cube(CubeSpec(nx=nx, ny=ny, nz=nz, seed=61, n_gal=4, snr=(3.0, 12.0), fwhm_xy=(2.0, 6.0),
                              fwhm_z=(5.0, 20.0)))
    for kernel in ((3.0, 3), (6.0, 1), (10.0, 7)):
        check_smooth(ctx, cube, kernel)


def check_run(ctx, cube, kernels, t=T, n=N_REPL, mode="mad"):
    from paper_2106_15789_gb300 import sc

    ctx.stats(reset=True)
    m, sig, s0 = ctx.run(cube.cuda(), kernels, t, mode, n, flags=sc.SC_FLAG_SAMPLED_GAUSS)
    kinds = ctx.stats()["smooth_kernel_pair"][: len(kernels)]
    m_ref, s_ref, s0_ref, ss = O.sc_filter(cube.numpy(), kernels, t, mode, n, return_smoothed=True,
                                           spatial="sampled")
    assert abs(s0 - s0_ref) <= SIG_RTOL * s0_ref, (s0, s0_ref)
    for k, (a, b) in enumerate(zip(sig, s_ref)):
        assert abs(a - b) <= SIG_RTOL * b, (k, kernels[k], a, b)
    diff = np.argwhere(m.cpu().numpy() != m_ref)
    for p in map(tuple, diff):
        assert any(sk > 0 and abs(abs(s[p]) / sk - t) < BAND for s, sk in zip(ss, s_ref)), p
    for k, ((fs, wz), kind) in enumerate(zip(kernels, kinds)):
        if fs > 1.0 and fs <= 10.0 and wz <= 31:
            shared = k > 0 and kernels[k - 1][0] == fs
            assert kind == (sc.SC_KERNEL_SHARED if shared else sc.SC_KERNEL_FIR), (fs, wz, kind)
        elif fs > 1.0:
            assert kind == sc.SC_KERNEL_GENERIC, (fs, wz, kind)
    return sig


def test_sc_small_cube_default_kernels(ctx):
    sig = check_run(ctx, make_cube(SMALL), KERNELS_12)
    # the cascade gives other sigmas for the smoothed pairs
    _, sig_c, _ = ctx.run(make_cube(SMALL).cuda(), KERNELS_12, T, "mad", N_REPL)
    assert sig[0] == sig_c[0] and sig[1] == sig_c[1]  # no spatial smoothing: same pairs
    assert all(a != b for a, b in zip(sig[4:], sig_c[4:]))


def test_sc_paper_kernels_and_options(ctx):
    cube = make_cube(SMALL)
    check_run(ctx, cube, [(0.0, 0), (5.0, 3), (10.0, 15), (10.0, 31), (6.0, 7)])
    check_run(ctx, cube, KERNELS_12, n=0.0)
    check_run(ctx, cube, KERNELS_12, t=2.5, n=1.5, mode="std")


def test_too_wide_is_refused(ctx):
    from paper_2106_15789_gb300 import sc

    cube = make_cube(SMALL).cuda()
    with pytest.raises(sc.ScError) as e:
        ctx.run(cube, [(0.0, 0), (30.0, 3)], T, "mad", N_REPL, flags=sc.SC_FLAG_SAMPLED_GAUSS)
    assert e.value.code == sc.SC_ERR_UNSUPPORTED
