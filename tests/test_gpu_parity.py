"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (from the method's target): smoothed voxels within 1e-5 * sigma,
sigma within 1e-6 relative, mask bit-exact except voxels whose smoothed value
lies within 1e-4 of the threshold (|S/sigma - t| < 1e-4) at some pair; those
are counted. The smoothing is exact fixed-point arithmetic, so a tighter bound
(a few float ulps of |S|) is checked as well.
"""
import numpy as np
import pytest
import torch

import oracle.sc_oracle as O
from synth.cubes import KERNELS_12, KERNELS_20, SMALL, CubeSpec, make_cube

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


def small_cube():
    return make_cube(SMALL)


def band_disagreements(mask_gpu, m_ref, ss, sigmas, t):
    diff = np.argwhere(mask_gpu != m_ref)
    bad = []
    for p in diff:
        p = tuple(p)
        if not any(sk > 0 and abs(abs(s[p]) / sk - t) < BAND for s, sk in zip(ss, sigmas)):
            bad.append(p)
    return len(diff), bad


def check_run(ctx, cube, kernels, t=T, mode="mad", n=N_REPL, flags=0, mask0=None):
    c_np = cube.numpy()
    dev = cube.cuda()
    mask = None
    if mask0 is not None:
        mask = torch.from_numpy(mask0.astype(np.uint8)).cuda()
    m, sig, s0 = ctx.run(dev, kernels, t, mode, n, mask=mask, flags=flags)
    m_ref, s_ref, s0_ref, ss = O.sc_filter(c_np, kernels, t, mode, n, mask=mask0, return_smoothed=True)
    assert abs(s0 - s0_ref) <= SIG_RTOL * s0_ref, (s0, s0_ref)
    for k, (a, b) in enumerate(zip(sig, s_ref)):
        assert abs(a - b) <= SIG_RTOL * b, (k, kernels[k], a, b)
    ndiff, bad = band_disagreements(m.cpu().numpy(), m_ref, ss, s_ref, t)
    assert not bad, f"{len(bad)} mask disagreements outside the threshold band, e.g. {bad[:5]}"
    return m, sig, s0, ndiff


# ---------------------------------------------------------------------------
def noise_cases():
    rng = np.random.default_rng(123)
    cases = {f"normal{n}": rng.standard_normal(n) for n in (1, 2, 3, 10, 101, 1000, 100_001, 2_000_000)}
    x = rng.standard_normal(300_000)
    x[rng.random(x.size) < 0.1] = np.nan
    x[:7] = np.inf
    x[7:9] = -np.inf
    cases["nan_inf"] = x
    cases["rounded"] = np.round(rng.standard_normal(200_000), 1)
    cases["integers"] = rng.integers(-3, 4, 100_000).astype(float)
    cases["offset"] = 1000.0 + rng.standard_normal(100_000)
    cases["tiny"] = 1e-20 * rng.standard_normal(50_000)
    cases["huge"] = 1e20 * rng.standard_normal(50_000)
    cases["cauchy"] = rng.standard_cauchy(300_000)
    cases["skewed"] = rng.exponential(1.0, 100_000)
    cases["constant"] = np.full(1000, 2.5)
    # subnormal float32 values (|x| < 2^-126), some exactly 0
    sub = rng.standard_normal(100_001) * 1e-40
    sub[::97] = 0.0
    cases["subnormal"] = sub
    # -0 and +0 as the two middle order statistics of an even count
    pm = np.concatenate([np.full(5000, -0.0), np.full(5000, 0.0), -1.0 - rng.random(4000), 1.0 + rng.random(4000)])
    cases["pm_zero_middle"] = rng.permutation(pm)
    # keys that share their top 24 bits or more: 1 + k 2^-23 with k < 256 (one
    # exponent, the top 15 mantissa bits equal), many duplicates
    cases["shared_top_bits"] = 1.0 + rng.integers(0, 256, 200_001) * 2.0 ** -23
    cases["shared_top_bits_neg"] = -(1.0 + rng.integers(0, 64, 50_000) * 2.0 ** -23)
    return cases


def sigma_close(got: float, ref: float) -> bool:
    """Within SIG_RTOL of the oracle, or within one float32 ulp of it where
    the library's float32 sigma is subnormal (its resolution there is 2^-149)."""
    if ref == 0.0:
        return got == 0.0
    return abs(got - ref) <= max(SIG_RTOL * ref, 2.0 ** -149)


@pytest.mark.parametrize("name", list(noise_cases().keys()))
def test_noise_matches_oracle(ctx, name):
    from paper_2106_15789_gb300 import sc

    v = noise_cases()[name].astype(np.float32)
    d = torch.from_numpy(v).cuda()
    fin = v[np.isfinite(v)].astype(np.float64)
    for mode in ("mad", "std"):
        ref = O.noise(fin, mode)
        got = ctx.noise(d, mode)
        assert sigma_close(got, ref), (mode, got, ref)
    # full passes instead of candidate lists: identical float result
    assert ctx.noise(d, "mad", flags=sc.SC_FLAG_NO_FAST_SELECT) == ctx.noise(d, "mad")


def test_noise_all_nan(ctx):
    from paper_2106_15789_gb300 import sc

    d = torch.full((1000,), float("nan"), device="cuda")
    with pytest.raises(sc.ScError) as e:
        ctx.noise(d)
    assert e.value.code == sc.SC_ERR_ALLNAN


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kernel", KERNELS_20 + [(5.0, 3), (2.2, 1), (14.0, 9)])
def test_smooth_matches_oracle(ctx, kernel):
    cube = small_cube()
    c_np = cube.numpy().astype(np.float64)
    rng = np.random.default_rng(5)
    mask = (rng.random(c_np.shape) < 0.03) | (np.abs(np.nan_to_num(c_np)) > 3.0)
    mask_t = torch.from_numpy(mask.astype(np.uint8)).cuda()
    value = float(np.float32(2.0 * 1.05))  # the library takes the value as float32
    for m_np, m_t in ((None, None), (mask, mask_t)):
        got = ctx.smooth(cube.cuda(), kernel, mask=m_t, replacement_value=value if m_t is not None else 0.0)
        got = got.cpu().numpy().astype(np.float64)
        ref = O.smoothed(c_np, m_np if m_np is not None else np.zeros(c_np.shape, bool), kernel[0], kernel[1],
                         value if m_np is not None else 0.0)
        assert np.array_equal(np.isnan(got), np.isnan(ref))
        fin = np.isfinite(ref)
        sig = O.noise(ref[fin], "mad")
        err = np.abs(got[fin] - ref[fin])
        assert err.max() <= S_TOL * sig, (kernel, err.max(), sig)
        # exact arithmetic: within a few float ulps of the true value, plus the
        # fixed-point quantum (2^-f with f >= 30 here)
        bound = 4.0 * np.spacing(np.abs(ref[fin]).astype(np.float32)).astype(np.float64) + 1e-9
        worst = int(np.argmax(err / bound))
        assert err[worst] <= bound[worst], (kernel, m_np is not None, got[fin][worst], ref[fin][worst], err[worst])


# ---------------------------------------------------------------------------
def test_small_cube_default(ctx):
    m, sig, s0, ndiff = check_run(ctx, small_cube(), KERNELS_12)
    assert m.sum().item() > 0
    print(f"small cube: sigma0={s0:.7f} band disagreements={ndiff}")


def test_small_cube_paper_kernels_and_wide(ctx):
    check_run(ctx, small_cube(), [(0.0, 0), (5.0, 3), (10.0, 15), (10.0, 31), (6.0, 7)])


def test_replacement_off(ctx):
    check_run(ctx, small_cube(), KERNELS_12, n=0.0)


def test_std_mode(ctx):
    check_run(ctx, small_cube(), KERNELS_12, mode="std")


def test_low_threshold(ctx):
    check_run(ctx, small_cube(), KERNELS_12, t=2.5, n=1.5)


def test_accumulate(ctx):
    from paper_2106_15789_gb300 import sc

    cube = small_cube()
    rng = np.random.default_rng(9)
    mask0 = rng.random(tuple(cube.shape)) < 0.01
    check_run(ctx, cube, KERNELS_12[3:], flags=sc.SC_FLAG_ACCUMULATE, mask0=mask0)


def test_full_passes_identical(ctx):
    from paper_2106_15789_gb300 import sc

    cube = small_cube().cuda()
    a = ctx.run(cube, KERNELS_12, T, "mad", N_REPL)
    b = ctx.run(cube, KERNELS_12, T, "mad", N_REPL, flags=sc.SC_FLAG_NO_FAST_SELECT)
    assert a[1] == b[1] and a[2] == b[2]
    assert torch.equal(a[0], b[0])


def test_run_host_matches_device(ctx):
    cube = small_cube()
    a = ctx.run(cube.cuda(), KERNELS_12, T, "mad", N_REPL)
    b = ctx.run_host(cube.contiguous(), KERNELS_12, T, "mad", N_REPL)
    assert a[1] == b[1] and a[2] == b[2]
    assert torch.equal(a[0].cpu(), b[0])


@pytest.mark.parametrize("shape", [(19, 23, 37), (1, 50, 40), (30, 1, 1), (5, 3, 200), (200, 2, 3), (7, 9, 1),
                                   (33, 65, 31), (2, 1, 1)])
def test_ragged_shapes(ctx, shape):
    rng = np.random.default_rng(sum(shape))
    c = rng.standard_normal(shape)
    for _ in range(4):
        p = tuple(int(rng.integers(0, n)) for n in shape)
        c[p] += rng.choice([-1, 1]) * 8.0
    c[rng.random(shape) < 0.05] = np.nan
    c = c.astype(np.float32)
    if not np.isfinite(c).any():
        c.flat[0] = 1.0
    kernels = [(0.0, 0), (3.0, 3), (10.0, 15), (6.0, 1), (0.0, 31)]
    check_run(ctx, torch.from_numpy(c), kernels, t=2.5)


def test_errors(ctx):
    from paper_2106_15789_gb300 import sc

    cube = torch.full((8, 8, 8), float("nan"), device="cuda")
    mask = torch.full(cube.shape, 7, dtype=torch.uint8, device="cuda")
    with pytest.raises(sc.ScError) as e:
        ctx.run(cube, KERNELS_12, T, mask=mask)
    assert e.value.code == sc.SC_ERR_ALLNAN
    assert mask.sum().item() == 0
    good = torch.randn(8, 8, 8, device="cuda")
    for kernels, t, mode, code in (([(3.0, 4)], T, "mad", sc.SC_ERR_ARG), ([(-1.0, 3)], T, "mad", sc.SC_ERR_ARG),
                                   ([(float("nan"), 3)], T, "mad", sc.SC_ERR_ARG), ([(3.0, 3)], 0.0, "mad", sc.SC_ERR_ARG),
                                   ([(3.0, 3)], T, 7, sc.SC_ERR_ARG), ([(3.0, 3)] * 65, T, "mad", sc.SC_ERR_ARG),
                                   ([(3.0, 129)], T, "mad", sc.SC_ERR_UNSUPPORTED)):
        with pytest.raises(sc.ScError) as e:
            ctx.run(good, kernels, t, mode)
        assert e.value.code == code, (kernels, t, mode)
    big = torch.empty((1, 1, ctx.max_voxels + 1), device="cuda")
    with pytest.raises(sc.ScError) as e:
        ctx.run(big, KERNELS_12, T)
    assert e.value.code == sc.SC_ERR_BUDGET


def test_stats_and_profiling(ctx):
    ctx.stats(reset=True)
    ctx.set_profiling(True)
    ctx.run(small_cube().cuda(), KERNELS_12, T)
    st = ctx.stats(reset=True)
    ctx.set_profiling(False)
    assert st["launches"] > 12 and st["runs"] == 1
    assert st["ms_smooth"] > 0 and st["smooth_launches"] == 11


def test_unaligned_cube_gives_the_same_result(ctx):
    """A cube starting 4 bytes past a 16-byte boundary takes the paths
    without 16-byte loads and TMA; the result must not change."""
    cube = small_cube().cuda()
    buf = torch.empty(cube.numel() + 1, device="cuda")
    buf[1:].copy_(cube.flatten())
    view = buf[1:].view(cube.shape)
    assert view.data_ptr() % 16 == 4
    m0, s0, z0 = ctx.run(cube, KERNELS_12, T)
    m0 = m0.clone()
    m1, s1, z1 = ctx.run(view, KERNELS_12, T)
    assert torch.equal(m0, m1) and s0 == s1 and z0 == z1


def test_kernel_of_each_pair(ctx):
    """The library reports which smoothing kernel each pair ran on: none for
    the unsmoothed cube, the spectral kernel for spatially unsmoothed pairs,
    the warp-specialised 64 x 32 one for FWHM 3 and 6 px with widths <= 15,
    the 64 x 16 one for width 31, the shared spatial passes for the later
    pairs of one spatial kernel, the generic one when forced."""
    from paper_2106_15789_gb300 import sc

    cube = small_cube().cuda()  # nx = 64: TMA-addressable
    for flags in (0, sc.SC_FLAG_NO_SHARE):
        ctx.run(cube, KERNELS_20, T, flags=flags)
        codes = ctx.stats()["smooth_kernel_pair"][:len(KERNELS_20)]
        for k, ((fwhm, wz), code) in enumerate(zip(KERNELS_20, codes)):
            if fwhm == 0:
                want = sc.SC_KERNEL_NONE if wz == 0 else sc.SC_KERNEL_Z
            elif flags == 0 and KERNELS_20[k - 1][0] == fwhm:
                want = sc.SC_KERNEL_SHARED
            else:
                want = sc.SC_KERNEL_WS32 if wz <= 15 else sc.SC_KERNEL_WS16
            assert code == want, ((fwhm, wz), flags, code)
    ctx.run(cube, KERNELS_12, T, flags=sc.SC_FLAG_GENERIC)
    codes = ctx.stats(reset=True)["smooth_kernel_pair"][:len(KERNELS_12)]
    assert codes[0] == sc.SC_KERNEL_NONE
    assert all(c == sc.SC_KERNEL_GENERIC for c in codes[1:]), codes


@pytest.mark.parametrize("shape", [(96, 64, 64), (37, 70, 131), (40, 33, 68)])
def test_every_variant_gives_the_same_floats(ctx, shape):
    """Each kernel variant the autotuner may choose, forced through sc_smooth,
    equals the generic kernel bit for bit (with and without replacement)."""
    from paper_2106_15789_gb300 import sc

    rng = np.random.default_rng(sum(shape))
    c = rng.standard_normal(shape).astype(np.float32)
    c[rng.random(shape) < 0.03] = np.nan
    cube = torch.from_numpy(c).cuda()
    mask = torch.from_numpy((rng.random(shape) < 0.05).astype(np.uint8)).cuda()
    spatial = [sc.SC_VARIANT_WS, sc.SC_VARIANT_WS16, sc.SC_VARIANT_TILE]
    spectral = [sc.SC_VARIANT_Z8, sc.SC_VARIANT_Z4, sc.SC_VARIANT_Z4_512, sc.SC_VARIANT_Z8_512]
    for kernel, variants in (((0.0, 3), spectral), ((0.0, 7), spectral), ((0.0, 15), spectral), ((3.0, 7), spatial),
                             ((6.0, 15), spatial), ((5.0, 1), spatial)):
        for m, v in ((None, 0.0), (mask, 2.5)):
            ref = ctx.smooth(cube, kernel, mask=m, replacement_value=v, flags=sc.SC_FLAG_GENERIC).clone()
            for var in variants:
                got = ctx.smooth(cube, kernel, mask=m, replacement_value=v, flags=sc.SC_SMOOTH_VARIANT(var))
                assert torch.equal(torch.isnan(got), torch.isnan(ref)), (kernel, var)
                assert torch.equal(torch.nan_to_num(got), torch.nan_to_num(ref)), (kernel, var)


@pytest.mark.parametrize("shape", [(128, 64, 64), (37, 70, 131), (9, 33, 65), (3, 1, 200)])
def test_specialised_kernels_equal_generic(ctx, shape):
    """Exact fixed-point arithmetic: every smoothing kernel variant gives the
    same floats, whatever its tiling."""
    from paper_2106_15789_gb300 import sc

    rng = np.random.default_rng(77)
    c = rng.standard_normal(shape).astype(np.float32)
    c[rng.random(shape) < 0.03] = np.nan
    cube = torch.from_numpy(c).cuda()
    mask = torch.from_numpy((rng.random(shape) < 0.05).astype(np.uint8)).cuda()
    for kernel in [(0.0, 3), (0.0, 7), (0.0, 15), (0.0, 31), (0.0, 63), (3.0, 0), (3.0, 3), (5.0, 7), (6.0, 1), (6.0, 7),
                   (10.0, 5), (6.0, 15)]:
        for m, v in ((None, 0.0), (mask, 2.5)):
            a = ctx.smooth(cube, kernel, mask=m, replacement_value=v)
            b = ctx.smooth(cube, kernel, mask=m, replacement_value=v, flags=sc.SC_FLAG_GENERIC)
            assert torch.equal(torch.nan_to_num(a, nan=7e7), torch.nan_to_num(b, nan=7e7)), (shape, kernel, m is None)


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("peak", [1e5, 1e7])
def test_bright_point_source(ctx, peak):
    """A point source of `peak` noise levels in unit noise. The fixed-point
    scale follows max|C|, so up to 1e5 sigma the smoothed values stay within
    1e-5 sigma_k of the oracle, or within 4 float32 ulps where |S| is so large
    that the float32 S itself cannot resolve 1e-5 sigma_k (next to the
    source), and the sigmas within 1e-6. Beyond 2^20 sigma_0 the library says
    that exactness may be lost (SC_WARN_RANGE); only sigma_0 and the warning
    are checked there."""
    from paper_2106_15789_gb300 import sc

    rng = np.random.default_rng(11)
    c = rng.standard_normal((64, 72, 80)).astype(np.float32)
    c[30, 36, 41] = peak
    kernels = [(0.0, 0), (6.0, 0), (6.0, 7), (10.0, 15)]
    ctx.stats(reset=True)
    m, sig, s0 = ctx.run(torch.from_numpy(c).cuda(), kernels, T, "mad", N_REPL)
    warned = bool(ctx.stats()["warnings"] & sc.SC_WARN_RANGE)
    assert warned == (peak > 2.0 ** 20 * s0), (peak, s0, warned)
    m_ref, s_ref, s0_ref, ss = O.sc_filter(c, kernels, T, "mad", N_REPL, return_smoothed=True)
    assert abs(s0 - s0_ref) <= SIG_RTOL * s0_ref
    if peak > 2.0 ** 20:
        return
    for a, b in zip(sig, s_ref):
        assert abs(a - b) <= SIG_RTOL * b, (a, b)
    ndiff, bad = band_disagreements(m.cpu().numpy(), m_ref, ss, s_ref, T)
    assert not bad
    got = ctx.copy_smoothed(c.shape).cpu().numpy().astype(np.float64)  # the last pair's S
    ref = ss[-1]
    err = np.abs(got - ref)
    tol = np.maximum(S_TOL * s_ref[-1], 4 * np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64))
    assert np.all(err <= tol), (err.max(), s_ref[-1])
    # without replacement the source itself is smoothed by every pair
    ctx.run(torch.from_numpy(c).cuda(), kernels, T, "mad", 0.0)
    got = ctx.copy_smoothed(c.shape).cpu().numpy().astype(np.float64)
    _, s_ref0, _, ss0 = O.sc_filter(c, kernels, T, "mad", 0.0, return_smoothed=True)
    ref = ss0[-1]
    assert np.abs(ref).max() > 10.0
    tol = np.maximum(S_TOL * s_ref0[-1], 4 * np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64))
    assert np.all(np.abs(got - ref) <= tol)
