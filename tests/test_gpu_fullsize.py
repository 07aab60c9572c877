"""Parity at the full WALLABY size (1200 x 1200 x 1024, 12 kernel pairs), in
the launch configuration bench.py times, on outputs the oracle can compute
one by one:

* sigma_0 against the oracle over all finite voxels;
* the 12 pairs run one at a time (accumulating the mask) reproduce the
  all-pairs run: same sigmas, same mask;
* at sampled voxels (random, cube edges, the NaN border, tile seams and the
  voxels each pair detects), S of every pair against the oracle's direct sum
  over the composed kernel, with the mask as it was when the pair started;
* every sampled voxel's new mask bit against |S| > t * sigma_k (except inside
  the 1e-4 band);
* the last pair's sigma against the oracle over its whole smoothed cube;
* the 16-bit forms (FP16, BF16) on both of their read paths equal S+C on the
  decoded cube bit for bit;
* the sampled-Gaussian spatial kernel: pairs one at a time reproduce the
  all-pairs run, and S of each spatial pair at sampled voxels matches the
  oracle's direct sum.
"""
import numpy as np
import pytest
import torch

import oracle.sc_oracle as O
from synth.cubes import KERNELS_12, SC_REPLACEMENT, SC_THRESHOLD, WALLABY, make_cube

pytestmark = pytest.mark.gpu

SIG_RTOL = 1e-6
BAND = 1e-4
TILE_X, TILE_Y = 64, 32  # smoothing tile of the warp-specialised kernel


@pytest.fixture(scope="module")
def wallaby():
    from paper_2106_15789_gb300 import Context

    with torch.no_grad():
        cube = make_cube(WALLABY, device="cuda")
    ctx = Context(0, cube.numel())
    yield ctx, cube
    ctx.close()


def sample_points(shape, rng, extra=()):
    nz, ny, nx = shape
    pts = [np.stack([rng.integers(0, n, 400) for n in shape], axis=1)]
    edge = []
    for z in (0, 1, nz // 2, nz - 2, nz - 1):
        for y in (0, 15, 16, 17, TILE_Y - 1, TILE_Y, 5 * TILE_Y - 1, ny - 17, ny - 1):
            for x in (0, 16, TILE_X - 1, TILE_X, 7 * TILE_X, nx - 17, nx - 16, nx - 1):
                edge.append((z, y, x))
    pts.append(np.array(edge))
    for e in extra:
        if len(e):
            pts.append(e[rng.choice(len(e), min(len(e), 200), replace=False)])
    return np.concatenate(pts).astype(np.int64)


def oracle_s_at(c_np, m_np, value, kernel, pts):
    """The oracle's S at each point from the cube window around it: the
    replaced input (NaN -> 0, masked finite voxels -> sign * value) of the
    kernel's support, zero outside the cube, summed over the composed kernel."""
    fwhm, wz = kernel
    h = (O.kernel_1d(fwhm).size - 1) // 2
    r = (wz - 1) // 2 if wz > 1 else 0
    nz, ny, nx = c_np.shape
    out = np.empty(len(pts))
    for i, (z, y, x) in enumerate(pts):
        z0, z1 = max(z - r, 0), min(z + r + 1, nz)
        y0, y1 = max(y - h, 0), min(y + h + 1, ny)
        x0, x1 = max(x - h, 0), min(x + h + 1, nx)
        sub = c_np[z0:z1, y0:y1, x0:x1].astype(np.float64)
        fin = np.isfinite(sub)
        xr = O.replaced_input(sub, m_np[z0:z1, y0:y1, x0:x1].astype(bool), fin, value)
        s = O.smoothed_at(xr, fwhm, wz, np.array([[z - z0, y - y0, x - x0]]))[0]
        out[i] = s if np.isfinite(c_np[z, y, x]) else np.nan
    return out


def test_wallaby_sampled_parity(wallaby):
    ctx, cube = wallaby
    t, n = SC_THRESHOLD, SC_REPLACEMENT
    rng = np.random.default_rng(11)
    c_np = cube.cpu().numpy()

    # all pairs at once, as the benchmark runs them
    m_all, sig_all, s0 = ctx.run(cube, KERNELS_12, t, "mad", n)
    torch.cuda.synchronize()

    # sigma_0 over the whole cube
    fin = np.isfinite(c_np)
    s0_ref = O.noise(c_np[fin], "mad")
    assert abs(s0 - s0_ref) <= SIG_RTOL * s0_ref, (s0, s0_ref)
    del fin

    # one pair at a time, accumulating the mask
    mask = torch.zeros(cube.shape, dtype=torch.uint8, device="cuda")
    out = torch.empty_like(cube)
    value = float(np.float32(n * s0))  # sc_smooth takes the replacement value as float32
    from paper_2106_15789_gb300 import sc

    last = None
    for k, kernel in enumerate(KERNELS_12):
        before = mask.clone()
        _, sig_k, s0_k = ctx.run(cube, [kernel], t, "mad", n, mask=mask, flags=sc.SC_FLAG_ACCUMULATE)
        assert s0_k == s0
        assert abs(sig_k[0] - sig_all[k]) <= SIG_RTOL * sig_all[k], (k, kernel, sig_k[0], sig_all[k])
        b_np = before.cpu().numpy()
        a_np = mask.cpu().numpy()
        new = np.argwhere(a_np & ~b_np)
        pts = sample_points(c_np.shape, rng, extra=(new,))
        # S of this pair with the mask as it was when the pair started
        ctx.smooth(cube, kernel, mask=before, replacement_value=value, out=out)
        pts_t = torch.from_numpy(pts).cuda()
        got = out[pts_t[:, 0], pts_t[:, 1], pts_t[:, 2]].double().cpu().numpy()
        ref = oracle_s_at(c_np, b_np, value, kernel, pts)
        assert np.array_equal(np.isnan(got), np.isnan(ref)), kernel
        ok = np.isfinite(ref)
        err = np.abs(got[ok] - ref[ok])
        assert err.max() <= 1e-5 * sig_all[k], (kernel, err.max())
        bound = 4.0 * np.spacing(np.abs(ref[ok]).astype(np.float32)).astype(np.float64) + 1e-9
        assert np.all(err <= bound), (kernel, float((err / bound).max()))
        # the new mask bits at the sampled voxels (S with the run's replacement value)
        ref_run = oracle_s_at(c_np, b_np, n * s0, kernel, pts)
        det = np.isfinite(ref_run) & (np.abs(ref_run) > t * sig_k[0])
        want = b_np[tuple(pts.T)].astype(bool) | det
        have = a_np[tuple(pts.T)].astype(bool)
        off = np.flatnonzero(want != have)
        band = np.abs(np.abs(ref_run[off]) / sig_k[0] - t) < BAND
        assert band.all(), (kernel, len(off), pts[off[~band][:5]])
        last = (kernel, before, sig_k[0])

    assert torch.equal(mask, m_all), "one pair at a time differs from all pairs at once"

    # the last pair's sigma over its whole smoothed cube
    kernel, before, sig_last = last
    ctx.smooth(cube, kernel, mask=before, replacement_value=value, out=out)
    s_np = out.cpu().numpy()
    fin = np.isfinite(s_np)
    sig_ref = O.noise(s_np[fin], "mad")
    assert abs(sig_last - sig_ref) <= SIG_RTOL * sig_ref, (sig_last, sig_ref)


def _decode_on_gpu(bits, scale, bf16):
    """decode(x) * scale[z] in float32 (one rounding), on the GPU."""
    if bf16:
        v = (bits.to(torch.int32) & 0xFFFF).bitwise_left_shift(16).view(torch.float32)
    else:
        v = bits.view(torch.float16).to(torch.float32)
    return v * scale[:, None, None]


@pytest.mark.parametrize("bf16", [False, True], ids=["fp16", "bf16"])
def test_wallaby_16_bit_equals_decoded(wallaby, bf16):
    """The precision form at full size, on both of its read paths for this
    shape (the histogram-made float32 copy, and every kernel reading 16-bit
    values): bit for bit S+C on the decoded cube."""
    from paper_2106_15789_gb300 import sc
    from synth.cubes import encode_half

    ctx, cube = wallaby
    t, n = SC_THRESHOLD, SC_REPLACEMENT
    bits, scale = encode_half(cube, bf16)
    dec = _decode_on_gpu(bits, scale, bf16)
    m_ref, sig_ref, s0_ref = ctx.run(dec, KERNELS_12, t, "mad", n)
    m_ref = m_ref.clone()
    del dec
    for flags, path in ((0, 3), (sc.SC_FLAG_HALF_DIRECT, 1)):
        m, sig, s0 = ctx.run_half(bits, bf16, scale, KERNELS_12, t, "mad", n, flags=flags)
        assert ctx.stats()["half_path"] == path
        assert s0 == s0_ref and sig == sig_ref, (flags, sig, sig_ref)
        assert torch.equal(m, m_ref), (flags, int((m != m_ref).sum().item()))


def test_wallaby_sampled_gaussian_parity(wallaby):
    """The sampled-Gaussian spatial kernel at full size: pairs run one at a
    time (accumulating the mask) reproduce the all-pairs run, and S of each
    spatial pair at sampled voxels matches the oracle's direct sum (within
    1e-5 sigma_k and 4 ulps + the fixed-point quantum)."""
    from paper_2106_15789_gb300 import sc

    ctx, cube = wallaby
    t, n = SC_THRESHOLD, SC_REPLACEMENT
    rng = np.random.default_rng(12)
    c_np = cube.cpu().numpy()
    fl = sc.SC_FLAG_SAMPLED_GAUSS
    m_all, sig_all, s0 = ctx.run(cube, KERNELS_12, t, "mad", n, flags=fl)
    m_all = m_all.clone()
    mask = torch.zeros(cube.shape, dtype=torch.uint8, device="cuda")
    out = torch.empty_like(cube)
    value = float(np.float32(n * s0))
    mx = max(float(np.nanmax(np.abs(c_np))), value)
    e = int(np.frexp(np.float32(mx))[1])
    for k, kernel in enumerate(KERNELS_12):
        before = mask.clone()
        _, sig_k, _ = ctx.run(cube, [kernel], t, "mad", n, mask=mask, flags=sc.SC_FLAG_ACCUMULATE | fl)
        assert abs(sig_k[0] - sig_all[k]) <= SIG_RTOL * sig_all[k], (k, kernel, sig_k[0], sig_all[k])
        if kernel[0] == 0.0:
            continue
        b_np = before.cpu().numpy()
        pts = np.concatenate([np.stack([rng.integers(0, s, 150) for s in c_np.shape], axis=1),
                              np.array([(0, 0, 0), (c_np.shape[0] - 1, 17, 16), (512, 31, 64), (512, 32, 63)])])
        ctx.smooth(cube, kernel, mask=before, replacement_value=value, out=out, flags=fl)
        pts_t = torch.from_numpy(pts).cuda()
        got = out[pts_t[:, 0], pts_t[:, 1], pts_t[:, 2]].double().cpu().numpy()
        fwhm, wz = kernel
        taps = O.gauss_taps(fwhm)
        h, r = (taps.size - 1) // 2, (wz - 1) // 2 if wz > 1 else 0
        ref = np.empty(len(pts))
        for i, (z, y, x) in enumerate(pts):
            z0, z1 = max(z - r, 0), min(z + r + 1, c_np.shape[0])
            y0, y1 = max(y - h, 0), min(y + h + 1, c_np.shape[1])
            x0, x1 = max(x - h, 0), min(x + h + 1, c_np.shape[2])
            sub = c_np[z0:z1, y0:y1, x0:x1].astype(np.float64)
            xr = O.replaced_input(sub, b_np[z0:z1, y0:y1, x0:x1].astype(bool), np.isfinite(sub), value)
            s = O.smoothed_at(xr, fwhm, wz, np.array([[z - z0, y - y0, x - x0]]), "sampled")[0]
            ref[i] = s if np.isfinite(c_np[z, y, x]) else np.nan
        assert np.array_equal(np.isnan(got), np.isnan(ref)), kernel
        ok = np.isfinite(ref)
        err = np.abs(got[ok] - ref[ok])
        assert err.max() <= 1e-5 * sig_all[k], (kernel, err.max())
        t_sum = int(taps.sum())
        f = 62 - e - int(t_sum * t_sum * max(wz, 31) - 1).bit_length()
        bound = 4.0 * np.spacing(np.abs(ref[ok]).astype(np.float32)).astype(np.float64) + 2.0 ** -f
        assert np.all(err <= bound), (kernel, float((err / bound).max()))
    assert torch.equal(mask, m_all), "one pair at a time differs from all pairs at once"
