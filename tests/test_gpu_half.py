"""The 16-bit precision form (sc_run_half), through the C ABI.

The library's result on a BF16 / FP16 cube with per-channel scales must be
the result of S+C on the decoded float32 cube (decode(x) * scale[z], one
float32 rounding): bit-identical to sc_run on that cube and within the usual
tolerances of the oracle on it, whichever way the cube is read: decoded into
the float32 working copy by the raw-cube histogram pass (the default for
rows of 16-byte multiples), by a decoding pass of its own (other shapes, the
generic kernels), or read as 16-bit values by every kernel
(SC_FLAG_HALF_DIRECT). Against the original float32 cube the 16-bit
storage itself changes sigma and the mask: the disagreement is bounded by the
storage's precision (below), which misses the 1e-6 target.
"""
import numpy as np
import pytest
import torch

import oracle.sc_oracle as O
from synth.cubes import KERNELS_12, SMALL, decode_half, encode_half, make_cube

pytestmark = pytest.mark.gpu

T, N_REPL = 3.5, 2.0
SIG_RTOL, BAND = 1e-6, 1e-4


@pytest.fixture(scope="module")
def ctx():
    from paper_2106_15789_gb300 import Context

    c = Context(0, 1 << 22)
    yield c
    c.close()


@pytest.mark.parametrize("bf16", [True, False], ids=["bf16", "fp16"])
def test_half_is_sc_run_on_the_decoded_cube(ctx, bf16):
    cube = make_cube(SMALL)
    bits, scale = encode_half(cube, bf16)
    dec = decode_half(bits.numpy(), scale.numpy(), bf16)
    m_h, sig_h, s0_h = ctx.run_half(bits.cuda(), bf16, scale.cuda(), KERNELS_12, T, "mad", N_REPL)
    m_f, sig_f, s0_f = ctx.run(torch.from_numpy(dec).cuda(), KERNELS_12, T, "mad", N_REPL)
    assert torch.equal(m_h, m_f)
    assert sig_h == sig_f and s0_h == s0_f
    # and the oracle on the decoded cube
    m_ref, s_ref, s0_ref, ss = O.sc_filter(dec, KERNELS_12, T, "mad", N_REPL, return_smoothed=True)
    assert abs(s0_h - s0_ref) <= SIG_RTOL * s0_ref
    for a, b in zip(sig_h, s_ref):
        assert abs(a - b) <= SIG_RTOL * b
    for p in map(tuple, np.argwhere(m_h.cpu().numpy() != m_ref)):
        assert any(sk > 0 and abs(abs(s[p]) / sk - T) < BAND for s, sk in zip(ss, s_ref)), p


@pytest.mark.parametrize("bf16", [True, False], ids=["bf16", "fp16"])
def test_half_precision_against_float32(ctx, bf16):
    """Against the original float32 cube. A value stored with p significant
    bits moves by up to 2^-p of itself (p = 8 BF16, 11 FP16, rounded: half
    that), so a smoothed value near the threshold t sigma moves by about
    t 2^-p sigma; the share of voxels within that distance of the threshold is
    2 phi(t) t 2^-p per pair (phi the normal density), i.e. 2.4e-5 (BF16) and
    3.0e-6 (FP16) per pair, 2.9e-4 and 3.6e-5 over the 12 pairs: the bounds.
    Both are above the 1e-6 target, which this storage cannot reach."""
    cube = make_cube(SMALL)
    bits, scale = encode_half(cube, bf16)
    m_h, sig_h, s0_h = ctx.run_half(bits.cuda(), bf16, scale.cuda(), KERNELS_12, T, "mad", N_REPL)
    m_f, sig_f, s0_f = ctx.run(cube.cuda(), KERNELS_12, T, "mad", N_REPL)
    rel = max(abs(a - b) / b for a, b in zip(sig_h + [s0_h], sig_f + [s0_f]))
    disagree = (m_h != m_f).sum().item() / m_f.numel()
    print(f"{'bf16' if bf16 else 'fp16'}: max sigma rel err {rel:.2e}, mask disagreement {disagree:.2e}")
    p = 8 if bf16 else 11
    assert rel < 2.0 ** -p  # sigma: an order statistic of values that moved by at most 2^-p (half: rounding)
    phi_t = np.exp(-T * T / 2) / np.sqrt(2 * np.pi)
    assert disagree <= len(KERNELS_12) * 2 * phi_t * T * 2.0 ** -p


def test_half_arguments(ctx):
    from paper_2106_15789_gb300 import sc

    cube = make_cube(SMALL)
    bits, scale = encode_half(cube, True)
    with pytest.raises(sc.ScError):
        ctx.run_half(bits.cuda(), True, scale[:-1].cuda(), KERNELS_12, T)
    with pytest.raises(sc.ScError):
        ctx.run_half(cube.cuda(), True, scale.cuda(), KERNELS_12, T)  # float storage is not 16-bit bits


def _decoded(bits, scale, bf16):
    return torch.from_numpy(decode_half(bits.cpu().numpy(), scale.cpu().numpy(), bf16)).cuda()


@pytest.mark.parametrize("bf16", [True, False], ids=["bf16", "fp16"])
@pytest.mark.parametrize("mode", ["mad", "std", "gauss"])
def test_kernels_read_16_bit_values(ctx, bf16, mode):
    """Rows of 16-byte multiples: the copy made by the histogram pass
    (half_path 3, also with the generic kernels, which have no 16-bit form)
    and every kernel reading 16-bit values (half_path 1, the 16-bit forms of
    the warp-specialised and spectral kernels) give the same floats as sc_run
    on the decoded cube; with a caller mask too."""
    from paper_2106_15789_gb300 import sc

    cube = make_cube(SMALL)
    bits, scale = encode_half(cube, bf16)
    bits, scale = bits.cuda(), scale.cuda()
    ref = ctx.run(_decoded(bits, scale, bf16), KERNELS_12, T, mode, N_REPL)
    got = ctx.run_half(bits, bf16, scale, KERNELS_12, T, mode, N_REPL)
    assert ctx.stats()["half_path"] == 3
    ctx.stats(reset=True)
    direct = ctx.run_half(bits, bf16, scale, KERNELS_12, T, mode, N_REPL, flags=sc.SC_FLAG_HALF_DIRECT)
    st = ctx.stats(reset=True)
    assert st["half_path"] == 1
    assert sc.SC_KERNEL_WS32 in st["smooth_kernel_pair"] and sc.SC_KERNEL_Z in st["smooth_kernel_pair"]
    staged = ctx.run_half(bits, bf16, scale, KERNELS_12, T, mode, N_REPL,
                          flags=sc.SC_FLAG_GENERIC | sc.SC_FLAG_HALF_DIRECT)
    assert ctx.stats()["half_path"] == 3
    for r in (ref, direct, staged):
        assert torch.equal(got[0], r[0]) and got[1] == r[1] and got[2] == r[2]
    # a caller mask (the 16-bit pack of the working mask)
    rng = np.random.default_rng(3)
    m0 = torch.from_numpy((rng.random(tuple(cube.shape)) < 0.02).astype(np.uint8)).cuda()
    b = ctx.run(_decoded(bits, scale, bf16), KERNELS_12, T, mode, N_REPL, mask=m0.clone(),
                flags=sc.SC_FLAG_ACCUMULATE)
    for fl in (0, sc.SC_FLAG_HALF_DIRECT):
        a = ctx.run_half(bits, bf16, scale, KERNELS_12, T, mode, N_REPL, mask=m0.clone(),
                         flags=sc.SC_FLAG_ACCUMULATE | fl)
        assert torch.equal(a[0], b[0]) and a[1] == b[1] and a[2] == b[2]


@pytest.mark.parametrize("shape", [(64, 40, 48), (67, 45, 40), (16, 3, 200), (200, 17, 8)])
def test_16_bit_shapes(ctx, shape):
    """Several tiles with ragged tails; widths that are not multiples of 8
    take the decoding pass. Always the decoded cube's result."""
    nx, ny, nz = shape
    from paper_2106_15789_gb300 import sc
    from synth.cubes import CubeSpec

    cube = make_cube(CubeSpec(nx=nx, ny=ny, nz=nz, seed=71, n_gal=5, snr=(3.0, 15.0), fwhm_xy=(2.0, 6.0),
                              fwhm_z=(5.0, 20.0)))
    for bf16 in (True, False):
        bits, scale = encode_half(cube, bf16)
        bits, scale = bits.cuda(), scale.cuda()
        ref = ctx.run(_decoded(bits, scale, bf16), KERNELS_12, T, "mad", N_REPL)
        for fl, path in ((0, 3), (sc.SC_FLAG_HALF_DIRECT, 1)):
            got = ctx.run_half(bits, bf16, scale, KERNELS_12, T, "mad", N_REPL, flags=fl)
            assert ctx.stats()["half_path"] == (path if nx % 8 == 0 else 2)
            assert torch.equal(got[0], ref[0]) and got[1] == ref[1] and got[2] == ref[2], (shape, bf16, fl)


def test_16_bit_value_overflowing_its_scale(ctx):
    """A finite FP16 value whose product with its channel's scale overflows to
    infinity is non-finite for the kernels, as for the decoding pass."""
    from synth.cubes import CubeSpec

    cube = make_cube(CubeSpec(nx=64, ny=32, nz=40, seed=72, n_gal=3, snr=(3.0, 10.0), fwhm_xy=(2.0, 5.0),
                              fwhm_z=(5.0, 15.0)))
    bits, scale = encode_half(cube, False)
    b = bits.numpy().copy().view(np.uint16)
    b[7, 10:14, 20:30] = 0x7BFF  # 65504, the largest FP16
    sc_np = scale.numpy().copy()
    sc_np[7] = 1e35  # 65504 * 1e35 overflows float32
    bits_d, scale_d = torch.from_numpy(b.view(np.int16)).cuda(), torch.from_numpy(sc_np).cuda()
    dec = _decoded(bits_d, scale_d, False)
    assert torch.isinf(dec[7, 10, 20])
    from paper_2106_15789_gb300 import sc

    ref = ctx.run(dec, KERNELS_12, T, "mad", N_REPL)
    for fl in (0, sc.SC_FLAG_HALF_DIRECT):
        got = ctx.run_half(bits_d, False, scale_d, KERNELS_12, T, "mad", N_REPL, flags=fl)
        assert torch.equal(got[0], ref[0]) and got[1] == ref[1] and got[2] == ref[2]
