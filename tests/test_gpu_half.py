"""The 16-bit precision form (sc_run_half), through the C ABI.

The library's result on a BF16 / FP16 cube with per-channel scales must be
the result of S+C on the decoded float32 cube (decode(x) * scale[z], one
float32 rounding): bit-identical to sc_run on that cube and within the usual
tolerances of the oracle on it. Against the original float32 cube the 16-bit
storage itself changes sigma and the mask; those differences are reported
and bounded loosely (they are a property of the storage, not of the code).
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
    cube = make_cube(SMALL)
    bits, scale = encode_half(cube, bf16)
    m_h, sig_h, s0_h = ctx.run_half(bits.cuda(), bf16, scale.cuda(), KERNELS_12, T, "mad", N_REPL)
    m_f, sig_f, s0_f = ctx.run(cube.cuda(), KERNELS_12, T, "mad", N_REPL)
    rel = max(abs(a - b) / b for a, b in zip(sig_h + [s0_h], sig_f + [s0_f]))
    disagree = (m_h != m_f).sum().item() / m_f.numel()
    print(f"{'bf16' if bf16 else 'fp16'}: max sigma rel err {rel:.2e}, mask disagreement {disagree:.2e}")
    # 8 (BF16) / 11 (FP16) significant bits: sigma moves by well under a percent
    assert rel < (5e-3 if bf16 else 5e-4)
    assert disagree < (2e-2 if bf16 else 2e-3)


def test_half_arguments(ctx):
    from paper_2106_15789_gb300 import sc

    cube = make_cube(SMALL)
    bits, scale = encode_half(cube, True)
    with pytest.raises(sc.ScError):
        ctx.run_half(bits.cuda(), True, scale[:-1].cuda(), KERNELS_12, T)
    with pytest.raises(sc.ScError):
        ctx.run_half(cube.cuda(), True, scale.cuda(), KERNELS_12, T)  # float storage is not 16-bit bits
