"""sc_run_host_many through the C ABI: a sequence of cubes in (pinned) host
memory, the next cube's copy in and the last mask's copy out overlapped with
the current cube's run. Each cube's mask and sigmas must be exactly those of
sc_run (float32) or sc_run_half (16-bit) on the same cube; a caller mask is
read first with SC_FLAG_ACCUMULATE; arguments are checked."""
import numpy as np
import pytest
import torch

from synth.cubes import KERNELS_12, CubeSpec, encode_half, make_cube

pytestmark = pytest.mark.gpu

T, N_REPL = 3.5, 2.0


@pytest.fixture(scope="module")
def ctx():
    from paper_2106_15789_gb300 import Context

    c = Context(0, 1 << 22)
    yield c
    c.close()


def cubes(shape, k, seed=81):
    nx, ny, nz = shape
    return [make_cube(CubeSpec(nx=nx, ny=ny, nz=nz, seed=seed + i, n_gal=5, snr=(3.0, 12.0), fwhm_xy=(2.0, 6.0),
                               fwhm_z=(5.0, 20.0))) for i in range(k)]


@pytest.mark.parametrize("shape", [(64, 48, 40), (67, 45, 33)])
def test_float32_sequence_equals_runs(ctx, shape):
    cs = cubes(shape, 5)
    hosts = [c.pin_memory() for c in cs]
    masks, sigs, s0s = ctx.run_host_many(hosts, KERNELS_12, T, "mad", N_REPL)
    for c, m, sg, s0 in zip(cs, masks, sigs, s0s):
        m_ref, sg_ref, s0_ref = ctx.run(c.cuda(), KERNELS_12, T, "mad", N_REPL)
        assert torch.equal(m, m_ref.cpu()) and sg == sg_ref and s0 == s0_ref


@pytest.mark.parametrize("bf16", [True, False], ids=["bf16", "fp16"])
def test_16_bit_sequence_equals_run_half(ctx, bf16):
    from paper_2106_15789_gb300 import sc

    cs = cubes((64, 40, 48), 3, seed=91)
    enc = [encode_half(c, bf16) for c in cs]
    hosts = [b.pin_memory() for b, _ in enc]
    scales = [s.pin_memory() for _, s in enc]
    storage = sc.SC_STORE_BF16 if bf16 else sc.SC_STORE_FP16
    masks, sigs, s0s = ctx.run_host_many(hosts, KERNELS_12, T, "mad", N_REPL, storage=storage,
                                         chan_scales_host=scales)
    for (b, s), m, sg, s0 in zip(enc, masks, sigs, s0s):
        m_ref, sg_ref, s0_ref = ctx.run_half(b.cuda(), bf16, s.cuda(), KERNELS_12, T, "mad", N_REPL)
        assert torch.equal(m, m_ref.cpu()) and sg == sg_ref and s0 == s0_ref


def test_accumulate_and_arguments(ctx):
    from paper_2106_15789_gb300 import sc

    cs = cubes((64, 32, 24), 2, seed=95)
    rng = np.random.default_rng(5)
    m0 = [torch.from_numpy((rng.random(tuple(c.shape)) < 0.02).astype(np.uint8)) for c in cs]
    masks, sigs, _ = ctx.run_host_many([c.pin_memory() for c in cs], KERNELS_12, T, "mad", N_REPL,
                                       masks_host=[m.clone().pin_memory() for m in m0],
                                       flags=sc.SC_FLAG_ACCUMULATE)
    for c, m_in, m, sg in zip(cs, m0, masks, sigs):
        ref = m_in.clone().cuda()
        _, sg_ref, _ = ctx.run(c.cuda(), KERNELS_12, T, "mad", N_REPL, mask=ref, flags=sc.SC_FLAG_ACCUMULATE)
        assert torch.equal(m, ref.cpu()) and sg == sg_ref
    lib = sc.lib()
    import ctypes

    dims = (ctypes.c_int64 * 3)(64, 32, 24)
    assert lib.sc_run_host_many(ctx.handle, 0, None, 0, None, dims, None, 12, 3.5, 0, 2.0, None, None, None, 0,
                                None) == sc.SC_ERR_ARG
    with pytest.raises(ValueError):  # 16-bit storage without scales (refused by the binding)
        ctx.run_host_many([encode_half(cs[0], True)[0]], KERNELS_12, T, storage=sc.SC_STORE_BF16)
    bits = encode_half(cs[0], True)[0]
    cubes_p = (ctypes.c_void_p * 1)(ctypes.c_void_p(bits.data_ptr()))
    masks_p = (ctypes.c_void_p * 1)(ctypes.c_void_p(m0[0].data_ptr()))
    kk = (sc.sc_kernel * 1)(sc.sc_kernel(0.0, 0))
    assert lib.sc_run_host_many(ctx.handle, 1, cubes_p, sc.SC_STORE_BF16, None, dims, kk, 1, 3.5, 0, 2.0, masks_p,
                                None, None, 0, None) == sc.SC_ERR_ARG  # and by the library
