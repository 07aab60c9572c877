"""Stream of sub-cubes: sc_submit / sc_poll with an admission budget, through
the C ABI. Every job must give exactly what the synchronous entry points give
for the same cube; admission must refuse a job that would exceed the budget.
"""
import numpy as np
import pytest
import torch

import oracle.sc_oracle as O
from synth.cubes import KERNELS_12, KERNELS_20, CubeSpec, decode_half, encode_half, make_cube

pytestmark = pytest.mark.gpu

T, N_REPL = 4.0, 2.0
SHAPES = [(48, 40, 64), (67, 96, 33), (100, 64, 128), (40, 37, 61), (80, 80, 80)]


@pytest.fixture(scope="module")
def setup():
    from paper_2106_15789_gb300 import Context

    cubes = [make_cube(CubeSpec(nx=nx, ny=ny, nz=nz, seed=300 + i, n_gal=5, snr=(3.0, 9.0), fwhm_xy=(2.0, 5.0),
                                fwhm_z=(4.0, 12.0), name=f"stream-{i}")).cuda()
             for i, (nz, ny, nx) in enumerate(SHAPES)]
    ctx = Context(0, max(c.numel() for c in cubes))
    yield ctx, cubes
    ctx.close()


def test_jobs_equal_synchronous_runs(setup):
    from paper_2106_15789_gb300 import sc

    ctx, cubes = setup
    ctx.set_budget(0)
    stores = [sc.SC_STORE_F32, sc.SC_STORE_BF16, sc.SC_STORE_FP16, sc.SC_STORE_F32, sc.SC_STORE_BF16]
    jobs = {}
    for c, store in zip(cubes, stores):
        if store == sc.SC_STORE_F32:
            jid, m = ctx.submit(c, KERNELS_12, T, "mad", N_REPL)
            jobs[jid] = (c, store, None, None, m)
        else:
            bits, scale = encode_half(c, store == sc.SC_STORE_BF16)
            bits, scale = bits.cuda(), scale.cuda()
            jid, m = ctx.submit(bits, KERNELS_12, T, "mad", N_REPL, storage=store, chan_scale=scale)
            jobs[jid] = (c, store, bits, scale, m)
    done = {}
    while len(done) < len(jobs):
        r = ctx.poll(len(KERNELS_12), wait=True)
        assert r is not None
        jid, status, latency, sig, sig0 = r
        assert status == sc.SC_OK and latency > 0.0
        done[jid] = (sig, sig0)
    assert ctx.poll(len(KERNELS_12)) is None
    for jid, (c, store, bits, scale, m) in jobs.items():
        if store == sc.SC_STORE_F32:
            m_ref, sig_ref, s0_ref = ctx.run(c, KERNELS_12, T, "mad", N_REPL)
        else:
            m_ref, sig_ref, s0_ref = ctx.run_half(bits, store == sc.SC_STORE_BF16, scale, KERNELS_12, T, "mad", N_REPL)
        assert torch.equal(m, m_ref), jid
        assert done[jid] == (sig_ref, s0_ref), jid


def test_admission_budget(setup):
    from paper_2106_15789_gb300 import sc

    ctx, cubes = setup
    c = cubes[0]
    job_bytes = c.numel() * 5  # float32 cube + uint8 mask
    ctx.set_budget(job_bytes - 1)
    with pytest.raises(sc.ScError) as e:
        ctx.submit(c, KERNELS_12, T)
    assert e.value.code == sc.SC_ERR_BUDGET
    ctx.set_budget(job_bytes)
    jid, _ = ctx.submit(c, KERNELS_12, T)
    with pytest.raises(sc.ScError) as e:  # still in flight until polled
        ctx.submit(c, KERNELS_12, T, mask=torch.empty_like(c, dtype=torch.uint8))
    assert e.value.code == sc.SC_ERR_BUDGET
    r = ctx.poll(len(KERNELS_12), wait=True)
    assert r[0] == jid
    jid2, _ = ctx.submit(c, KERNELS_12, T)  # admitted again once the first is returned
    assert ctx.poll(len(KERNELS_12), wait=True)[0] == jid2
    ctx.set_budget(0)


def test_config5_jobs_against_the_oracle(setup):
    """Jobs with the stream's own kernel list ({0,3,6,10} px x {0,3,7,15,31}
    ch, t = 4; widths 31 run on the 64 x 16 tiles, FWHM 10 on the 7-9-9
    cascade) against the FP64 oracle: a float32 job on its cube, a BF16 job
    on the decoded cube. Sigmas within 1e-6, the mask outside the band."""
    from paper_2106_15789_gb300 import sc

    ctx, cubes = setup
    ctx.set_budget(0)
    c = make_cube(CubeSpec(nx=72, ny=56, nz=96, seed=333, n_gal=6, snr=(3.0, 12.0), fwhm_xy=(2.0, 6.0),
                           fwhm_z=(5.0, 30.0), name="stream-oracle"))
    bits, scale = encode_half(c, True)
    dec = decode_half(bits.numpy(), scale.numpy(), True)
    j1, m1 = ctx.submit(c.cuda(), KERNELS_20, T, "mad", N_REPL)
    j2, m2 = ctx.submit(bits.cuda(), KERNELS_20, T, "mad", N_REPL, storage=sc.SC_STORE_BF16, chan_scale=scale.cuda())
    res = {}
    while len(res) < 2:
        r = ctx.poll(len(KERNELS_20), wait=True)
        assert r is not None and r[1] == sc.SC_OK
        res[r[0]] = (r[3], r[4])
    for jid, m, cube in ((j1, m1, c.numpy()), (j2, m2, dec)):
        sig, s0 = res[jid]
        m_ref, s_ref, s0_ref, ss = O.sc_filter(cube, KERNELS_20, T, "mad", N_REPL, return_smoothed=True)
        assert abs(s0 - s0_ref) <= 1e-6 * s0_ref
        for k, (a, b) in enumerate(zip(sig, s_ref)):
            assert abs(a - b) <= 1e-6 * b, (jid, KERNELS_20[k], a, b)
        for p in map(tuple, np.argwhere(m.cpu().numpy() != m_ref)):
            assert any(sk > 0 and abs(abs(s[p]) / sk - T) < 1e-4 for s, sk in zip(ss, s_ref)), (jid, p)
