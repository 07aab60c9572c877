"""sc_copy_sigmas: the sigmas of runs made without sigma pointers, copied in
stream order, equal the synchronous runs' (the same float32 values); a run
whose device-side status is an error leaves zeros."""
import numpy as np
import pytest
import torch

from synth.cubes import KERNELS_12, SMALL, CubeSpec, make_cube

pytestmark = pytest.mark.gpu

T, N_REPL = 3.5, 2.0


@pytest.fixture(scope="module")
def ctx():
    from paper_2106_15789_gb300 import Context

    c = Context(0, 1 << 20)
    yield c
    c.close()


def test_pipeline_without_synchronisation(ctx):
    cubes = [make_cube(CubeSpec(**{**SMALL.__dict__, "seed": SMALL.seed + i})).cuda() for i in range(2)]
    ref = [ctx.run(c, KERNELS_12, T, "mad", N_REPL) for c in cubes]  # synchronous sigmas
    nk = len(KERNELS_12)
    dev = [torch.full((nk,), -1.0, device="cuda") for _ in cubes]
    dev0 = [torch.full((1,), -1.0, device="cuda") for _ in cubes]
    host = [torch.full((nk,), -1.0).pin_memory() for _ in cubes]
    host0 = [torch.full((1,), -1.0).pin_memory() for _ in cubes]
    masks = [torch.empty(c.shape, dtype=torch.uint8, device="cuda") for c in cubes]
    for i, c in enumerate(cubes):  # run, copy, run, copy: nothing waits in between
        ctx.run(c, KERNELS_12, T, "mad", N_REPL, mask=masks[i], want_sigma=False)
        ctx.copy_sigmas(dev[i], dev0[i], nk)
        ctx.copy_sigmas(host[i], host0[i], nk)
    torch.cuda.synchronize()
    for i, (m, sig, s0) in enumerate(ref):
        want = [float(np.float32(x)) for x in sig]
        assert dev[i].cpu().tolist() == want and host[i].tolist() == want
        assert dev0[i].item() == s0 and host0[i].item() == s0
        assert torch.equal(masks[i], m)
    # a prefix of the pairs, and one destination only
    part = torch.full((3,), -1.0, device="cuda")
    ctx.copy_sigmas(part, None, 3)
    torch.cuda.synchronize()
    assert part.cpu().tolist() == [float(np.float32(x)) for x in ref[-1][1][:3]]


def test_error_status_leaves_zeros(ctx):
    """An all-NaN cube run without sigma pointers returns once enqueued; its
    device-side status (no finite voxel) makes the copies zeros, and the next
    good run's copies are its sigmas again."""
    nk = len(KERNELS_12)
    bad = torch.full((16, 24, 32), float("nan"), device="cuda")
    ctx.run(bad, KERNELS_12, T, "mad", N_REPL, want_sigma=False)
    dev = torch.full((nk,), -1.0, device="cuda")
    host0 = torch.full((1,), -1.0).pin_memory()
    ctx.copy_sigmas(dev, host0, nk)
    torch.cuda.synchronize()
    assert dev.cpu().tolist() == [0.0] * nk and host0.item() == 0.0
    good = make_cube(SMALL).cuda()
    _, sig, s0 = ctx.run(good, KERNELS_12, T, "mad", N_REPL)
    ctx.copy_sigmas(dev, host0, nk)
    torch.cuda.synchronize()
    assert dev.cpu().tolist() == [float(np.float32(x)) for x in sig] and host0.item() == s0


def test_arguments(ctx):
    from paper_2106_15789_gb300 import sc

    d = torch.empty(2 * sc.SC_MAX_KERNELS, device="cuda")
    for n in (0, sc.SC_MAX_KERNELS + 1):
        with pytest.raises(sc.ScError) as e:
            ctx.copy_sigmas(d, None, n)
        assert e.value.code == sc.SC_ERR_ARG
    with pytest.raises(ValueError):
        ctx.copy_sigmas(torch.empty(4), None, 4)  # pageable host memory
