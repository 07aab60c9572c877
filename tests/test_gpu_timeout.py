"""The device-side failure path, through the C ABI, without a GPU fault.

Every wait of the warp-specialised smoothing kernel is bounded in wall time;
a wait that runs out marks the run's device state, and the run reports
SC_ERR_TIMEOUT instead of hanging. A test hook of the library makes one
producer warp skip its hand-off of one plane (and limits the kernel's waits
to 1 ms), so a consumer waits for an arrival that never comes. The run must
return SC_ERR_TIMEOUT, quickly, and the next runs on the same context must be
correct again (against the FP64 oracle).
"""
import time

import numpy as np
import pytest
import torch

import oracle.sc_oracle as O
from synth.cubes import SMALL, make_cube

pytestmark = pytest.mark.gpu

T, N_REPL = 3.5, 2.0


@pytest.fixture(scope="module")
def ctx():
    from paper_2106_15789_gb300 import Context

    c = Context(0, 1 << 20)
    yield c
    c.close()


def check_against_oracle(ctx, cube, kernels):
    m, sig, s0 = ctx.run(cube.cuda(), kernels, T, "mad", N_REPL)
    m_ref, s_ref, s0_ref, ss = O.sc_filter(cube.numpy(), kernels, T, "mad", N_REPL, return_smoothed=True)
    assert abs(s0 - s0_ref) <= 1e-6 * s0_ref
    for a, b in zip(sig, s_ref):
        assert abs(a - b) <= 1e-6 * b
    for p in map(tuple, np.argwhere(m.cpu().numpy() != m_ref)):
        assert any(sk > 0 and abs(abs(s[p]) / sk - T) < 1e-4 for s, sk in zip(ss, s_ref)), p


@pytest.mark.parametrize("kernels", [[(6.0, 0)], [(3.0, 7), (3.0, 15)], [(0.0, 0), (10.0, 3), (10.0, 7)]])
def test_missing_handoff_times_out_and_the_context_recovers(ctx, kernels):
    from paper_2106_15789_gb300 import sc

    cube = make_cube(SMALL)  # nx = 64: the TMA form of the kernel
    ctx.test_skip_handoff(True)
    t0 = time.perf_counter()
    with pytest.raises(sc.ScError) as e:
        ctx.run(cube.cuda(), kernels, T, "mad", N_REPL)
    assert e.value.code == sc.SC_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 10.0
    # the hook served one run; the context is usable and correct again
    check_against_oracle(ctx, cube, kernels)
    check_against_oracle(ctx, cube, kernels)


def test_unaligned_cube_times_out_too(ctx):
    """The same on a cube TMA cannot address (consumers fill the tiles)."""
    from paper_2106_15789_gb300 import sc

    cube = make_cube(SMALL)[:, :, :61].contiguous()  # 61 columns: rows not 16-byte multiples
    ctx.test_skip_handoff(True)
    with pytest.raises(sc.ScError) as e:
        ctx.run(cube.cuda(), [(6.0, 3)], T, "mad", N_REPL)
    assert e.value.code == sc.SC_ERR_TIMEOUT
    check_against_oracle(ctx, cube, [(6.0, 3)])
