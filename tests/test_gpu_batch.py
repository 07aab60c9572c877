"""Batched S+C (sc_run_batch) and the autotuner (sc_autotune), through the C ABI.

A batch is many independent sub-cubes (each with its own sigma_0 and
sigma_k); it must equal running sc_run on every cube in turn, bit for bit,
with or without CUDA-graph capture, and one of its cubes is checked against
the oracle. The autotuner may only change the time, never the results.
"""
import numpy as np
import pytest
import torch

import oracle.sc_oracle as O
from synth.cubes import KERNELS_12, CubeSpec, make_cube

pytestmark = pytest.mark.gpu

T, N_REPL = 3.5, 2.0
SIG_RTOL, BAND = 1e-6, 1e-4

# uneven shapes: a ragged tail in every axis, some not TMA-addressable (nx % 4 != 0)
SHAPES = [(40, 37, 67), (96, 64, 129), (70, 101, 48), (128, 33, 80), (61, 90, 55), (132, 96, 100)]


@pytest.fixture(scope="module")
def batch():
    from paper_2106_15789_gb300 import Context

    cubes = []
    for i, (nz, ny, nx) in enumerate(SHAPES):
        spec = CubeSpec(nx=nx, ny=ny, nz=nz, seed=100 + i, n_gal=6, snr=(3.0, 8.0), fwhm_xy=(2.0, 5.0),
                        fwhm_z=(4.0, 12.0), nan_corner=(8, 8, 5) if i == 2 else None, name=f"batch-{i}")
        cubes.append(make_cube(spec).cuda())
    ctx = Context(0, max(c.numel() for c in cubes))
    yield ctx, cubes
    ctx.close()


def run_each(ctx, cubes, kernels):
    out = []
    for c in cubes:
        m, sig, s0 = ctx.run(c, kernels, T, "mad", N_REPL)
        out.append((m.clone(), sig, s0))
    return out


@pytest.mark.parametrize("graph", [False, True])
def test_batch_equals_single_runs(batch, graph):
    from paper_2106_15789_gb300 import sc

    ctx, cubes = batch
    ref = run_each(ctx, cubes, KERNELS_12)
    flags = sc.SC_FLAG_GRAPH if graph else 0
    for _ in range(2 if graph else 1):  # with a graph: capture, then replay
        masks, sigs, s0s = ctx.run_batch(cubes, KERNELS_12, T, "mad", N_REPL, flags=flags)
        for i, (m_ref, sig_ref, s0_ref) in enumerate(ref):
            assert torch.equal(masks[i], m_ref), i
            assert sigs[i] == sig_ref, i
            assert s0s[i] == s0_ref, i


def test_graph_replay_reads_current_data(batch):
    from paper_2106_15789_gb300 import sc

    ctx, cubes = batch
    work = [c.clone() for c in cubes]
    masks = [torch.empty(c.shape, dtype=torch.uint8, device="cuda") for c in work]
    ctx.run_batch(work, KERNELS_12, T, "mad", N_REPL, masks=masks, flags=sc.SC_FLAG_GRAPH)
    # new contents in the same buffers: the replayed graph must see them
    for w, c in zip(work, cubes):
        w.copy_(torch.flip(c, dims=[2]))
    got, sigs, s0s = ctx.run_batch(work, KERNELS_12, T, "mad", N_REPL, masks=masks, flags=sc.SC_FLAG_GRAPH)
    ref = run_each(ctx, work, KERNELS_12)
    for i, (m_ref, sig_ref, s0_ref) in enumerate(ref):
        assert torch.equal(got[i], m_ref), i
        assert sigs[i] == sig_ref and s0s[i] == s0_ref, i


def test_batch_cube_against_oracle(batch):
    ctx, cubes = batch
    i = 2  # the cube with NaN
    masks, sigs, s0s = ctx.run_batch(cubes, KERNELS_12, T, "mad", N_REPL)
    c_np = cubes[i].cpu().numpy()
    m_ref, s_ref, s0_ref, ss = O.sc_filter(c_np, KERNELS_12, T, "mad", N_REPL, return_smoothed=True)
    assert abs(s0s[i] - s0_ref) <= SIG_RTOL * s0_ref
    for a, b in zip(sigs[i], s_ref):
        assert abs(a - b) <= SIG_RTOL * b
    diff = np.argwhere(masks[i].cpu().numpy() != m_ref)
    for p in map(tuple, diff):
        assert any(sk > 0 and abs(abs(s[p]) / sk - T) < BAND for s, sk in zip(ss, s_ref)), p


def test_autotune_keeps_results(batch):
    ctx, cubes = batch
    before = run_each(ctx, cubes, KERNELS_12)
    for c in cubes:
        ctx.autotune(c.shape, KERNELS_12)
    after = run_each(ctx, cubes, KERNELS_12)
    for (m0, s0, z0), (m1, s1, z1) in zip(before, after):
        assert torch.equal(m0, m1)
        assert s0 == s1 and z0 == z1


def test_batch_errors(batch):
    from paper_2106_15789_gb300 import sc

    ctx, cubes = batch
    with pytest.raises(sc.ScError) as e:
        ctx.run_batch(cubes, [(3.0, 4)], T)  # even boxcar
    assert e.value.code == sc.SC_ERR_ARG
    big = torch.zeros((ctx.max_voxels // (64 * 64) + 1, 64, 64), device="cuda")
    with pytest.raises(sc.ScError) as e:
        ctx.run_batch([cubes[0], big], KERNELS_12, T)
    assert e.value.code == sc.SC_ERR_BUDGET
    with pytest.raises(sc.ScError):
        ctx.run_batch([], KERNELS_12, T)
