"""Linker (sc_link) through the C ABI against the oracle (oracle/linker.py).

Integer work: labels and extents must be identical (both number detections
by their first voxel in raster order, so the numbering is unique).
"""
import numpy as np
import pytest
import torch

import oracle.linker as LK
import oracle.sc_oracle as O
from synth.cubes import KERNELS_12, SMALL, make_cube

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2106_15789_gb300 import Context

    c = Context(0, 1 << 22)
    yield c
    c.close()


def check(ctx, mask_np, r_xy, r_z, **filt):
    mask = torch.from_numpy(mask_np.astype(np.uint8)).cuda()
    lab, n, ext = ctx.link(mask, r_xy, r_z, **filt)
    ref, ext_ref = LK.link(mask_np, r_xy, r_z, **filt)
    assert n == int(ref.max())
    np.testing.assert_array_equal(lab.cpu().numpy(), ref.astype(np.int32))
    np.testing.assert_array_equal(ext.astype(np.int64), ext_ref)
    return n


@pytest.mark.parametrize("r_xy,r_z", [(0, 0), (1, 1), (2, 2), (2, 0), (3, 1), (1, 4)])
@pytest.mark.parametrize("density", [0.02, 0.1, 0.3])
def test_random_masks(ctx, r_xy, r_z, density):
    rng = np.random.default_rng(int(1000 * density) + 7 * r_xy + r_z)
    check(ctx, rng.random((23, 31, 37)) < density, r_xy, r_z)


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 1, 50), (50, 1, 1), (3, 70, 2), (130, 9, 33)])
def test_ragged_and_thin(ctx, shape):
    rng = np.random.default_rng(sum(shape))
    check(ctx, rng.random(shape) < 0.2, 2, 2)


def test_empty_and_full(ctx):
    assert check(ctx, np.zeros((10, 11, 12), bool), 2, 2) == 0
    assert check(ctx, np.ones((10, 11, 12), bool), 1, 1) == 1
    assert check(ctx, np.ones((10, 11, 12), bool), 1, 0) == 10  # r_z = 0: the planes do not link
    assert check(ctx, np.ones((10, 11, 12), bool), 0, 0) == 10 * 11 * 12


def test_sc_mask_with_the_papers_filters(ctx):
    """The S+C mask of the small cube, linked with radius 2 and minimum sizes
    8 pixels / 5 channels (the paper's settings)."""
    m, _, _ = O.sc_filter(make_cube(SMALL).numpy(), KERNELS_12, 3.5, "mad", 2.0)
    n = check(ctx, m, 2, 2, min_xy=8, min_z=5)
    assert n > 0
    check(ctx, m, 2, 2, min_xy=3, min_z=3, max_xy=20, max_z=40)


def test_larger_random(ctx):
    rng = np.random.default_rng(3)
    m = rng.random((96, 128, 160)) < 0.04
    m[40:60, 50:90, 20:30] = True  # one big blob among the noise
    check(ctx, m, 2, 2, min_xy=2, min_z=2)


def test_arguments(ctx):
    from paper_2106_15789_gb300 import sc

    m = torch.zeros((4, 4, 4), dtype=torch.uint8, device="cuda")
    for args in ((-1, 1), (1, 33)):
        with pytest.raises(sc.ScError) as e:
            ctx.link(m, *args)
        assert e.value.code == sc.SC_ERR_ARG
