"""Pins for the linker oracle (oracle/linker.py), checked against things other
than the oracle itself: a pure-Python breadth-first search over explicit
friend tests on tiny masks, hand-built cases whose answer follows from the
readings (distances just inside and outside the merging radius, the disk
against the box, chains, sizes at the filter limits, numbering order), and
invariants. The last test plants plausible mistakes in the oracle and checks
that each trips a pin.
"""
from collections import deque

import numpy as np
import pytest

import oracle.linker as LK


def bf_components(mask, r_xy, r_z):
    """Breadth-first search over all pairs of mask voxels with the friend test
    written out; components numbered by their first voxel in raster order."""
    vox = [tuple(int(c) for c in v) for v in np.argwhere(mask != 0)]  # raster order (z, y, x)
    friend = lambda a, b: (a[2] - b[2]) ** 2 + (a[1] - b[1]) ** 2 <= r_xy * r_xy and abs(a[0] - b[0]) <= r_z
    lab = np.zeros(mask.shape, dtype=np.int64)
    nxt = 1
    for v in vox:
        if lab[v]:
            continue
        lab[v] = nxt
        q = deque([v])
        while q:
            a = q.popleft()
            for b in vox:
                if not lab[b] and friend(a, b):
                    lab[b] = nxt
                    q.append(b)
        nxt += 1
    return lab


@pytest.mark.parametrize("r_xy,r_z", [(0, 0), (1, 1), (1, 0), (2, 1), (2, 2), (3, 0)])
@pytest.mark.parametrize("density", [0.05, 0.15])
def test_brute_force_tiny(r_xy, r_z, density):
    rng = np.random.default_rng(int(100 * density) + 10 * r_xy + r_z)
    mask = (rng.random((6, 7, 8)) < density).astype(np.uint8)
    np.testing.assert_array_equal(LK.components(mask, r_xy, r_z), bf_components(mask, r_xy, r_z))


def cube_with(points, shape=(9, 9, 12)):
    m = np.zeros(shape, dtype=np.uint8)
    for z, y, x in points:
        m[z, y, x] = 1
    return m


def n_sources(mask, r_xy, r_z):
    return int(LK.components(mask, r_xy, r_z).max())


def test_radius_limits():
    assert n_sources(cube_with([(4, 4, 2), (4, 4, 4)]), 2, 2) == 1   # dx = 2 = r
    assert n_sources(cube_with([(4, 4, 2), (4, 4, 5)]), 2, 2) == 2   # dx = 3
    assert n_sources(cube_with([(4, 4, 2), (4, 5, 4)]), 2, 2) == 2   # dx^2 + dy^2 = 5 > 4: a disk, not a box
    assert n_sources(cube_with([(4, 4, 2), (4, 5, 3)]), 1, 0) == 2   # 2 > 1
    assert n_sources(cube_with([(4, 4, 2), (4, 5, 3)]), 2, 0) == 1   # 2 <= 4
    assert n_sources(cube_with([(2, 4, 4), (4, 4, 4)]), 0, 2) == 1   # dz = 2 = r_z
    assert n_sources(cube_with([(1, 4, 4), (4, 4, 4)]), 5, 2) == 2   # dz = 3, whatever r_xy
    assert n_sources(cube_with([(4, 4, 4), (5, 4, 4)]), 0, 0) == 2   # radius 0: nothing links


def test_chain_links_transitively():
    pts = [(4, 4, x) for x in range(0, 12, 2)]  # gaps of 2
    assert n_sources(cube_with(pts), 2, 0) == 1
    assert n_sources(cube_with(pts), 1, 3) == len(pts)


def test_numbering_by_first_voxel():
    # three separate sources; first voxels in raster order: B (z=1), C (z=2, y=0), A (z=2, y=5)
    m = cube_with([(2, 5, 1), (3, 5, 1), (1, 8, 8), (2, 0, 11), (6, 0, 11)])
    lab = LK.components(m, 1, 1)
    assert lab[1, 8, 8] == 1 and lab[2, 0, 11] == 2 and lab[2, 5, 1] == 3 and lab[3, 5, 1] == 3
    assert lab[6, 0, 11] == 4  # z gap of 4 > r_z: its own source


def test_size_filters():
    m = np.zeros((12, 10, 10), dtype=np.uint8)
    m[2:7, 3:5, 1:4] = 1    # x extent 3, y 2, z 5
    m[9:11, 7:9, 7:9] = 1   # 2 x 2 x 2
    lab, ext = LK.link(m, 1, 1, min_xy=2, min_z=5)
    assert lab.max() == 1 and (lab[2:7, 3:5, 1:4] == 1).all() and (lab[9:11] == 0).all()
    assert list(ext[0]) == [1, 3, 3, 4, 2, 6, 30]
    lab, _ = LK.link(m, 1, 1, min_xy=3, min_z=1)      # y extent 2 < 3 and 2 < 3
    assert lab.max() == 0
    lab, _ = LK.link(m, 1, 1, max_z=4)                # the first is 5 channels long
    assert lab.max() == 1 and (lab[9:11, 7:9, 7:9] == 1).all() and (lab[2:7] == 0).all()
    lab, _ = LK.link(m, 1, 1, max_xy=2)               # x extent 3 > 2
    assert lab.max() == 1 and lab[10, 8, 8] == 1


def test_invariants_random():
    rng = np.random.default_rng(5)
    m = (rng.random((20, 24, 28)) < 0.06).astype(np.uint8)
    lab = LK.components(m, 2, 2)
    assert np.array_equal(lab != 0, m != 0)
    # no friend pair crosses two sources
    for dz, dy, dx in LK.offsets(2, 2):
        a = lab[max(0, -dz):lab.shape[0] - max(0, dz), max(0, -dy):lab.shape[1] - max(0, dy),
                max(0, -dx):lab.shape[2] - max(0, dx)]
        b = lab[max(0, dz):lab.shape[0] - max(0, -dz) if dz < 0 else None, max(0, dy):lab.shape[1] - max(0, -dy)
                if dy < 0 else None, max(0, dx):lab.shape[2] - max(0, -dx) if dx < 0 else None]
        both = (a != 0) & (b != 0)
        assert (a[both] == b[both]).all()
    # first voxels in raster order carry increasing ids
    flat = lab.ravel()
    ids, first = np.unique(flat[flat > 0], return_index=True)
    assert (np.diff(np.flatnonzero(flat > 0)[first]) > 0).all() and (ids == np.arange(1, ids.size + 1)).all()


# ----------------------------------------------------------------------------
# Planted mistakes.

PINS = [
    lambda: test_brute_force_tiny(2, 1, 0.15), lambda: test_brute_force_tiny(1, 0, 0.05), test_radius_limits,
    test_chain_links_transitively, test_numbering_by_first_voxel, test_size_filters, test_invariants_random,
]


def _mut_box_not_disk(orig):
    def f(r_xy, r_z):
        return [(dz, dy, dx) for dz in range(-r_z, r_z + 1) for dy in range(-r_xy, r_xy + 1)
                for dx in range(-r_xy, r_xy + 1) if (dz, dy, dx) > (0, 0, 0)]
    return f


def _mut_radius_strict(orig):
    def f(r_xy, r_z):
        return [o for o in orig(r_xy, r_z) if o[1] ** 2 + o[2] ** 2 < r_xy * r_xy or (o[1] == 0 and o[2] == 0)]
    return f


def _mut_number_by_last_voxel(orig):
    def f(mask, r_xy, r_z):
        lab = orig(mask, r_xy, r_z)
        n = int(lab.max())
        return np.where(lab > 0, n + 1 - lab, 0)
    return f


def _mut_extent_without_plus_one(orig):
    def f(labels, n):
        e = orig(labels, n).copy()
        e[:, 1] -= 1
        return e
    return f


MUTATIONS = [("offsets", _mut_box_not_disk), ("offsets", _mut_radius_strict),
             ("components", _mut_number_by_last_voxel), ("extents", _mut_extent_without_plus_one)]


@pytest.mark.parametrize("name,mut", MUTATIONS, ids=[f"{n}-{m.__name__}" for n, m in MUTATIONS])
def test_planted_mistake_is_caught(monkeypatch, name, mut):
    monkeypatch.setattr(LK, name, mut(getattr(LK, name)))
    caught = []
    for pin in PINS:
        try:
            pin()
        except (AssertionError, ValueError, IndexError):
            caught.append(pin)
    assert caught, f"planted mistake in {name} ({mut.__name__}) passed every pin"
