"""CPU oracle of SoFiA 2's linker.

TEST INFRASTRUCTURE ONLY. Nothing in the library imports this module: only
tests/ and the CPU-baseline / reference legs of bench.py use it. It shares no
code with the CUDA path.

What the paper says (Westmeier et al. 2021, SoFiA 2):

* Sect. 4.3 "Linking": the linker turns the binary mask of the source finder
  into individual detections with a friends-of-friends algorithm that links
  all mask pixels within a user-given merging radius, in the spatial plane
  and along the spectral axis (sources are 3-D collections of pixels), and
  gives every detection a unique identifier. Minimum and maximum size
  filters, spatial and spectral, remove detections that are too small or
  too large.
* Sect. 6: merging radius 2 pixels / channels, minimum size 8 spatial pixels
  and 5 spectral channels.

The paper gives no more than that; these readings fill the gaps (each is
listed with its reason in the design notes):

1. Friends. Two mask voxels are friends when dx^2 + dy^2 <= r_xy^2 (within
   the merging radius in the spatial plane) and |dz| <= r_z (along the
   spectral axis). Friends-of-friends: a detection is a connected component
   of the mask under this relation.
2. Identifiers. Detections are numbered 1, 2, ... in raster order (z, then
   y, then x) of their first voxel; voxels outside the mask get 0.
3. Sizes. A detection's size along an axis is its extent, max - min + 1 of
   its voxels' coordinates. It is removed when its x or y extent is below
   min_xy or its z extent below min_z, or, for a maximum above 0, when its x
   or y extent exceeds max_xy or its z extent max_z. The kept detections are
   renumbered 1, 2, ... in the same order; removed voxels get 0.
"""
from __future__ import annotations

import numpy as np
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components


def offsets(r_xy: int, r_z: int) -> list[tuple[int, int, int]]:
    """(dz, dy, dx) of the friends of a voxel that come after it in raster
    order (reading 1); the other half is their mirror image."""
    if r_xy < 0 or r_z < 0:
        raise ValueError("merging radii must be non-negative")
    out = []
    for dz in range(-r_z, r_z + 1):
        for dy in range(-r_xy, r_xy + 1):
            for dx in range(-r_xy, r_xy + 1):
                if dx * dx + dy * dy > r_xy * r_xy:
                    continue
                if (dz, dy, dx) > (0, 0, 0):
                    out.append((dz, dy, dx))
    return out


def components(mask: np.ndarray, r_xy: int, r_z: int) -> np.ndarray:
    """Friends-of-friends components (reading 1), numbered by first voxel in
    raster order (reading 2); int64 labels, 0 outside the mask."""
    m = np.asarray(mask) != 0
    nz, ny, nx = m.shape
    idx = -np.ones(m.shape, dtype=np.int64)
    vox = np.flatnonzero(m)
    idx.ravel()[vox] = np.arange(vox.size)
    rows, cols = [], []
    for dz, dy, dx in offsets(r_xy, r_z):
        # pairs (v, v + d) with both in the cube and in the mask
        z0, z1 = max(0, -dz), min(nz, nz - dz)
        y0, y1 = max(0, -dy), min(ny, ny - dy)
        x0, x1 = max(0, -dx), min(nx, nx - dx)
        if z0 >= z1 or y0 >= y1 or x0 >= x1:
            continue
        a = idx[z0:z1, y0:y1, x0:x1]
        b = idx[z0 + dz:z1 + dz, y0 + dy:y1 + dy, x0 + dx:x1 + dx]
        both = (a >= 0) & (b >= 0)
        rows.append(a[both])
        cols.append(b[both])
    n = vox.size
    lab = np.zeros(m.shape, dtype=np.int64)
    if n == 0:
        return lab
    r = np.concatenate(rows) if rows else np.zeros(0, dtype=np.int64)
    c = np.concatenate(cols) if cols else np.zeros(0, dtype=np.int64)
    graph = coo_matrix((np.ones(r.size, dtype=np.int8), (r, c)), shape=(n, n))
    _, comp = connected_components(graph, directed=False)
    # renumber by the first voxel (vox is in raster order)
    first = np.full(comp.max() + 1, n, dtype=np.int64)
    np.minimum.at(first, comp, np.arange(n))
    order = np.argsort(first, kind="stable")
    new_id = np.empty_like(order)
    new_id[order] = np.arange(1, order.size + 1)
    lab.ravel()[vox] = new_id[comp]
    return lab


def extents(labels: np.ndarray, n: int) -> np.ndarray:
    """Bounding box of every detection 1 .. n: rows (x_min, x_max, y_min,
    y_max, z_min, z_max) and the voxel count."""
    out = np.zeros((n, 7), dtype=np.int64)
    if n == 0:
        return out
    z, y, x = np.nonzero(labels)
    l = labels[z, y, x] - 1
    for col, (arr, fn, init) in enumerate([(x, np.minimum, np.iinfo(np.int64).max), (x, np.maximum, -1),
                                           (y, np.minimum, np.iinfo(np.int64).max), (y, np.maximum, -1),
                                           (z, np.minimum, np.iinfo(np.int64).max), (z, np.maximum, -1)]):
        v = np.full(n, init, dtype=np.int64)
        fn.at(v, l, arr)
        out[:, col] = v
    out[:, 6] = np.bincount(l, minlength=n)
    return out


def link(mask: np.ndarray, r_xy: int, r_z: int, min_xy: int = 1, min_z: int = 1, max_xy: int = 0,
         max_z: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Labels (int64, 0 = background) of the detections that pass the size
    filters (reading 3), numbered 1 .. n in raster order of their first
    voxel, and their extents (rows as in :func:`extents`)."""
    lab = components(mask, r_xy, r_z)
    n = int(lab.max())
    ext = extents(lab, n)
    sx = ext[:, 1] - ext[:, 0] + 1
    sy = ext[:, 3] - ext[:, 2] + 1
    sz = ext[:, 5] - ext[:, 4] + 1
    keep = (sx >= min_xy) & (sy >= min_xy) & (sz >= min_z)
    if max_xy > 0:
        keep &= (sx <= max_xy) & (sy <= max_xy)
    if max_z > 0:
        keep &= sz <= max_z
    new_id = np.zeros(n + 1, dtype=np.int64)
    new_id[1:][keep] = np.arange(1, int(keep.sum()) + 1)
    return new_id[lab], ext[keep]
