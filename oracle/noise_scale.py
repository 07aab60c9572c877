"""CPU FP64 oracle of SoFiA 2's local noise normalisation.

TEST INFRASTRUCTURE ONLY. Nothing in the library imports this module: only
tests/, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
bench.py use it. It shares no code with the CUDA path.

What the paper says (Westmeier et al. 2021, SoFiA 2):

* Sect. 4.1 "Input and preconditioning": when the noise level is not constant
  across the cube, SoFiA 2 can measure the local noise level in a running
  window and divide the data by it, so that a constant threshold can then be
  applied for source finding.
* Sect. 5: the speed test enables this local noise scaling with a spatial and
  spectral window of 31 pixels / channels, before S+C.
* Sect. 4.1: the noise is estimated robustly from the median absolute
  deviation (the S+C noise statistic, ``sc_oracle.noise``).

The paper gives no more than that; these readings fill the gaps (each is
listed with its reason in the design notes):

1. Cells. The cube is cut into cells of gx x gy x gz voxels (the last cell
   along an axis may be shorter). A grid of (1, 1, 1) is the literal running
   window: one cell, hence one window, per voxel.
2. Window. wx x wy x wz voxels (odd sizes) centred on the cell's centre
   voxel, start + (extent - 1) // 2 along each axis, clipped to the cube (no
   padding, so edge windows hold fewer voxels).
3. Noise. The S+C noise statistic of the chosen mode over the finite voxels of
   the window.
4. Division. Every voxel of the cell is divided by its window's noise. Where
   that noise is 0, or the window holds no finite voxel, the cell's voxels
   become NaN (no noise level to divide by). NaN voxels stay NaN.

Everything is float64; the cube itself is float32 data.
"""
from __future__ import annotations

import numpy as np

from . import sc_oracle


def cells(n: int, g: int) -> list[tuple[int, int, int]]:
    """(start, stop, centre) of every cell of size g along an axis of length n
    (reading 1 and the centre of reading 2)."""
    if n <= 0 or g <= 0:
        raise ValueError("axis length and cell size must be positive")
    out = []
    for start in range(0, n, g):
        stop = min(start + g, n)
        out.append((start, stop, start + (stop - start - 1) // 2))
    return out


def window_slice(centre: int, w: int, n: int) -> slice:
    """Voxels within (w - 1) / 2 of the centre, clipped to [0, n) (reading 2)."""
    if w <= 0 or w % 2 == 0:
        raise ValueError("window sizes must be odd and positive")
    r = (w - 1) // 2
    return slice(max(centre - r, 0), min(centre + r + 1, n))


def noise_grid(cube: np.ndarray, window, grid, mode: str = "mad") -> np.ndarray:
    """Noise level of every cell's window, shape (cells along z, y, x);
    NaN for a window without finite voxels (readings 1-3)."""
    c = np.asarray(cube)
    nz, ny, nx = c.shape
    wx, wy, wz = window
    gx, gy, gz = grid
    cx, cy, cz = cells(nx, gx), cells(ny, gy), cells(nz, gz)
    out = np.empty((len(cz), len(cy), len(cx)), dtype=np.float64)
    for k, (_, _, zc) in enumerate(cz):
        for j, (_, _, yc) in enumerate(cy):
            for i, (_, _, xc) in enumerate(cx):
                v = c[window_slice(zc, wz, nz), window_slice(yc, wy, ny), window_slice(xc, wx, nx)]
                v = v[np.isfinite(v)].astype(np.float64)
                out[k, j, i] = sc_oracle.noise(v, mode) if v.size else np.nan
    return out


def noise_scale(cube: np.ndarray, window, grid, mode: str = "mad") -> tuple[np.ndarray, np.ndarray]:
    """The cube divided by its local noise level (reading 4), float64, and the
    noise grid it used."""
    c = np.asarray(cube)
    nz, ny, nx = c.shape
    gx, gy, gz = grid
    sig = noise_grid(c, window, grid, mode)
    # every voxel's cell, then its window's noise
    per_voxel = sig[np.arange(nz)[:, None, None] // gz, np.arange(ny)[None, :, None] // gy,
                    np.arange(nx)[None, None, :] // gx]
    good = np.isfinite(per_voxel) & (per_voxel > 0) & np.isfinite(c)
    out = np.full(c.shape, np.nan, dtype=np.float64)
    out[good] = c[good].astype(np.float64) / per_voxel[good]
    return out, sig
