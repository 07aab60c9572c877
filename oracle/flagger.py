"""CPU oracle of SoFiA 2's auto-flagger.

TEST INFRASTRUCTURE ONLY. Nothing in the library imports this module: only
tests/ and the CPU-baseline leg of bench.py use it. It shares no code with the
CUDA path.

What the paper says (Westmeier et al. 2021, SoFiA 2, Sect. 4.1 "Input and
preconditioning"): an auto-flagging algorithm flags spatial pixels or
spectral channels whose noise deviates from the median noise across all
pixels or channels by more than a user-given multiple of the RMS, the RMS
being estimated robustly from the median absolute deviation; it targets
channels hit by radio-frequency interference and pixels with residual
continuum emission.

The paper gives no more than that; these readings fill the gaps (each is
listed with its reason in the design notes):

1. Noise of a channel: the S+C noise statistic (``sc_oracle.noise``, chosen
   mode) of the channel's finite voxels; of a spatial pixel: of the finite
   voxels of its spectrum. A channel or pixel without finite voxels has no
   noise and takes no part in what follows.
2. Across the channels (or pixels): M = median of their noises and
   R = 1.4826 * median(|noise - M|), the MAD-based RMS.
3. A channel (pixel) is flagged when |noise - M| > k * R. Flagged channels and
   pixels are blanked (NaN) in the output; with both kinds requested, both are
   measured on the input cube and blanked together.
4. The noises are rounded to float32 before steps 2 and 3 (the precision in
   which the library keeps them); M, R and the test are then exact float64.
"""
from __future__ import annotations

import numpy as np

from . import sc_oracle


def _noise_or_nan(v: np.ndarray, mode: str) -> float:
    v = v[np.isfinite(v)].astype(np.float64)
    return sc_oracle.noise(v, mode) if v.size else np.nan


def channel_noise(cube: np.ndarray, mode: str = "mad") -> np.ndarray:
    """Noise of every channel (reading 1), float32-rounded (reading 4); NaN
    for a channel without finite voxels."""
    c = np.asarray(cube)
    return np.array([_noise_or_nan(c[z].ravel(), mode) for z in range(c.shape[0])], dtype=np.float32)


def pixel_noise(cube: np.ndarray, mode: str = "mad") -> np.ndarray:
    """Noise of every spatial pixel's spectrum, shape (ny, nx), float32."""
    c = np.asarray(cube)
    nz, ny, nx = c.shape
    out = np.empty((ny, nx), dtype=np.float32)
    for y in range(ny):
        for x in range(nx):
            out[y, x] = _noise_or_nan(c[:, y, x], mode)
    return out


def flags(noise: np.ndarray, k: float) -> tuple[np.ndarray, float, float]:
    """Readings 2 and 3: the flags of a set of noise values and (M, R)."""
    v = np.asarray(noise, dtype=np.float64)
    ok = np.isfinite(v)
    if not ok.any():
        return np.zeros(v.shape, dtype=bool), np.nan, np.nan
    m = sc_oracle.median(v[ok])
    r = sc_oracle.MAD_TO_SIGMA * sc_oracle.median(np.abs(v[ok] - m))
    f = np.zeros(v.shape, dtype=bool)
    f[ok] = np.abs(v[ok] - m) > k * r
    return f, m, r


def autoflag(cube: np.ndarray, k: float, channels: bool = True, pixels: bool = True, mode: str = "mad"):
    """The blanked cube (float32) and the channel flags [nz] and pixel flags
    [ny, nx] (all False for a kind not requested)."""
    c = np.asarray(cube)
    nz, ny, nx = c.shape
    fc = flags(channel_noise(c, mode), k)[0] if channels else np.zeros(nz, dtype=bool)
    fp = flags(pixel_noise(c, mode), k)[0] if pixels else np.zeros((ny, nx), dtype=bool)
    out = c.astype(np.float32).copy()
    out[fc, :, :] = np.nan
    out[:, fp] = np.nan
    return out, fc, fp
