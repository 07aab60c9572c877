"""CPU FP64 oracle of the smooth-and-clip (S+C) source finder.

TEST INFRASTRUCTURE ONLY. Nothing in the library imports this module: only
tests/, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
bench.py use it. It shares no code, header, table or constant generator with
the CUDA path; the two meet only in the seeded input generator (synth/), which
holds none of the method's arithmetic.

What it computes, and where the paper says so (Westmeier et al. 2021, SoFiA 2):

* Sect. 4.2 "Source finding": S+C smooths the cube on several spatial and
  spectral scales and keeps emission above a threshold relative to the noise on
  each scale; the output is a binary mask. Both positive and negative
  excursions enter the mask (second paragraph of Sect. 4.2).
* Sect. 5: spatial kernels of 0, 5 and 10 px, spectral kernels of 0, 3, 7 and
  15 channels, threshold 3.5 times the noise "in each smoothing iteration".
* Hydra-field figure caption (Sect. 7): spatial smoothing is a Gaussian given
  by its FWHM in pixels, spectral smoothing is a boxcar of w channels.
* Sect. 6.2 "Integrated flux": at the start of each iteration, voxels already
  in the mask are set to +-n times the noise level, keeping their sign, before
  smoothing. Default n = 2.
* Sect. 4.1: the RMS is estimated robustly from the median absolute deviation.
* Sect. 5: the method holds two float32 cube copies plus an 8-bit mask.

The paper gives no formulas for S+C, so the readings below fill its gaps
(each is listed with its reason in the design notes):

1. Gaussian of FWHM f: a cascade of 3 centred boxcars (Kovesi 2010, "Fast
   almost-Gaussian filtering") with widths from :func:`cascade_widths`, applied
   along x and then y. f <= 0 means no spatial smoothing.
1b. The sampled variant (spatial="sampled"): the Gaussian itself, sampled at
   the integer offsets within +-4 sigma (sigma = f / sqrt(8 ln 2)), each sample
   expressed in units of 1/1024 of the central one and rounded to an integer
   (:func:`gauss_taps`), the kernel being these taps over their sum, applied
   along x and then y with zero padding.
2. Spectral boxcar of odd width w: mean of w channels centred on z. w <= 1
   means no spectral smoothing. Even w is rejected.
3. Edges: zero padding outside the cube, kernels not renormalised.
4. NaN voxels count as 0 inside smoothing windows; the smoothed cube is NaN
   again at every NaN input voxel; NaN voxels never enter the noise sample or
   the mask.
5. Replacement value: n * sigma_0, where sigma_0 is the noise of the raw cube
   measured once with the same noise mode. Every masked finite voxel becomes
   sign(C) * n * sigma_0 with sign(0) = +1; n <= 0 switches replacement off.
6. Kernel pairs run in the order given (default: spatial outer, spectral
   inner, ascending).
7. Noise, MAD mode: 1.4826 * median(|S - median(S)|) over the finite voxels,
   medians exact; for even counts the median is the mean of the two middle
   order statistics. STD mode: sqrt(sum((S - mean)^2) / (n - 1)).
7b. Noise, Gaussian-fit mode (the paper names no such mode; this is the
   library's own definition). With sigma_M the MAD noise of reading 7 and
   k = fl32(128 / (5 sigma_M)) bins per data unit, every finite value s goes
   to bin floor(fl32(s * k)) + 128 if that lies in [0, 256): 256 equal bins
   over about +-5 sigma_M, the index taken in float32 as the kernel takes it.
   A Gaussian A exp(-xi^2 / (2 tau^2)), centred at 0, is fitted by least
   squares to the counts at the bin centres xi_i = (i + 0.5) / 128 - 1; the
   noise is tau * 128 / k. The fit profiles A out and bisects the
   stationarity condition over tau in [0.05, 0.8] (:func:`gauss_fit`). When
   the ends of that bracket do not straddle a root the noise is sigma_M;
   when sigma_M is 0 it is 0.
8. Clip: |S| > t * sigma (strict). A pair whose sigma is 0 adds nothing.

Everything is float64; the cube itself is float32 data.
"""
from __future__ import annotations

import math

import numpy as np

MAD_TO_SIGMA = 1.4826  # the literal constant of the MAD noise estimator
N_BOXES = 3  # boxcars in the almost-Gaussian cascade


class AllNaNError(ValueError):
    """The cube has no finite voxel, so no noise level exists."""


def cascade_widths(fwhm: float, n: int = N_BOXES) -> tuple[int, ...]:
    """Odd boxcar widths whose n-fold cascade approximates a Gaussian of this FWHM.

    Kovesi (2010): with sigma = FWHM / sqrt(8 ln 2), the ideal common width is
    w = sqrt(12 sigma^2 / n + 1). Take w_l as the largest odd integer not above
    it and w_u = w_l + 2; use m passes of w_l and n - m of w_u, with m the
    integer nearest to (12 sigma^2 - n w_l^2 - 4 n w_l - 3 n) / (-4 w_l - 4),
    which makes the cascade's variance sum((w_i^2 - 1) / 12) as close to
    sigma^2 as these two widths allow. Returns () for FWHM <= 0.
    """
    if not fwhm > 0:
        return ()
    sigma = fwhm / math.sqrt(8.0 * math.log(2.0))
    w_ideal = math.sqrt(12.0 * sigma * sigma / n + 1.0)
    w_l = int(math.floor(w_ideal))
    if w_l % 2 == 0:
        w_l -= 1
    w_u = w_l + 2
    m_real = (12.0 * sigma * sigma - n * w_l * w_l - 4.0 * n * w_l - 3.0 * n) / (-4.0 * w_l - 4.0)
    m = int(math.floor(m_real + 0.5))
    m = min(max(m, 0), n)
    return tuple([w_l] * m + [w_u] * (n - m))


def box_mean(x: np.ndarray, w: int, axis: int) -> np.ndarray:
    """Centred boxcar mean of odd width w along one axis, zero outside the array.

    out[i] = (1/w) * sum_{d=-r..r} x[i + d], r = (w - 1) / 2.
    """
    if w <= 1:
        return x.copy()
    if w % 2 == 0:
        raise ValueError("boxcar width must be odd")
    r = (w - 1) // 2
    n = x.shape[axis]
    out = np.zeros_like(x)
    for d in range(-r, r + 1):
        if abs(d) >= n:
            continue
        src = [slice(None)] * x.ndim
        dst = [slice(None)] * x.ndim
        src[axis] = slice(max(d, 0), n + min(d, 0))
        dst[axis] = slice(max(-d, 0), n - max(d, 0))
        out[tuple(dst)] += x[tuple(src)]
    return out / w


def smooth(x: np.ndarray, fwhm: float, wz: int, spatial: str = "cascade") -> np.ndarray:
    """Separable 3-D smoothing of an (nz, ny, nx) float64 array with no NaNs:
    the spatial kernel along x, the same along y, then the spectral boxcar
    along z.

    spatial="cascade" (reading 1): the cube is zero-padded once, by the
    cascade's half-width h = sum((w-1)/2), and the cascade runs over the
    padded array, so the result is the convolution of the zero-padded cube
    with the composed kernel (the intermediate boxcar outputs just outside the
    cube are kept, not cut). spatial="sampled" (reading 1b): one zero-padded
    pass of the sampled Gaussian along x, then one along y.
    """
    s = np.asarray(x, dtype=np.float64)
    if spatial == "cascade":
        widths = cascade_widths(fwhm)
        h = sum((w - 1) // 2 for w in widths)
        if widths:
            s = np.pad(s, ((0, 0), (h, h), (h, h)))
            for w in widths:
                s = box_mean(s, w, axis=2)
            for w in widths:
                s = box_mean(s, w, axis=1)
            s = s[:, h:s.shape[1] - h, h:s.shape[2] - h]
    elif spatial == "sampled":
        if fwhm > 0:
            k = kernel_1d(fwhm, "sampled")
            s = fir_along(s, k, axis=2)
            s = fir_along(s, k, axis=1)
    else:
        raise ValueError(f"unknown spatial kernel {spatial!r}")
    if wz > 1:
        s = box_mean(s, wz, axis=0)
    return s


GAUSS_TAP_UNIT = 1024  # the central tap of the sampled Gaussian (reading 1b)
GAUSS_TRUNCATE = 4.0   # its support, in sigmas either side


def gauss_taps(fwhm: float) -> np.ndarray:
    """Integer taps of the sampled spatial Gaussian of this FWHM (reading 1b).

    sigma = FWHM / sqrt(8 ln 2); offsets i = -h..h with h = floor(4 sigma);
    tap i = the Gaussian's value exp(-i^2 / (2 sigma^2)) times 1024 (the
    central value's units), rounded to the nearest integer. FWHM <= 0 gives
    the single tap 1024 (no smoothing).
    """
    if not fwhm > 0:
        return np.array([GAUSS_TAP_UNIT], dtype=np.int64)
    sigma = fwhm / math.sqrt(8.0 * math.log(2.0))
    h = int(math.floor(GAUSS_TRUNCATE * sigma))
    i = np.arange(-h, h + 1, dtype=np.float64)
    return np.rint(GAUSS_TAP_UNIT * np.exp(-i * i / (2.0 * sigma * sigma))).astype(np.int64)


def fir_along(x: np.ndarray, k: np.ndarray, axis: int) -> np.ndarray:
    """Centred FIR of odd length 2h+1 along one axis, zero outside the array:
    out[i] = sum_{d=-h..h} k[d + h] * x[i + d]."""
    h = (k.size - 1) // 2
    n = x.shape[axis]
    out = np.zeros_like(x)
    for d in range(-h, h + 1):
        if abs(d) >= n:
            continue
        src = [slice(None)] * x.ndim
        dst = [slice(None)] * x.ndim
        src[axis] = slice(max(d, 0), n + min(d, 0))
        dst[axis] = slice(max(-d, 0), n - max(d, 0))
        out[tuple(dst)] += k[d + h] * x[tuple(src)]
    return out


def kernel_1d(fwhm: float, spatial: str = "cascade") -> np.ndarray:
    """The composed 1-D spatial kernel: the convolution of the cascade's boxes,
    or the sampled Gaussian's taps over their sum."""
    if spatial == "sampled":
        t = gauss_taps(fwhm).astype(np.float64)
        return t / t.sum()
    k = np.ones(1)
    for w in cascade_widths(fwhm):
        k = np.convolve(k, np.full(w, 1.0 / w))
    return k


def median(v: np.ndarray) -> float:
    """Exact median: the middle order statistic, or the mean of the two middle
    ones for an even count."""
    v = np.asarray(v, dtype=np.float64)
    n = v.size
    lo, hi = (n - 1) // 2, n // 2
    p = np.partition(v, [lo, hi])
    return 0.5 * (p[lo] + p[hi])


def noise(v: np.ndarray, mode: str = "mad") -> float:
    """Noise level of a sample of finite values."""
    v = np.asarray(v, dtype=np.float64)
    if v.size == 0:
        raise AllNaNError("no finite values")
    if mode == "mad":
        m = median(v)
        return MAD_TO_SIGMA * median(np.abs(v - m))
    if mode == "std":
        if v.size < 2:
            return 0.0
        mean = v.sum() / v.size
        return math.sqrt(float(((v - mean) ** 2).sum()) / (v.size - 1))
    if mode == "gauss":
        return gauss_noise(v)
    raise ValueError(f"unknown noise mode {mode!r}")


GAUSS_HALF_RANGE = 5.0            # the histogram spans +-5 MAD noises
GAUSS_BINS = 256
GAUSS_TAU_BRACKET = (0.05, 0.8)   # sigma / half-range searched by the fit


def gauss_scale(sigma_mad: float) -> np.float32:
    """Bins per data unit, k = fl32(128 / (5 sigma_M)) (reading 7b)."""
    return np.float32((GAUSS_BINS // 2) / (GAUSS_HALF_RANGE * sigma_mad))


def gauss_histogram(v: np.ndarray, sigma_mad: float) -> np.ndarray:
    """Counts of the 256 bins of reading 7b. v holds float32 data values."""
    k = gauss_scale(sigma_mad)
    q = np.floor(np.asarray(v, dtype=np.float32) * k)  # one float32 product, rounded once
    half = GAUSS_BINS // 2
    q = q[(q >= -half) & (q < half)]
    return np.bincount(q.astype(np.int64) + half, minlength=GAUSS_BINS).astype(np.int64)


def gauss_bin_centres() -> np.ndarray:
    """xi_i = (i + 0.5) / 128 - 1: the bin centres in units of the half-range."""
    return (np.arange(GAUSS_BINS) + 0.5) / (GAUSS_BINS // 2) - 1.0


def gauss_fit(h: np.ndarray) -> float | None:
    """tau of the least-squares Gaussian through the counts (reading 7b).

    E(A, tau) = sum_i (h_i - A g_i)^2 with g_i = exp(-xi_i^2 / (2 tau^2)). For
    a fixed tau the best A is sum(h g) / sum(g^2), and the profile E(tau) is
    stationary where
        D(tau) = sum(g^2) * sum(h xi^2 g) - sum(h g) * sum(xi^2 g^2) = 0,
    i.e. where the h g-weighted and the g^2-weighted means of xi^2 agree. D is
    positive for Gaussians much narrower than the counts and negative for much
    wider ones: bisection from the bracket's ends keeps D(lo) > 0 >= D(hi) and
    halves until the midpoint is one of the ends. None when D(0.05) <= 0 or
    D(0.8) >= 0.
    """
    x2 = gauss_bin_centres() ** 2
    h = np.asarray(h, dtype=np.float64)

    def d(tau: float) -> float:
        g = np.exp(-x2 / (2.0 * tau * tau))
        return float(np.sum(g * g) * np.sum(h * x2 * g) - np.sum(h * g) * np.sum(x2 * g * g))

    lo, hi = GAUSS_TAU_BRACKET
    if not (d(lo) > 0.0 and d(hi) < 0.0):
        return None
    while True:
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            return mid
        if d(mid) > 0.0:
            lo = mid
        else:
            hi = mid


def gauss_noise(v: np.ndarray) -> float:
    """Gaussian-fit noise of a sample of finite float32 values (reading 7b)."""
    s_mad = noise(v, "mad")
    if not s_mad > 0.0:
        return 0.0
    k = gauss_scale(s_mad)
    tau = gauss_fit(gauss_histogram(v, s_mad))
    if tau is None:
        return s_mad
    return tau * (GAUSS_BINS // 2) / float(k)


def replaced_input(c: np.ndarray, mask: np.ndarray, finite: np.ndarray, value: float) -> np.ndarray:
    """X = C with NaN set to 0 and, where the mask is set and C is finite,
    sign(C) * value (sign(0) = +1). value <= 0 leaves masked voxels alone."""
    x = np.where(finite, c, 0.0)
    if value > 0:
        sgn = np.where(c >= 0, 1.0, -1.0)
        x = np.where(mask & finite, sgn * value, x)
    return x


def smoothed(c: np.ndarray, mask: np.ndarray, fwhm: float, wz: int, value: float,
             spatial: str = "cascade") -> np.ndarray:
    """S for one kernel pair: replace, smooth, re-blank NaN input voxels."""
    c = np.asarray(c, dtype=np.float64)
    finite = np.isfinite(c)
    s = smooth(replaced_input(c, mask, finite, value), fwhm, wz, spatial)
    s[~finite] = np.nan
    return s


def sc_filter(cube: np.ndarray, kernels, threshold: float, noise_mode: str = "mad",
              replacement: float = 2.0, mask: np.ndarray | None = None, return_smoothed: bool = False,
              spatial: str = "cascade"):
    """Smooth-and-clip over a list of (spatial FWHM px, spectral width ch) pairs,
    with the spatial kernel of reading 1 (cascade) or 1b (sampled).

    Returns (mask uint8, [sigma_k], sigma_0) and, if asked, the list of smoothed
    cubes S_k.
    """
    c = np.asarray(cube, dtype=np.float64)
    finite = np.isfinite(c)
    if not finite.any():
        raise AllNaNError("cube has no finite voxel")
    for fs, wz in kernels:
        if fs < 0 or (wz > 1 and wz % 2 == 0) or wz < 0:
            raise ValueError(f"bad kernel ({fs}, {wz})")
    sigma0 = noise(c[finite], noise_mode)
    m = np.zeros(c.shape, dtype=bool) if mask is None else np.asarray(mask).astype(bool).copy()
    value = replacement * sigma0 if replacement > 0 else 0.0
    sigmas, all_s = [], []
    for fs, wz in kernels:
        s = smoothed(c, m, fs, wz, value, spatial)
        ok = np.isfinite(s)
        sk = noise(s[ok], noise_mode)
        if sk > 0:
            m |= ok & (np.abs(s) > threshold * sk)
        sigmas.append(sk)
        if return_smoothed:
            all_s.append(s)
    out = (m.astype(np.uint8), sigmas, sigma0)
    return out + (all_s,) if return_smoothed else out


def smoothed_at(x: np.ndarray, fwhm: float, wz: int, points: np.ndarray, spatial: str = "cascade") -> np.ndarray:
    """S at a few voxels by direct summation over the composed 3-D kernel.

    x is the already replaced input (NaN -> 0); points is an (m, 3) array of
    (z, y, x) indices. S(p) = sum_{i,j,l} kz[l] ky[j] kx[i] x(p + offsets),
    zero outside the cube. Used for sampled checks of cubes too large for
    :func:`smooth`.
    """
    kxy = kernel_1d(fwhm, spatial)
    kz = np.full(wz, 1.0 / wz) if wz > 1 else np.ones(1)
    h, r = (kxy.size - 1) // 2, (kz.size - 1) // 2
    nz, ny, nx = x.shape
    k3 = kz[:, None, None] * kxy[None, :, None] * kxy[None, None, :]
    out = np.empty(len(points))
    for i, (z, y, xx) in enumerate(np.asarray(points, dtype=np.int64)):
        z0, z1 = z - r, z + r + 1
        y0, y1 = y - h, y + h + 1
        x0, x1 = xx - h, xx + h + 1
        nb = np.zeros(k3.shape)
        cz0, cz1 = max(z0, 0), min(z1, nz)
        cy0, cy1 = max(y0, 0), min(y1, ny)
        cx0, cx1 = max(x0, 0), min(x1, nx)
        nb[cz0 - z0:cz1 - z0, cy0 - y0:cy1 - y0, cx0 - x0:cx1 - x0] = x[cz0:cz1, cy0:cy1, cx0:cx1]
        out[i] = float((nb * k3).sum())
    return out
