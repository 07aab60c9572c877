"""Seeded synthetic H I data cubes shaped like the paper's test data.

This module only makes inputs. It holds none of the smooth-and-clip
arithmetic, and both the CUDA path and the CPU oracle read its output.

The paper measures on real cubes that are not available here: WSRT noise with
WHISP galaxies (Sect. 5), ASKAP Eridanus noise with galmod galaxies (Sect. 6)
and the Hydra pilot field (Sect. 7). What is reproduced is their shape and
statistics only:

* beam-correlated Gaussian noise: white N(0, 1) convolved in each channel with a
  sampled circular Gaussian beam (5 px FWHM, i.e. a 30" beam on 6" pixels as in
  Sect. 6), then rescaled to a measured standard deviation of 1;
* optional per-channel noise ripple sigma_c = 1 + a*sin(2*pi*c/128);
* mock galaxies as 3-D ellipsoidal Gaussians (peak S/N, major-axis FWHM,
  axis ratio U(0.3, 1), position angle U(0, pi), spectral FWHM), centred
  uniformly in the cube;
* NaN-blanked regions (a corner block or a spatial border).

Layout: a C-contiguous array of shape (nz, ny, nx), x fastest, matching the
FITS axis order (Sect. 4.1). Values are float32.

Random draws use torch generators so the same code makes small cubes on the
CPU (bit-reproducible) and WALLABY-sized cubes directly on a GPU.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

FWHM_TO_SIGMA = 1.0 / math.sqrt(8.0 * math.log(2.0))


@dataclass(frozen=True)
class CubeSpec:
    """Recipe for one synthetic cube."""

    nx: int
    ny: int
    nz: int
    seed: int
    n_gal: int = 20
    snr: tuple = (2.0, 8.0)
    snr_log: bool = False  # log-uniform instead of uniform S/N
    fwhm_xy: tuple = (2.0, 6.0)
    fwhm_z: tuple = (5.0, 30.0)
    beam_fwhm: float = 5.0
    ripple: float = 0.0
    nan_corner: tuple | None = None  # (x_end, y_end, z_end): C[:z_end, :y_end, :x_end] = NaN
    nan_border: int = 0
    name: str = field(default="cube", compare=False)


def _gauss_taps(fwhm: float) -> torch.Tensor:
    s = fwhm * FWHM_TO_SIGMA
    r = int(math.ceil(4.0 * s))
    k = torch.arange(-r, r + 1, dtype=torch.float64)
    g = torch.exp(-0.5 * (k / s) ** 2)
    return g / g.sum()


def _conv_axis(x: torch.Tensor, taps: torch.Tensor, dim: int) -> torch.Tensor:
    """Zero-padded 'same' convolution along one axis as a sum of shifted copies."""
    r = (taps.numel() - 1) // 2
    out = torch.zeros_like(x)
    n = x.shape[dim]
    for i, g in enumerate(taps.tolist()):
        d = i - r  # out[j] += g * x[j + d]
        if abs(d) >= n:
            continue
        src = x.narrow(dim, max(d, 0), n - abs(d))
        dst = out.narrow(dim, max(-d, 0), n - abs(d))
        dst.add_(src, alpha=g)
    return out


def _galaxy_params(spec: CubeSpec) -> list[dict]:
    g = torch.Generator(device="cpu").manual_seed(1_000_003 * (spec.seed + 1))
    u = torch.rand((spec.n_gal, 8), generator=g, dtype=torch.float64).tolist()
    out = []
    for r in u:
        lo, hi = spec.snr
        snr = math.exp(math.log(lo) + r[0] * (math.log(hi) - math.log(lo))) if spec.snr_log else lo + r[0] * (hi - lo)
        out.append(
            dict(
                snr=snr,
                fwhm_maj=spec.fwhm_xy[0] + r[1] * (spec.fwhm_xy[1] - spec.fwhm_xy[0]),
                axis_ratio=0.3 + 0.7 * r[2],
                pa=math.pi * r[3],
                fwhm_z=spec.fwhm_z[0] + r[4] * (spec.fwhm_z[1] - spec.fwhm_z[0]),
                x=r[5] * (spec.nx - 1),
                y=r[6] * (spec.ny - 1),
                z=r[7] * (spec.nz - 1),
            )
        )
    return out


def _add_galaxy(cube: torch.Tensor, p: dict) -> None:
    nz, ny, nx = cube.shape
    s_maj = p["fwhm_maj"] * FWHM_TO_SIGMA
    s_min = s_maj * p["axis_ratio"]
    s_z = p["fwhm_z"] * FWHM_TO_SIGMA
    rx = int(math.ceil(3.0 * s_maj))
    rz = int(math.ceil(3.0 * s_z))
    x0, x1 = max(0, int(p["x"]) - rx), min(nx, int(p["x"]) + rx + 2)
    y0, y1 = max(0, int(p["y"]) - rx), min(ny, int(p["y"]) + rx + 2)
    z0, z1 = max(0, int(p["z"]) - rz), min(nz, int(p["z"]) + rz + 2)
    dev = cube.device
    xs = torch.arange(x0, x1, device=dev, dtype=torch.float32) - p["x"]
    ys = torch.arange(y0, y1, device=dev, dtype=torch.float32) - p["y"]
    zs = torch.arange(z0, z1, device=dev, dtype=torch.float32) - p["z"]
    c, s = math.cos(p["pa"]), math.sin(p["pa"])
    u = c * xs[None, :] + s * ys[:, None]
    v = -s * xs[None, :] + c * ys[:, None]
    sky = torch.exp(-0.5 * ((u / s_maj) ** 2 + (v / s_min) ** 2))
    spec = torch.exp(-0.5 * (zs / s_z) ** 2)
    cube[z0:z1, y0:y1, x0:x1] += float(p["snr"]) * spec[:, None, None] * sky[None, :, :]


def make_cube(spec: CubeSpec, device: str | torch.device = "cpu") -> torch.Tensor:
    """Build the cube described by ``spec`` on ``device`` (float32, shape (nz, ny, nx))."""
    gen = torch.Generator(device=device).manual_seed(spec.seed)
    cube = torch.randn((spec.nz, spec.ny, spec.nx), generator=gen, device=device, dtype=torch.float32)
    if spec.beam_fwhm > 0:
        taps = _gauss_taps(spec.beam_fwhm)
        cube = _conv_axis(cube, taps, 2)
        cube = _conv_axis(cube, taps, 1)
        cube /= cube.std()
    if spec.ripple:
        c = torch.arange(spec.nz, device=device, dtype=torch.float32)
        cube *= (1.0 + spec.ripple * torch.sin(2.0 * math.pi * c / 128.0))[:, None, None]
    for p in _galaxy_params(spec):
        _add_galaxy(cube, p)
    if spec.nan_corner is not None:
        xe, ye, ze = spec.nan_corner
        cube[:ze, :ye, :xe] = float("nan")
    b = spec.nan_border
    if b > 0:
        cube[:, :b, :] = float("nan")
        cube[:, -b:, :] = float("nan")
        cube[:, :, :b] = float("nan")
        cube[:, :, -b:] = float("nan")
    return cube.contiguous()


# ---------------------------------------------------------------------------
# Workloads. Kernel pairs are (spatial FWHM in px, spectral boxcar in channels),
# spatial outer and spectral inner, ascending.

def kernel_list(spatial, spectral) -> list[tuple[float, int]]:
    return [(float(s), int(w)) for s in spatial for w in spectral]


KERNELS_12 = kernel_list((0, 3, 6), (0, 3, 7, 15))
KERNELS_20 = kernel_list((0, 3, 6, 10), (0, 3, 7, 15, 31))
KERNELS_PAPER = kernel_list((0, 5, 10), (0, 3, 7, 15))

# 64x64x128, 20 galaxies with peak S/N 2-8, 5 % NaN corner block.
SMALL = CubeSpec(nx=64, ny=64, nz=128, seed=0, n_gal=20, snr=(2.0, 8.0), fwhm_xy=(2.0, 6.0),
                 fwhm_z=(5.0, 30.0), nan_corner=(24, 24, 47), name="small-64x64x128")

# WALLABY-shaped 1200x1200x1024 (~5.9 GB), 3000 galaxies, log-uniform S/N 3-50,
# 10 % channel ripple, 16 px NaN border.
WALLABY = CubeSpec(nx=1200, ny=1200, nz=1024, seed=2, n_gal=3000, snr=(3.0, 50.0), snr_log=True,
                   fwhm_xy=(2.0, 15.0), fwhm_z=(5.0, 60.0), ripple=0.1, nan_border=16,
                   name="wallaby-1200x1200x1024")

SC_THRESHOLD = 3.5
SC_REPLACEMENT = 2.0


def batch_specs(n_cubes: int = 64, first_seed: int = 0) -> list[CubeSpec]:
    """Uneven sub-cubes: nx, ny log-uniform in [128, 512], nz in [256, 1024];
    noise and galaxies as the small cube, one seed per cube."""
    out = []
    for i in range(first_seed, first_seed + n_cubes):
        g = torch.Generator(device="cpu").manual_seed(7_919 * (i + 1))
        r = torch.rand(3, generator=g, dtype=torch.float64).tolist()
        nx = int(round(math.exp(math.log(128) + r[0] * (math.log(512) - math.log(128)))))
        ny = int(round(math.exp(math.log(128) + r[1] * (math.log(512) - math.log(128)))))
        nz = int(round(math.exp(math.log(256) + r[2] * (math.log(1024) - math.log(256)))))
        out.append(CubeSpec(nx=nx, ny=ny, nz=nz, seed=i, n_gal=20, snr=(2.0, 8.0), fwhm_xy=(2.0, 6.0),
                            fwhm_z=(5.0, 30.0), name=f"sub-{i}"))
    return out


def encode_half(cube: torch.Tensor, bf16: bool) -> tuple[torch.Tensor, torch.Tensor]:
    """A cube's 16-bit storage form with one float32 scale per channel: BF16
    with scale = max|C_c| / 256, or FP16 with scale = max|C_c| / 2^14 (finite
    values; 1 for an all-zero or all-NaN channel). Returns (int16 bit patterns,
    float32 scales [nz]) on the cube's device."""
    a = torch.nan_to_num(cube.abs(), nan=0.0, posinf=0.0, neginf=0.0)
    mx = a.reshape(cube.shape[0], -1).amax(dim=1)
    scale = torch.where(mx > 0, mx / (256.0 if bf16 else 16384.0), torch.ones_like(mx)).to(torch.float32)
    x = cube / scale[:, None, None]
    half = x.to(torch.bfloat16 if bf16 else torch.float16)
    return half.view(torch.int16).contiguous(), scale.contiguous()


def decode_half(bits: np.ndarray, scale: np.ndarray, bf16: bool) -> np.ndarray:
    """float32 cube of a 16-bit storage form: float32(value) * scale[z], one
    float32 rounding (numpy, for test and benchmark references)."""
    b = np.ascontiguousarray(bits).view(np.uint16)
    v = (b.astype(np.uint32) << 16).view(np.float32) if bf16 else b.view(np.float16).astype(np.float32)
    return (v * np.asarray(scale, dtype=np.float32)[:, None, None]).astype(np.float32)


def to_numpy(cube: torch.Tensor) -> np.ndarray:
    return cube.detach().to("cpu").numpy()
