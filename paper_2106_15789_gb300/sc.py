"""ctypes binding of libsc.so (include/sc.h), with the C names.

Argument marshalling only: every step of smooth-and-clip runs in the CUDA
library. Device arrays are torch CUDA tensors (contiguous); the stream is the
tensor device's current torch stream unless one is passed. Loading fails
loudly when the library has not been built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsc.so")

SC_OK = 0
SC_ERR_ARG = -1
SC_ERR_NOMEM = -2
SC_ERR_CUDA = -3
SC_ERR_ALLNAN = -4
SC_ERR_TIMEOUT = -5
SC_ERR_UNSUPPORTED = -6
SC_ERR_BUDGET = -7
SC_ERR_INTERNAL = -8

SC_NOISE_MAD = 0
SC_NOISE_STD = 1
SC_NOISE_GAUSS = 2
NOISE_MODES = {"mad": SC_NOISE_MAD, "std": SC_NOISE_STD, "gauss": SC_NOISE_GAUSS}

SC_FLAG_ACCUMULATE = 0x1
SC_FLAG_GENERIC = 0x2
SC_FLAG_NO_FAST_SELECT = 0x4
SC_FLAG_GRAPH = 0x8
SC_FLAG_NO_SHARE = 0x10
SC_FLAG_SAMPLED_GAUSS = 0x20
SC_FLAG_HALF_DIRECT = 0x40
SC_AUTOFLAG_CHANNELS, SC_AUTOFLAG_PIXELS = 0x1, 0x2
# sc_smooth kernel variants (flags |= variant << 16)
SC_VARIANT_WS, SC_VARIANT_TILE, SC_VARIANT_GENERIC, SC_VARIANT_Z8, SC_VARIANT_Z4, SC_VARIANT_WS16, SC_VARIANT_Z4_512, \
    SC_VARIANT_Z8_512 = range(1, 9)


def SC_SMOOTH_VARIANT(v: int) -> int:
    return (int(v) & 0xFF) << 16
SC_STORE_F32, SC_STORE_BF16, SC_STORE_FP16 = 0, 1, 2

SC_WARN_ZERO_SIGMA = 0x1
SC_WARN_FULL_SELECT = 0x2
SC_WARN_FULL_CLIP = 0x4
SC_WARN_RANGE = 0x8
SC_WARN_GAUSS_FALLBACK = 0x10

SC_MAX_KERNELS = 64

# smoothing kernel a pair ran on (stats()["smooth_kernel_pair"])
SC_KERNEL_NONE, SC_KERNEL_IDENTITY, SC_KERNEL_Z, SC_KERNEL_WS32, SC_KERNEL_WS16, SC_KERNEL_TILE, SC_KERNEL_GENERIC, \
    SC_KERNEL_SHARED, SC_KERNEL_FIR = range(9)


class sc_kernel(C.Structure):
    _fields_ = [("fwhm_spatial_px", C.c_float), ("boxcar_chan", C.c_int32)]


class sc_stats(C.Structure):
    _fields_ = [("launches", C.c_uint64), ("runs", C.c_uint64), ("warnings", C.c_uint32), ("half_path", C.c_uint32),
                ("ms_smooth", C.c_double), ("ms_select", C.c_double), ("ms_clip", C.c_double),
                ("smooth_launches", C.c_uint64), ("smooth_voxels", C.c_uint64),
                ("ms_smooth_pair", C.c_double * SC_MAX_KERNELS), ("smooth_launches_pair", C.c_uint64 * SC_MAX_KERNELS),
                ("smooth_kernel_pair", C.c_int32 * SC_MAX_KERNELS), ("ms_noise_window", C.c_double),
                ("ms_noise_apply", C.c_double), ("ms_gauss_hist", C.c_double), ("ms_gauss_fit", C.c_double),
                ("gauss_hist_values", C.c_uint64), ("ms_share_prep", C.c_double)]


class ScError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = f"{what}: {sc_strerror(code)} ({code})" if what else f"{sc_strerror(code)} ({code})"
        if code == SC_ERR_CUDA:
            msg += f": {sc_last_cuda_error()}"
        super().__init__(msg)


def sc_last_cuda_error() -> str:
    return lib().sc_last_cuda_error().decode()


_lib = None

_P = C.c_void_p
_SIGS = {
    "sc_create": (C.c_int, [C.POINTER(_P), C.c_int, C.c_size_t]),
    "sc_destroy": (None, [_P]),
    "sc_strerror": (C.c_char_p, [C.c_int]),
    "sc_last_cuda_error": (C.c_char_p, []),
    "sc_cascade_widths": (C.c_int, [C.c_float, C.POINTER(C.c_int32)]),
    "sc_gauss_taps": (C.c_int, [C.c_float, C.POINTER(C.c_int32), C.c_int]),
    "sc_run": (C.c_int, [_P, _P, C.POINTER(C.c_int64), C.POINTER(sc_kernel), C.c_int, C.c_float, C.c_int, C.c_float,
                         _P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_uint32, _P]),
    "sc_run_host_many": (C.c_int, [_P, C.c_int, C.POINTER(_P), C.c_int, C.POINTER(_P), C.POINTER(C.c_int64),
                                   C.POINTER(sc_kernel), C.c_int, C.c_float, C.c_int, C.c_float, C.POINTER(_P),
                                   C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_uint32, _P]),
    "sc_run_host": (C.c_int, [_P, _P, C.POINTER(C.c_int64), C.POINTER(sc_kernel), C.c_int, C.c_float, C.c_int,
                              C.c_float, _P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_uint32, _P]),
    "sc_run_batch": (C.c_int, [_P, C.c_int, C.POINTER(_P), C.POINTER(C.c_int64), C.POINTER(sc_kernel), C.c_int,
                               C.c_float, C.c_int, C.c_float, C.POINTER(_P), C.POINTER(C.c_double),
                               C.POINTER(C.c_double), C.c_uint32, _P]),
    "sc_autotune": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(sc_kernel), C.c_int, _P]),
    "sc_set_budget": (C.c_int, [_P, C.c_uint64]),
    "sc_submit": (C.c_int, [_P, _P, C.c_int, _P, C.POINTER(C.c_int64), C.POINTER(sc_kernel), C.c_int, C.c_float, C.c_int,
                            C.c_float, _P, C.c_uint32, C.POINTER(C.c_int64), _P]),
    "sc_poll": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int), C.POINTER(C.c_double),
                          C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "sc_run_half": (C.c_int, [_P, _P, C.c_int, _P, C.POINTER(C.c_int64), C.POINTER(sc_kernel), C.c_int, C.c_float,
                              C.c_int, C.c_float, _P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_uint32, _P]),
    "sc_smooth": (C.c_int, [_P, _P, C.POINTER(C.c_int64), sc_kernel, _P, C.c_float, _P, C.c_uint32, _P]),
    "sc_noise": (C.c_int, [_P, _P, C.c_int64, C.c_int, C.POINTER(C.c_double), C.c_uint32, _P]),
    "sc_copy_sigmas": (C.c_int, [_P, _P, _P, C.c_int, _P]),
    "sc_set_share_limit": (C.c_int, [_P, C.c_uint64]),
    "sc_test_skip_handoff": (C.c_int, [_P, C.c_int]),
    "sc_copy_smoothed": (C.c_int, [_P, _P, C.c_int64, _P]),
    "sc_noise_static": (C.c_int, [_P, C.c_int64, C.c_int, C.POINTER(C.c_double), _P]),
    "sc_noise_scale": (C.c_int, [_P, _P, C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.c_int,
                                 _P, C.POINTER(C.c_double), C.c_uint32, _P]),
    "sc_autoflag": (C.c_int, [_P, _P, C.POINTER(C.c_int64), C.c_double, C.c_uint32, C.c_int, _P, _P, _P, _P, _P,
                              C.POINTER(C.c_int64), C.c_uint32, _P]),
    "sc_link": (C.c_int, [_P, _P, C.POINTER(C.c_int64), C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _P,
                          C.POINTER(C.c_int64), _P, C.c_int64, C.c_uint32, _P]),
    "sc_set_profiling": (C.c_int, [_P, C.c_int]),
    "sc_get_stats": (C.c_int, [_P, C.POINTER(sc_stats), C.c_int]),
}


def lib() -> C.CDLL:
    """Load libsc.so (built in-tree by paper_2106_15789_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def sc_strerror(code: int) -> str:
    return lib().sc_strerror(int(code)).decode()


def _check(code: int, what: str) -> int:
    if code != SC_OK:
        raise ScError(code, what)
    return code


def _kernels(kernels) -> tuple:
    arr = (sc_kernel * len(kernels))()
    for i, (fs, wz) in enumerate(kernels):
        arr[i].fwhm_spatial_px = float(fs)
        arr[i].boxcar_chan = int(wz)
    return arr, len(kernels)


def _dims(shape) -> C.Array:
    nz, ny, nx = shape
    return (C.c_int64 * 3)(nx, ny, nz)


def _stream(t: torch.Tensor, stream) -> C.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream(t.device)
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dev(t: torch.Tensor, dtype, name: str) -> None:
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor of {dtype}")


def sc_cascade_widths(fwhm_px: float) -> tuple:
    w = (C.c_int32 * 3)()
    _check(lib().sc_cascade_widths(float(fwhm_px), w), "sc_cascade_widths")
    return tuple(int(x) for x in w)


def sc_gauss_taps(fwhm_px: float, max_taps: int = 8193) -> tuple:
    t = (C.c_int32 * max_taps)()
    n = lib().sc_gauss_taps(float(fwhm_px), t, int(max_taps))
    _check(min(n, 0), "sc_gauss_taps")
    return tuple(int(x) for x in t[:n])


def sc_create(device: int, max_voxels: int) -> C.c_void_p:
    h = C.c_void_p()
    _check(lib().sc_create(C.byref(h), int(device), int(max_voxels)), "sc_create")
    return h


def sc_destroy(ctx) -> None:
    if ctx:
        lib().sc_destroy(ctx)


def sc_run(ctx, cube: torch.Tensor, kernels, threshold: float, noise_mode="mad", replacement: float = 2.0,
           mask: torch.Tensor | None = None, flags: int = 0, stream=None, want_sigma: bool = True):
    """S+C on a CUDA cube of shape (nz, ny, nx). Returns (mask uint8, sigmas, sigma0)."""
    _dev(cube, torch.float32, "cube")
    if mask is None:
        mask = torch.empty(cube.shape, dtype=torch.uint8, device=cube.device)
    _dev(mask, torch.uint8, "mask")
    kk, nk = _kernels(kernels)
    mode = NOISE_MODES.get(noise_mode, noise_mode)
    sig = (C.c_double * nk)() if want_sigma else None
    sig0 = (C.c_double * 1)() if want_sigma else None
    code = lib().sc_run(ctx, C.c_void_p(cube.data_ptr()), _dims(cube.shape), kk, nk, float(threshold), int(mode),
                        float(replacement), C.c_void_p(mask.data_ptr()), sig, sig0, int(flags),
                        _stream(cube, stream))
    _check(code, "sc_run")
    if not want_sigma:
        return mask, None, None
    return mask, [float(x) for x in sig], float(sig0[0])


def sc_run_batch(ctx, cubes, kernels, threshold: float, noise_mode="mad", replacement: float = 2.0, masks=None,
                 flags: int = 0, stream=None, want_sigma: bool = True):
    """S+C over a list of CUDA cubes (each (nz, ny, nx) float32). Returns
    (masks, sigmas [n_cubes][n_kernels], sigma0s [n_cubes])."""
    n = len(cubes)
    if n < 1:
        raise ScError(SC_ERR_ARG, "sc_run_batch: no cubes")
    for c in cubes:
        _dev(c, torch.float32, "cube")
    if masks is None:
        masks = [torch.empty(c.shape, dtype=torch.uint8, device=c.device) for c in cubes]
    for m in masks:
        _dev(m, torch.uint8, "mask")
    kk, nk = _kernels(kernels)
    cp = (_P * n)(*[C.c_void_p(c.data_ptr()) for c in cubes])
    mp = (_P * n)(*[C.c_void_p(m.data_ptr()) for m in masks])
    dims = (C.c_int64 * (3 * n))()
    for i, c in enumerate(cubes):
        nz, ny, nx = c.shape
        dims[3 * i], dims[3 * i + 1], dims[3 * i + 2] = nx, ny, nz
    sig = (C.c_double * (n * nk))() if want_sigma else None
    sig0 = (C.c_double * n)() if want_sigma else None
    mode = NOISE_MODES.get(noise_mode, noise_mode)
    code = lib().sc_run_batch(ctx, n, cp, dims, kk, nk, float(threshold), int(mode), float(replacement), mp, sig, sig0,
                              int(flags), _stream(cubes[0], stream))
    _check(code, "sc_run_batch")
    if not want_sigma:
        return masks, None, None
    return masks, [[float(sig[i * nk + k]) for k in range(nk)] for i in range(n)], [float(x) for x in sig0]


def sc_run_half(ctx, cube16: torch.Tensor, bf16: bool, chan_scale: torch.Tensor, kernels, threshold: float,
                noise_mode="mad", replacement: float = 2.0, mask: torch.Tensor | None = None, flags: int = 0,
                stream=None, want_sigma: bool = True):
    """S+C on a CUDA cube of 16-bit patterns (torch.int16 / uint16 storage of
    BF16 or FP16 values, shape (nz, ny, nx)) with float32 per-channel scales
    chan_scale [nz]. Returns (mask uint8, sigmas, sigma0)."""
    if not isinstance(cube16, torch.Tensor) or not cube16.is_cuda or cube16.element_size() != 2 or \
            cube16.is_floating_point() or not cube16.is_contiguous():
        raise ScError(SC_ERR_ARG, "cube16 must be a contiguous CUDA tensor of 16-bit integers (bit patterns)")
    _dev(chan_scale, torch.float32, "chan_scale")
    if chan_scale.numel() != cube16.shape[0]:
        raise ScError(SC_ERR_ARG, "chan_scale needs one value per channel")
    if mask is None:
        mask = torch.empty(cube16.shape, dtype=torch.uint8, device=cube16.device)
    _dev(mask, torch.uint8, "mask")
    kk, nk = _kernels(kernels)
    mode = NOISE_MODES.get(noise_mode, noise_mode)
    sig = (C.c_double * nk)() if want_sigma else None
    sig0 = (C.c_double * 1)() if want_sigma else None
    code = lib().sc_run_half(ctx, C.c_void_p(cube16.data_ptr()), 1 if bf16 else 0, C.c_void_p(chan_scale.data_ptr()),
                             _dims(cube16.shape), kk, nk, float(threshold), int(mode), float(replacement),
                             C.c_void_p(mask.data_ptr()), sig, sig0, int(flags), _stream(cube16, stream))
    _check(code, "sc_run_half")
    if not want_sigma:
        return mask, None, None
    return mask, [float(x) for x in sig], float(sig0[0])


def sc_set_budget(ctx, nbytes: int) -> None:
    _check(lib().sc_set_budget(ctx, int(nbytes)), "sc_set_budget")


def sc_submit(ctx, cube: torch.Tensor, kernels, threshold: float, noise_mode="mad", replacement: float = 2.0,
              mask: torch.Tensor | None = None, storage: int = SC_STORE_F32, chan_scale: torch.Tensor | None = None,
              flags: int = 0, stream=None):
    """Enqueue S+C of one CUDA cube (float32, or 16-bit bit patterns with
    chan_scale for SC_STORE_BF16 / SC_STORE_FP16). Returns (job_id, mask); the
    caller keeps cube, chan_scale and mask alive until sc_poll returns the job.
    Raises ScError with code SC_ERR_BUDGET when the job is not admitted."""
    if storage == SC_STORE_F32:
        _dev(cube, torch.float32, "cube")
        sp = None
    else:
        if not (isinstance(cube, torch.Tensor) and cube.is_cuda and cube.element_size() == 2 and
                not cube.is_floating_point() and cube.is_contiguous()):
            raise ScError(SC_ERR_ARG, "cube must hold 16-bit bit patterns")
        _dev(chan_scale, torch.float32, "chan_scale")
        sp = C.c_void_p(chan_scale.data_ptr())
    if mask is None:
        mask = torch.empty(cube.shape, dtype=torch.uint8, device=cube.device)
    _dev(mask, torch.uint8, "mask")
    kk, nk = _kernels(kernels)
    jid = C.c_int64(0)
    code = lib().sc_submit(ctx, C.c_void_p(cube.data_ptr()), int(storage), sp, _dims(cube.shape), kk, nk,
                           float(threshold), int(NOISE_MODES.get(noise_mode, noise_mode)), float(replacement),
                           C.c_void_p(mask.data_ptr()), int(flags), C.byref(jid), _stream(cube, stream))
    _check(code, "sc_submit")
    return int(jid.value), mask


def sc_poll(ctx, n_kernels: int, wait: bool = False):
    """One finished job as (job_id, status, latency_s, sigmas, sigma0), or None."""
    jid, st, lat = C.c_int64(0), C.c_int(0), C.c_double(0.0)
    sig, sig0 = (C.c_double * max(1, n_kernels))(), C.c_double(0.0)
    code = lib().sc_poll(ctx, 1 if wait else 0, C.byref(jid), C.byref(st), C.byref(lat), sig, C.byref(sig0))
    if code < 0:
        _check(code, "sc_poll")
    if code == 0:
        return None
    return int(jid.value), int(st.value), float(lat.value), [float(sig[k]) for k in range(n_kernels)], float(sig0.value)


def sc_autotune(ctx, shape, kernels, device: int = 0, stream=None) -> None:
    """Time the smoothing variants for cubes of this (nz, ny, nx) shape and keep
    the fastest per kernel pair in the context (synchronises)."""
    kk, nk = _kernels(kernels)
    if stream is None:
        stream = torch.cuda.current_stream(device)
    s = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib().sc_autotune(ctx, _dims(shape), kk, nk, s), "sc_autotune")


def sc_run_host(ctx, cube_host: torch.Tensor, kernels, threshold: float, noise_mode="mad", replacement: float = 2.0,
                mask_host: torch.Tensor | None = None, flags: int = 0, stream=None, device: int = 0):
    """S+C on a host (CPU) cube; copies in and out are part of the call."""
    if cube_host.device.type != "cpu" or cube_host.dtype != torch.float32 or not cube_host.is_contiguous():
        raise ValueError("cube_host must be a contiguous CPU float32 tensor")
    if mask_host is None:
        mask_host = torch.empty(cube_host.shape, dtype=torch.uint8)
    kk, nk = _kernels(kernels)
    mode = NOISE_MODES.get(noise_mode, noise_mode)
    sig = (C.c_double * nk)()
    sig0 = (C.c_double * 1)()
    if stream is None:
        stream = torch.cuda.current_stream(device)
    code = lib().sc_run_host(ctx, C.c_void_p(cube_host.data_ptr()), _dims(cube_host.shape), kk, nk, float(threshold),
                             int(mode), float(replacement), C.c_void_p(mask_host.data_ptr()), sig, sig0, int(flags),
                             C.c_void_p(stream.cuda_stream))
    _check(code, "sc_run_host")
    return mask_host, [float(x) for x in sig], float(sig0[0])


def sc_run_host_many(ctx, cubes_host, kernels, threshold: float, noise_mode="mad", replacement: float = 2.0,
                     masks_host=None, storage: int = SC_STORE_F32, chan_scales_host=None, flags: int = 0,
                     stream=None, device: int = 0):
    """S+C on a sequence of same-shape host (CPU) cubes with the copies
    overlapped (cube i + 1 in and mask i - 1 out while cube i runs). cubes_host:
    contiguous CPU tensors (float32, or int16/uint16 bit patterns for 16-bit
    storage, then with chan_scales_host: float32 [nz] CPU tensors). Returns
    (masks, sigmas [n][n_kernels], sigma0s [n]); pinned tensors copy fastest."""
    n = len(cubes_host)
    if n < 1:
        raise ValueError("at least one cube")
    shape = tuple(cubes_host[0].shape)
    for i, cb in enumerate(cubes_host):
        want = 4 if storage == SC_STORE_F32 else 2
        if cb.device.type != "cpu" or not cb.is_contiguous() or tuple(cb.shape) != shape or cb.element_size() != want:
            raise ValueError(f"cube {i}: a contiguous CPU tensor of the first cube's shape and {want}-byte values")
    if masks_host is None:
        masks_host = [torch.empty(shape, dtype=torch.uint8) for _ in range(n)]
    if storage != SC_STORE_F32:
        if chan_scales_host is None or len(chan_scales_host) != n:
            raise ValueError("16-bit storage needs a scale tensor per cube")
        sc_arr = (_P * n)(*[C.c_void_p(t.data_ptr()) for t in chan_scales_host])
    else:
        sc_arr = None
    kk, nk = _kernels(kernels)
    mode = NOISE_MODES.get(noise_mode, noise_mode)
    sig = (C.c_double * (n * nk))()
    sig0 = (C.c_double * n)()
    if stream is None:
        stream = torch.cuda.current_stream(device)
    cubes = (_P * n)(*[C.c_void_p(t.data_ptr()) for t in cubes_host])
    masks = (_P * n)(*[C.c_void_p(t.data_ptr()) for t in masks_host])
    code = lib().sc_run_host_many(ctx, n, cubes, int(storage), sc_arr, _dims(shape), kk, nk, float(threshold),
                                  int(mode), float(replacement), masks, sig, sig0, int(flags),
                                  C.c_void_p(stream.cuda_stream))
    _check(code, "sc_run_host_many")
    return masks_host, [[float(sig[i * nk + k]) for k in range(nk)] for i in range(n)], [float(x) for x in sig0]


def sc_smooth(ctx, cube: torch.Tensor, kernel, mask: torch.Tensor | None = None, replacement_value: float = 0.0,
              out: torch.Tensor | None = None, flags: int = 0, stream=None) -> torch.Tensor:
    """Smoothed cube S of one (spatial FWHM, spectral width) pair."""
    _dev(cube, torch.float32, "cube")
    if out is None:
        out = torch.empty_like(cube)
    _dev(out, torch.float32, "out")
    if mask is not None:
        _dev(mask, torch.uint8, "mask")
    k = sc_kernel(float(kernel[0]), int(kernel[1]))
    code = lib().sc_smooth(ctx, C.c_void_p(cube.data_ptr()), _dims(cube.shape), k,
                           C.c_void_p(mask.data_ptr()) if mask is not None else None, float(replacement_value),
                           C.c_void_p(out.data_ptr()), int(flags), _stream(cube, stream))
    _check(code, "sc_smooth")
    return out


def sc_copy_sigmas(ctx, sigma: torch.Tensor | None, sigma0: torch.Tensor | None, n_kernels: int, stream=None) -> None:
    """Enqueue copies of the latest run's float32 sigmas into sigma
    [n_kernels] and sigma0 [1] (CUDA or pinned host float32 tensors, or None);
    nothing synchronises."""
    ref = None
    for t, n, name in ((sigma, n_kernels, "sigma"), (sigma0, 1, "sigma0")):
        if t is None:
            continue
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float32 or not t.is_contiguous() or t.numel() < n \
                or not (t.is_cuda or t.is_pinned()):
            raise ValueError(f"{name} must be a contiguous CUDA or pinned float32 tensor of at least {n} values")
        ref = t if t.is_cuda else ref
    if stream is None:
        stream = torch.cuda.current_stream(ref.device if ref is not None else None)
    s = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
    _check(lib().sc_copy_sigmas(ctx, ptr(sigma), ptr(sigma0), int(n_kernels), s), "sc_copy_sigmas")


def sc_noise(ctx, data: torch.Tensor, noise_mode="mad", flags: int = 0, stream=None) -> float:
    """Noise level of the finite values of a CUDA float32 tensor."""
    _dev(data, torch.float32, "data")
    out = C.c_double()
    mode = NOISE_MODES.get(noise_mode, noise_mode)
    code = lib().sc_noise(ctx, C.c_void_p(data.data_ptr()), int(data.numel()), int(mode), C.byref(out), int(flags),
                          _stream(data, stream))
    _check(code, "sc_noise")
    return out.value


def sc_noise_static(data: torch.Tensor, noise_mode="mad", stream=None) -> float:
    """Noise level without a context or any allocation (scratch in a static
    device array; at most 4 Mi values; calls must not overlap on the GPU)."""
    _dev(data, torch.float32, "data")
    out = C.c_double()
    mode = NOISE_MODES.get(noise_mode, noise_mode)
    with torch.cuda.device(data.device):
        code = lib().sc_noise_static(C.c_void_p(data.data_ptr()), int(data.numel()), int(mode), C.byref(out),
                                     _stream(data, stream))
    _check(code, "sc_noise_static")
    return out.value


def sc_noise_scale(ctx, cube: torch.Tensor, window=(31, 31, 31), grid=(16, 16, 16), noise_mode="mad",
                   out: torch.Tensor | None = None, want_sigma: bool = False, stream=None):
    """Local noise normalisation of a CUDA cube (nz, ny, nx); window and grid
    are (x, y, z). Returns (normalised cube, per-cell noise as a numpy array
    of shape (cells z, y, x), or None)."""
    import numpy as np

    _dev(cube, torch.float32, "cube")
    if out is None:
        out = torch.empty_like(cube)
    _dev(out, torch.float32, "out")
    if out.shape != cube.shape:
        raise ValueError("out must have the cube's shape")
    nz, ny, nx = cube.shape
    gx, gy, gz = (int(v) for v in grid)
    sig = None
    if want_sigma and min(gx, gy, gz) > 0:
        sig = np.empty((-(-nz // gz), -(-ny // gy), -(-nx // gx)), dtype=np.float64)
    mode = NOISE_MODES.get(noise_mode, noise_mode)
    code = lib().sc_noise_scale(ctx, C.c_void_p(cube.data_ptr()), _dims(cube.shape),
                                (C.c_int32 * 3)(*(int(v) for v in window)), (C.c_int32 * 3)(gx, gy, gz), int(mode),
                                C.c_void_p(out.data_ptr()),
                                sig.ctypes.data_as(C.POINTER(C.c_double)) if sig is not None else None, 0,
                                _stream(cube, stream))
    _check(code, "sc_noise_scale")
    return out, sig


def sc_link(ctx, mask: torch.Tensor, r_xy: int = 2, r_z: int = 2, min_xy: int = 1, min_z: int = 1, max_xy: int = 0,
            max_z: int = 0, labels: torch.Tensor | None = None, extents_cap: int | None = None, stream=None):
    """Friends-of-friends detections of a CUDA uint8 mask (nz, ny, nx) with
    size filters. Returns (int32 labels, n, extents as a numpy int32 array
    [min(n, extents_cap)][7]: x_min, x_max, y_min, y_max, z_min, z_max, count)."""
    import numpy as np

    _dev(mask, torch.uint8, "mask")
    if labels is None:
        labels = torch.empty(mask.shape, dtype=torch.int32, device=mask.device)
    _dev(labels, torch.int32, "labels")
    if labels.shape != mask.shape:
        raise ValueError("labels must have the mask's shape")
    cap = (1 << 20) if extents_cap is None else max(0, int(extents_cap))
    ext = np.zeros((cap, 7), dtype=np.int32)
    n = C.c_int64()
    code = lib().sc_link(ctx, C.c_void_p(mask.data_ptr()), _dims(mask.shape), int(r_xy), int(r_z), int(min_xy),
                         int(min_z), int(max_xy), int(max_z), C.c_void_p(labels.data_ptr()), C.byref(n),
                         ext.ctypes.data_as(C.c_void_p) if cap > 0 else None, cap, 0, _stream(mask, stream))
    _check(code, "sc_link")
    return labels, int(n.value), ext[:min(int(n.value), cap)]


def sc_autoflag(ctx, cube: torch.Tensor, k: float, channels: bool = True, pixels: bool = True, noise_mode="mad",
                out: torch.Tensor | None = None, stream=None):
    """Auto-flagging of a CUDA cube (nz, ny, nx). Returns (blanked cube,
    channel flags [nz] bool, pixel flags [ny, nx] bool, channel noises [nz]
    float32, pixel noises [ny, nx] float32) as numpy arrays besides the cube."""
    import numpy as np

    _dev(cube, torch.float32, "cube")
    if out is None:
        out = torch.empty_like(cube)
    _dev(out, torch.float32, "out")
    nz, ny, nx = cube.shape
    fc, fp = np.zeros(nz, dtype=np.uint8), np.zeros((ny, nx), dtype=np.uint8)
    cn, pn = np.full(nz, np.nan, dtype=np.float32), np.full((ny, nx), np.nan, dtype=np.float32)
    what = (SC_AUTOFLAG_CHANNELS if channels else 0) | (SC_AUTOFLAG_PIXELS if pixels else 0)
    mode = NOISE_MODES.get(noise_mode, noise_mode)
    ptr = lambda a: a.ctypes.data_as(C.c_void_p)
    code = lib().sc_autoflag(ctx, C.c_void_p(cube.data_ptr()), _dims(cube.shape), float(k), int(what), int(mode),
                             C.c_void_p(out.data_ptr()), ptr(fc), ptr(fp), ptr(cn) if channels else None,
                             ptr(pn) if pixels else None, None, 0, _stream(cube, stream))
    _check(code, "sc_autoflag")
    return out, fc.astype(bool), fp.astype(bool), cn, pn


def sc_copy_smoothed(ctx, shape, device: int = 0, stream=None) -> torch.Tensor:
    """The smoothed cube of the last pair of the latest run, as a new device tensor."""
    n = 1
    for d in shape:
        n *= int(d)
    out = torch.empty(tuple(shape), dtype=torch.float32, device=f"cuda:{device}")
    _check(lib().sc_copy_smoothed(ctx, C.c_void_p(out.data_ptr()), n, _stream(out, stream)), "sc_copy_smoothed")
    return out


def sc_set_share_limit(ctx, max_entries: int) -> None:
    _check(lib().sc_set_share_limit(ctx, int(max_entries)), "sc_set_share_limit")


def sc_set_profiling(ctx, on: bool) -> None:
    _check(lib().sc_set_profiling(ctx, 1 if on else 0), "sc_set_profiling")


def sc_get_stats(ctx, reset: bool = False) -> dict:
    st = sc_stats()
    _check(lib().sc_get_stats(ctx, C.byref(st), 1 if reset else 0), "sc_get_stats")
    out = {}
    for name, _ in sc_stats._fields_:
        v = getattr(st, name)
        out[name] = list(v) if name.endswith("_pair") else v
    return out


class Context:
    """Owns one sc_ctx (device workspace for cubes of up to max_voxels voxels)."""

    def __init__(self, device: int = 0, max_voxels: int = 1 << 20):
        self.device = device
        self.max_voxels = int(max_voxels)
        self.handle = sc_create(device, self.max_voxels)

    def close(self) -> None:
        if self.handle:
            sc_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, cube, kernels, threshold, noise_mode="mad", replacement=2.0, mask=None, flags=0, stream=None,
            want_sigma=True):
        return sc_run(self.handle, cube, kernels, threshold, noise_mode, replacement, mask, flags, stream, want_sigma)

    def run_batch(self, cubes, kernels, threshold, noise_mode="mad", replacement=2.0, masks=None, flags=0, stream=None,
                  want_sigma=True):
        return sc_run_batch(self.handle, cubes, kernels, threshold, noise_mode, replacement, masks, flags, stream,
                            want_sigma)

    def run_host_many(self, cubes_host, kernels, threshold, noise_mode="mad", replacement=2.0, masks_host=None,
                      storage=SC_STORE_F32, chan_scales_host=None, flags=0, stream=None):
        return sc_run_host_many(self.handle, cubes_host, kernels, threshold, noise_mode, replacement, masks_host,
                                storage, chan_scales_host, flags, stream, self.device)

    def run_half(self, cube16, bf16, chan_scale, kernels, threshold, noise_mode="mad", replacement=2.0, mask=None,
                 flags=0, stream=None, want_sigma=True):
        return sc_run_half(self.handle, cube16, bf16, chan_scale, kernels, threshold, noise_mode, replacement, mask,
                           flags, stream, want_sigma)

    def set_budget(self, nbytes):
        sc_set_budget(self.handle, nbytes)

    def submit(self, cube, kernels, threshold, noise_mode="mad", replacement=2.0, mask=None, storage=SC_STORE_F32,
               chan_scale=None, flags=0, stream=None):
        return sc_submit(self.handle, cube, kernels, threshold, noise_mode, replacement, mask, storage, chan_scale,
                         flags, stream)

    def poll(self, n_kernels, wait=False):
        return sc_poll(self.handle, n_kernels, wait)

    def autotune(self, shape, kernels, stream=None):
        sc_autotune(self.handle, shape, kernels, self.device, stream)

    def run_host(self, cube_host, kernels, threshold, noise_mode="mad", replacement=2.0, mask_host=None, flags=0,
                 stream=None):
        return sc_run_host(self.handle, cube_host, kernels, threshold, noise_mode, replacement, mask_host, flags,
                           stream, self.device)

    def smooth(self, cube, kernel, mask=None, replacement_value=0.0, out=None, flags=0, stream=None):
        return sc_smooth(self.handle, cube, kernel, mask, replacement_value, out, flags, stream)

    def noise(self, data, noise_mode="mad", flags=0, stream=None):
        return sc_noise(self.handle, data, noise_mode, flags, stream)

    def noise_scale(self, cube, window=(31, 31, 31), grid=(16, 16, 16), noise_mode="mad", out=None,
                    want_sigma=False, stream=None):
        return sc_noise_scale(self.handle, cube, window, grid, noise_mode, out, want_sigma, stream)

    def autoflag(self, cube, k, channels=True, pixels=True, noise_mode="mad", out=None, stream=None):
        return sc_autoflag(self.handle, cube, k, channels, pixels, noise_mode, out, stream)

    def link(self, mask, r_xy=2, r_z=2, min_xy=1, min_z=1, max_xy=0, max_z=0, labels=None, extents_cap=None,
             stream=None):
        return sc_link(self.handle, mask, r_xy, r_z, min_xy, min_z, max_xy, max_z, labels, extents_cap, stream)

    def copy_sigmas(self, sigma, sigma0, n_kernels, stream=None):
        sc_copy_sigmas(self.handle, sigma, sigma0, n_kernels, stream)

    def copy_smoothed(self, shape, stream=None):
        return sc_copy_smoothed(self.handle, shape, self.device, stream)

    def test_skip_handoff(self, enable=True):
        _check(lib().sc_test_skip_handoff(self.handle, 1 if enable else 0), "sc_test_skip_handoff")

    def set_share_limit(self, max_entries):
        sc_set_share_limit(self.handle, max_entries)

    def set_profiling(self, on=True):
        sc_set_profiling(self.handle, on)

    def stats(self, reset=False):
        return sc_get_stats(self.handle, reset)
