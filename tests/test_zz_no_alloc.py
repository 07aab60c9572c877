"""sc_noise_static: the noise measurement for callers that cannot allocate
device memory (memory owned by another allocator or a fixed pool, real-time
code that must not allocate while running, plug-ins handed only a stream and
buffers). It keeps its scratch in a static device array instead of a context.

Checked through the C ABI against sc_noise (the context-based entry point) at
the parity tolerance of the other tests, on two calls in a row so that the
second call starts from the first call's leftovers in the shared array. The
file is collected last: it passes alone in a fresh process and after the
other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

SIG_RTOL = 1e-6


def _static(lib, data, mode):
    out = ctypes.c_double()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = lib.sc_noise_static(ctypes.c_void_p(data.data_ptr()), int(data.numel()), mode, ctypes.byref(out), stream)
    return code, out.value


def test_static_noise_matches_sc_noise_twice():
    from paper_2106_15789_gb300 import Context, sc

    lib = sc.lib()
    rng = np.random.default_rng(2024)
    a = rng.standard_normal(3_000_001).astype(np.float32)
    a[rng.random(a.size) < 0.05] = np.nan
    b = (0.3 * rng.standard_cauchy(1_500_000) + 7.0).astype(np.float32)
    with Context(0, 1 << 22) as ctx:
        for data in (a, b):  # two calls in a row on different data
            d = torch.from_numpy(data).cuda()
            for mode, name in ((sc.SC_NOISE_MAD, "mad"), (sc.SC_NOISE_STD, "std")):
                code, got = _static(lib, d, mode)
                assert code == sc.SC_OK, sc.sc_strerror(code)
                ref = ctx.noise(d, name)
                assert abs(got - ref) <= SIG_RTOL * ref, (name, got, ref)


def test_static_noise_limits():
    from paper_2106_15789_gb300 import sc

    lib = sc.lib()
    big = torch.zeros((1 << 22) + 1, device="cuda")
    code, _ = _static(lib, big, sc.SC_NOISE_MAD)
    assert code == sc.SC_ERR_BUDGET
    nan = torch.full((1000,), float("nan"), device="cuda")
    code, _ = _static(lib, nan, sc.SC_NOISE_MAD)
    assert code == sc.SC_ERR_ALLNAN
    ok = torch.randn(1000, device="cuda")
    code, got = _static(lib, ok, sc.SC_NOISE_MAD)
    assert code == sc.SC_OK and got > 0
