"""sc_noise_static: the noise measurement for callers that cannot allocate
device memory (memory owned by another allocator or a fixed pool, real-time
code that must not allocate while running, plug-ins handed only a stream and
buffers). It keeps its scratch in a static device array instead of a context.

Checked through the C ABI against sc_noise (the context-based entry point) at
the parity tolerance of the other tests, on two calls in a row so that the
second call starts from the first call's leftovers in the shared array, and
against the FP64 oracle in every noise mode, including inputs of the maximum
size whose candidate sets overflow the array's fixed lists (rounded and
constant values), so that the full-pass plan runs. The file is collected
last: it passes alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle.sc_oracle as O
from tests.gauss_common import close_to_any, gauss_refs

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
            for mode, name in ((sc.SC_NOISE_MAD, "mad"), (sc.SC_NOISE_STD, "std"), (sc.SC_NOISE_GAUSS, "gauss")):
                code, got = _static(lib, d, mode)
                assert code == sc.SC_OK, sc.sc_strerror(code)
                ref = ctx.noise(d, name)
                assert abs(got - ref) <= SIG_RTOL * ref, (name, got, ref)


def _cases():
    rng = np.random.default_rng(99)
    n = 1 << 22  # the maximum size
    yield "normal_nan", np.where(rng.random(1_000_003) < 0.02, np.nan, rng.standard_normal(1_000_003))
    yield "cauchy", 2.0 + 0.5 * rng.standard_cauchy(700_001)
    # a tenth of a unit resolution: the middle bins hold far more values than
    # the 64 Ki / 512 Ki candidate lists, so the plan switches to full passes
    yield "rounded_max", np.round(rng.standard_normal(n), 1)
    yield "constant_max", np.full(n, -3.25)


@pytest.mark.parametrize("name", [c[0] for c in _cases()])
def test_static_noise_against_the_oracle(name):
    """Every mode against the oracle on the finite values, twice in a row."""
    from paper_2106_15789_gb300 import sc

    lib = sc.lib()
    v = dict(_cases())[name].astype(np.float32)
    fin = v[np.isfinite(v)].astype(np.float64)
    d = torch.from_numpy(v).cuda()
    for _ in range(2):
        for mode, oname in ((sc.SC_NOISE_MAD, "mad"), (sc.SC_NOISE_STD, "std")):
            code, got = _static(lib, d, mode)
            assert code == sc.SC_OK, sc.sc_strerror(code)
            ref = O.noise(fin, oname)
            assert (got == 0.0) if ref == 0.0 else abs(got - ref) <= SIG_RTOL * ref, (oname, got, ref)
        code, got = _static(lib, d, sc.SC_NOISE_GAUSS)
        assert code == sc.SC_OK
        assert close_to_any(got, gauss_refs(fin)), (got, gauss_refs(fin))


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
