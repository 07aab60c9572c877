"""CPU-side checks of the C ABI: the library builds and loads, exports every
symbol include/sc.h declares, and its host-only entry points behave (no GPU
compute here)."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle.sc_oracle import cascade_widths

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sc.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2106_15789_gb300 import build, sc

    if not os.path.exists(sc.LIB_PATH):
        build.build()
    return sc.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w]+\s*\*?\s*(sc_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("sc_create", "sc_destroy", "sc_strerror", "sc_run", "sc_run_host", "sc_smooth", "sc_noise",
                 "sc_cascade_widths", "sc_get_stats", "sc_set_profiling"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_strerror(lib):
    from paper_2106_15789_gb300 import sc

    for code in range(0, -9, -1):
        s = sc.sc_strerror(code)
        assert s and s != "unknown status code"
    assert sc.sc_strerror(-99) == "unknown status code"


def test_cascade_widths_match_oracle(lib):
    from paper_2106_15789_gb300 import sc

    for f in np.linspace(0.05, 60.0, 1200):
        f32 = float(np.float32(f))
        assert sc.sc_cascade_widths(f32) == (cascade_widths(f32) or (1, 1, 1)), f32
    assert sc.sc_cascade_widths(0.0) == (1, 1, 1)
    with pytest.raises(sc.ScError):
        sc.sc_cascade_widths(float("nan"))
    w = (ctypes.c_int32 * 3)()
    assert lib.sc_cascade_widths(ctypes.c_float(1e9), w) == sc.SC_ERR_ARG


def test_sampled_gauss_taps_match_oracle(lib):
    """The library's sampled-Gaussian taps (its own host code) equal the
    oracle's for 2,400 FWHMs; too small a buffer or a bad FWHM is refused."""
    from oracle.sc_oracle import gauss_taps
    from paper_2106_15789_gb300 import sc

    for f in np.linspace(0.05, 60.0, 2400):
        f32 = float(np.float32(f))
        assert sc.sc_gauss_taps(f32) == tuple(int(v) for v in gauss_taps(f32)), f32
    assert sc.sc_gauss_taps(0.0) == (1024,)
    t = (ctypes.c_int32 * 5)()
    assert lib.sc_gauss_taps(ctypes.c_float(6.0), t, 5) == sc.SC_ERR_ARG  # needs 21 taps
    assert lib.sc_gauss_taps(ctypes.c_float(2.0), t, 5) == sc.SC_ERR_ARG  # needs 7
    assert lib.sc_gauss_taps(ctypes.c_float(float("nan")), t, 5) == sc.SC_ERR_ARG
    assert lib.sc_gauss_taps(ctypes.c_float(1.0), t, 5) == 3


def test_null_and_bad_args(lib):
    from paper_2106_15789_gb300 import sc

    assert lib.sc_create(None, 0, 10) == sc.SC_ERR_ARG
    h = ctypes.c_void_p()
    assert lib.sc_create(ctypes.byref(h), 0, 0) == sc.SC_ERR_ARG
    dims = (ctypes.c_int64 * 3)(4, 4, 4)
    assert lib.sc_run(None, None, dims, None, 1, 3.5, 0, 2.0, None, None, None, 0, None) == sc.SC_ERR_ARG
    assert lib.sc_noise(None, None, 10, 0, None, 0, None) == sc.SC_ERR_ARG
    lib.sc_destroy(None)  # accepted


def test_create_without_gpu_fails_cleanly(lib):
    import torch

    from paper_2106_15789_gb300 import sc

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.sc_create(ctypes.byref(h), 0, 1000) == sc.SC_ERR_CUDA
    assert not h.value


def test_struct_layouts_match_header(tmp_path):
    """The ctypes mirrors of sc_stats and sc_kernel have the C header's size and
    field offsets (a C program built against include/sc.h prints them)."""
    import shutil
    import subprocess

    from paper_2106_15789_gb300 import sc

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"sc_stats": sc.sc_stats, "sc_kernel": sc.sc_kernel}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "sc.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for field, _ in py._fields_:
            assert got[(cname, field)] == getattr(py, field).offset, (cname, field)
