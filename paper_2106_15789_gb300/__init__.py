"""GB300-native smooth-and-clip (S+C) source finder of SoFiA 2 (arXiv:2106.15789).

The compute path is the CUDA library libsc.so (C ABI in include/sc.h); this
package holds its sources (csrc/), its build step (build.py) and a ctypes
binding with the C names (sc.py).
"""
from .sc import (Context, ScError, sc_cascade_widths, sc_create, sc_destroy, sc_get_stats, sc_noise, sc_run,
                 sc_run_host, sc_set_profiling, sc_smooth, sc_strerror)

__all__ = ["Context", "ScError", "sc_cascade_widths", "sc_create", "sc_destroy", "sc_get_stats", "sc_noise", "sc_run",
           "sc_run_host", "sc_set_profiling", "sc_smooth", "sc_strerror"]
