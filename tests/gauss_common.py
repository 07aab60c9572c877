"""Reference values for the Gaussian-fit noise mode, shared by the GPU tests.

The library's MAD noise sigma_M comes from float32 keys of |s - median| (exact
order statistics, rounded once), the oracle's from exact float64 ones: they
differ by at most 2^-23 relative, so the histogram scale k = fl32(128 / (5
sigma_M)) can differ by an ulp and values within that ulp of a bin edge change
bins. A library result is accepted when it is within SIG_RTOL of the oracle's
Gaussian-fit noise with sigma_M scaled by (1 + j 2^-24), j = -2..2: the oracle
at the sigma_M values that rounding allows (no library value enters it).
"""
import numpy as np

import oracle.sc_oracle as O

SIG_RTOL = 1e-6


def gauss_refs(v: np.ndarray) -> list[float]:
    """The oracle's Gaussian-fit noise of the finite float32 values v at the
    exact sigma_M and at sigma_M moved by up to two float32 ulps ([nan] when v
    is empty, [0.0] when sigma_M is 0)."""
    v = np.asarray(v, dtype=np.float64)
    v = v[np.isfinite(v)]
    if v.size == 0:
        return [float("nan")]
    s_mad = O.noise(v, "mad")
    if not s_mad > 0.0:
        return [0.0]
    out = []
    for j in (-2, -1, 0, 1, 2):
        sm = s_mad * (1.0 + j * 2.0 ** -24)
        tau = O.gauss_fit(O.gauss_histogram(v, sm))
        out.append(sm if tau is None else tau * 128.0 / float(O.gauss_scale(sm)))
    return out


def close_to_any(got: float, refs: list[float], rtol: float = SIG_RTOL) -> bool:
    if np.isnan(refs[0]):
        return bool(np.isnan(got))
    return any((got == 0.0) if r == 0.0 else abs(got - r) <= rtol * r for r in refs)
