"""CPU checks of the seeded input generator (synth/cubes.py) against the recipe
it states: unit beam-correlated noise, channel ripple, NaN blocks, galaxy
parameter ranges, uneven batch shapes, and the 16-bit storage form."""
import math

import numpy as np
import torch

from synth import cubes as S


def test_deterministic_per_seed():
    a, b = S.make_cube(S.SMALL), S.make_cube(S.SMALL)
    assert torch.equal(torch.nan_to_num(a, nan=7.0), torch.nan_to_num(b, nan=7.0))
    c = S.make_cube(S.CubeSpec(**{**S.SMALL.__dict__, "seed": 1}))
    assert not torch.equal(torch.nan_to_num(a, nan=7.0), torch.nan_to_num(c, nan=7.0))


def test_noise_is_unit_and_beam_correlated():
    """White N(0, 1) convolved with a 5 px FWHM Gaussian beam in x and y, then
    scaled to unit standard deviation: neighbours along x and y correlate as
    exp(-d^2 / (4 s^2)) with s = 5 / sqrt(8 ln 2), and channels not at all."""
    spec = S.CubeSpec(nx=160, ny=160, nz=40, seed=3, n_gal=0, name="noise")
    c = S.make_cube(spec).numpy().astype(np.float64)
    assert abs(c.std() - 1.0) < 1e-5 and abs(c.mean()) < 0.05
    s = 5.0 / math.sqrt(8.0 * math.log(2.0))
    inner = c[:, 20:-20, 20:-20]  # away from the zero-padded edges
    for d in (1, 2, 4):
        rx = np.corrcoef(inner[:, :, :-d].ravel(), inner[:, :, d:].ravel())[0, 1]
        ry = np.corrcoef(inner[:, :-d, :].ravel(), inner[:, d:, :].ravel())[0, 1]
        want = math.exp(-d * d / (4.0 * s * s))
        assert abs(rx - want) < 0.02 and abs(ry - want) < 0.02, (d, rx, ry, want)
    rz = np.corrcoef(inner[:-1].ravel(), inner[1:].ravel())[0, 1]
    assert abs(rz) < 0.02


def test_channel_ripple():
    spec = S.CubeSpec(nx=96, ny=96, nz=256, seed=4, n_gal=0, ripple=0.1, name="ripple")
    c = S.make_cube(spec).numpy().astype(np.float64)
    ch = c[:, 10:-10, 10:-10].reshape(256, -1).std(axis=1)
    want = 1.0 + 0.1 * np.sin(2.0 * np.pi * np.arange(256) / 128.0)
    # one channel holds ~100 independent beams (7 % scatter of its std), so
    # compare channels grouped by ripple phase: 8 phase bins of 32 channels
    phase = (np.arange(256) % 128) // 16
    got = np.array([ch[phase == b].mean() for b in range(8)])
    exp = np.array([want[phase == b].mean() for b in range(8)])
    scale = got.mean() / exp.mean()
    assert np.all(np.abs(got / (scale * exp) - 1.0) < 0.03), got / (scale * exp)
    assert np.corrcoef(got, exp)[0, 1] > 0.95


def test_nan_blocks():
    c = S.make_cube(S.SMALL).numpy()
    nan = np.isnan(c)
    block = np.zeros_like(nan)
    block[:47, :24, :24] = True
    assert np.array_equal(nan, block)
    assert abs(nan.mean() - 24 * 24 * 47 / (64 * 64 * 128)) < 1e-12
    spec = S.CubeSpec(nx=40, ny=30, nz=8, seed=5, n_gal=3, nan_border=3, name="border")
    c = S.make_cube(spec).numpy()
    nan = np.isnan(c)
    assert nan[:, :3, :].all() and nan[:, -3:, :].all() and nan[:, :, :3].all() and nan[:, :, -3:].all()
    assert not nan[:, 3:-3, 3:-3].any()


def test_galaxy_parameters_in_range():
    for spec in (S.SMALL, S.CubeSpec(**{**S.WALLABY.__dict__, "n_gal": 500})):
        ps = S._galaxy_params(spec)
        assert len(ps) == spec.n_gal
        lo, hi = spec.snr
        for p in ps:
            assert lo <= p["snr"] <= hi and 0.3 <= p["axis_ratio"] <= 1.0 and 0.0 <= p["pa"] <= math.pi
            assert spec.fwhm_xy[0] <= p["fwhm_maj"] <= spec.fwhm_xy[1]
            assert spec.fwhm_z[0] <= p["fwhm_z"] <= spec.fwhm_z[1]
            assert 0 <= p["x"] <= spec.nx - 1 and 0 <= p["y"] <= spec.ny - 1 and 0 <= p["z"] <= spec.nz - 1
    # log-uniform S/N: the median of log S/N sits near the middle of the log range
    snr = np.array([p["snr"] for p in S._galaxy_params(S.CubeSpec(**{**S.WALLABY.__dict__, "n_gal": 2000}))])
    assert abs(np.median(np.log(snr)) - 0.5 * (math.log(3.0) + math.log(50.0))) < 0.1


def test_batch_shapes():
    specs = S.batch_specs(64)
    assert len(specs) == 64 and len({(s.nx, s.ny, s.nz) for s in specs}) > 60
    for s in specs:
        assert 128 <= s.nx <= 512 and 128 <= s.ny <= 512 and 256 <= s.nz <= 1024
    assert [(s.nx, s.ny, s.nz) for s in S.batch_specs(4)] == [(s.nx, s.ny, s.nz) for s in specs[:4]]


def test_half_storage_round_trip():
    """decode(encode(C)) is C to the storage's precision: BF16 with scale
    max|C_z| / 256 keeps 8 significant bits, FP16 with max|C_z| / 2^14 keeps 11."""
    c = S.make_cube(S.SMALL)
    for bf16, rel in ((True, 2.0 ** -8), (False, 2.0 ** -11)):
        bits, scale = S.encode_half(c, bf16)
        d = S.decode_half(bits.numpy(), scale.numpy(), bf16)
        x = c.numpy()
        ok = np.isfinite(x)
        assert np.array_equal(np.isnan(d), ~ok)
        err = np.abs(d[ok] - x[ok])
        assert np.all(err <= rel * np.abs(x[ok]) + 1e-30 + 2.0 ** -24 * scale.numpy().max()), (bf16, err.max())
