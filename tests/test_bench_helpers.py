"""CPU checks of bench.py's host-side helpers: the DRAM-traffic record, the
per-pair kernel names and algorithmic bytes, the roofline arithmetic of the
dominant smoothing kernel and of the Gaussian-fit histogram pass, and the
sub-cubes of the CPU baseline."""
import csv
import json
import os

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_committed_traffic_record_matches_the_sources():
    """The bench uses profiles/smooth_traffic.json only while it matches the
    smoothing sources as they stand; a stale record reports traffic as null."""
    rec = json.load(open(os.path.join(ROOT, "profiles", "smooth_traffic.json")))
    if rec["source_sha256_16"] != bench.smooth_source_hash():
        assert bench.smooth_traffic_record() is None
        return
    assert bench.smooth_traffic_record() is not None
    for name, b in rec["kernels"].items():
        # near the algorithmic bytes: 8.125 full kernels, 12 shared passes, 16.125 full kernels storing P;
        # a shared pass also re-reads the 2r halo planes of P at each of its z chunks (on the 512^3 capture
        # cube 32-plane chunks for boxcars of 3 and 7: up to 6 / 32 more P reads), so it may sit above 12
        want = 16.125 if name.endswith("+P") else (12.0 if name.startswith("k_smooth_p") else 8.125)
        above = 1.0 if name.startswith("k_smooth_p") else 0.5
        assert want - 0.5 < b < want + above, (name, b)


def test_record_traffic_means(tmp_path, monkeypatch):
    """One-kernel captures: two launches of one kernel (read + write in MB
    and GB, a time metric that is ignored), one launch of another; mean
    bytes per voxel of each key."""
    head = ["ID", "Process ID", "Process Name", "Host Name", "Kernel Name", "Context", "Stream", "Block Size",
            "Grid Size", "Device", "CC", "Section Name", "Metric Name", "Metric Unit", "Metric Value"]
    nv = bench.TRAFFIC_WORKLOAD_VOXELS

    def row(i, name, metric, unit, value):
        return [str(i), "1", "python", "h", name, "1", "7", "(512,1,1)", "(152,1,1)", "0", "10.3", "Command line",
                metric, unit, value]

    p = "void sc::k_smooth_p<32, 6>(CUtensorMap_st, sc::SmoothArgs, sc::ShareArgs)"
    z = "void sc::k_smooth_z<4, 1, 1, 512>(sc::SmoothArgs)"
    a = [head,
         row(0, p, "dram__bytes_read.sum", "Mbyte", f"{8.0 * nv / 1e6:,.6f}"),
         row(0, p, "dram__bytes_write.sum", "Mbyte", f"{4.0 * nv / 1e6:,.6f}"),
         row(1, p, "dram__bytes_read.sum", "Gbyte", f"{8.2 * nv / 1e9:.9f}"),
         row(1, p, "dram__bytes_write.sum", "Gbyte", f"{4.0 * nv / 1e9:.9f}"),
         row(1, p, "gpu__time_duration.sum", "usecond", "1000")]
    b = [head,
         row(0, z, "dram__bytes_read.sum", "byte", str(int(4.1 * nv))),
         row(0, z, "dram__bytes_write.sum", "byte", str(int(3.9 * nv)))]
    for name, rows in (("p.csv", a), ("z.csv", b)):
        with open(tmp_path / name, "w", newline="") as f:
            csv.writer(f).writerows(rows)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "smooth_source_hash", lambda: "0123456789abcdef")
    specs = [f"k_smooth_p<5,5,5>={tmp_path / 'p.csv'}", f"k_smooth_z={tmp_path / 'z.csv'}"]
    assert bench.record_traffic(specs, "cmd") == 0
    rec = json.load(open(tmp_path / "profiles" / "smooth_traffic.json"))
    assert rec["source_sha256_16"] == "0123456789abcdef" and rec["command"] == "cmd"
    assert rec["launches"] == {"k_smooth_p<5,5,5>": 2, "k_smooth_z": 1}
    assert rec["kernels"]["k_smooth_p<5,5,5>"] == pytest.approx(12.1, abs=1e-3)
    assert rec["kernels"]["k_smooth_z"] == pytest.approx(8.0, abs=1e-3)


class _FakeSc:
    SC_KERNEL_NONE, SC_KERNEL_IDENTITY, SC_KERNEL_Z, SC_KERNEL_WS32, SC_KERNEL_WS16 = 0, 1, 2, 3, 4
    SC_KERNEL_TILE, SC_KERNEL_GENERIC, SC_KERNEL_SHARED, SC_KERNEL_FIR = 5, 6, 7, 8

    @staticmethod
    def sc_cascade_widths(fwhm):
        from oracle.sc_oracle import cascade_widths

        return cascade_widths(fwhm) or (1, 1, 1)


def test_dominant_kernel_roofline(monkeypatch):
    """Two spatial kernels on the warp-specialised kernel and one spectral-only
    pair: the group with the most time is the dominant kernel, and achieved =
    8.125 B x voxels / its mean launch time."""
    monkeypatch.setattr(bench, "smooth_traffic_record", lambda: None)
    kernels = [(0.0, 3), (3.0, 0), (3.0, 7), (6.0, 0), (6.0, 7)]
    st = {"smooth_launches_pair": [1, 1, 1, 1, 1] + [0] * 59, "smooth_kernel_pair": [2, 3, 3, 3, 3] + [0] * 59,
          "ms_smooth_pair": [4.0, 7.0, 7.5, 10.0, 10.5] + [0.0] * 59, "ms_smooth": 39.0}
    r = bench.dominant_kernel(_FakeSc, kernels, st, 1_000_000_000, 1, 6674.2, "measured")
    assert r["kernel"] == "k_smooth_ws<5,5,5>"
    assert r["launch_ms"] == pytest.approx(10.25)
    assert r["achieved"] == pytest.approx(8.125e9 / 10.25e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6674.2)
    assert r["share_of_smoothing"] == pytest.approx(20.5 / 39.0)
    assert r["smoothing_ms_by_kernel"] == {"k_smooth_z": 4.0, "k_smooth_ws<1,3,3>": 14.5, "k_smooth_ws<5,5,5>": 20.5}
    assert r["traffic"] is None


def test_pair_kernels_with_shared_passes():
    """The first pair of a shared run also writes its spatial sums (16.125 B),
    the shared pairs read them and write S (12 B), other pairs 8.125 B; the
    dominant group's bytes are the sum over its launches."""
    kernels = [(0.0, 0), (0.0, 3), (3.0, 0), (3.0, 3), (3.0, 7), (6.0, 0), (6.0, 3)]
    codes = [0, 2, 3, 7, 7, 3, 7] + [0] * 57
    pk = bench.pair_kernels(_FakeSc, kernels, codes)
    assert pk == [("none", 8.125), ("k_smooth_z", 8.125), ("k_smooth_ws<1,3,3>+P", 16.125),
                  ("k_smooth_p<1,3,3>", 12.0), ("k_smooth_p<1,3,3>", 12.0), ("k_smooth_ws<5,5,5>+P", 16.125),
                  ("k_smooth_p<5,5,5>", 12.0)]
    st = {"smooth_launches_pair": [0, 1, 1, 1, 1, 1, 1] + [0] * 57, "smooth_kernel_pair": codes,
          "ms_smooth_pair": [0.0, 4.0, 8.0, 3.0, 4.0, 10.0, 3.0] + [0.0] * 57, "ms_smooth": 32.0}
    r = bench.dominant_kernel(_FakeSc, kernels, st, 1_000_000_000, 1, 6674.2, "measured")
    assert r["kernel"] == "k_smooth_ws<5,5,5>+P" and r["algorithmic_bytes_per_voxel"] == 16.125
    st["ms_smooth_pair"][3] = 9.0  # the shared FWHM-3 pairs now dominate: 13 ms for two launches
    r = bench.dominant_kernel(_FakeSc, kernels, st, 1_000_000_000, 1, 6674.2, "measured")
    assert r["kernel"] == "k_smooth_p<1,3,3>" and r["launch_ms"] == pytest.approx(6.5)
    assert r["achieved"] == pytest.approx(2 * 12.0e9 / 13e-3 / 1e9)


def test_gauss_hist_roofline():
    r = bench.gauss_hist_roofline({"ms_gauss_hist": 10.0, "gauss_hist_values": 1_500_000_000}, 6674.2, "measured")
    assert r["achieved"] == pytest.approx(4 * 1.5e9 / 10e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6674.2) and r["bound"] == "hbm"
    assert bench.gauss_hist_roofline({"ms_gauss_hist": 0.0, "gauss_hist_values": 0}, 6674.2, "measured") is None


def test_interior_subcubes():
    """Disjoint sub-cubes clear of the NaN border, z-major, as many as asked
    (144 fit the WALLABY-shaped cube)."""
    corners, shape = bench.interior_subcubes((1024, 1200, 1200), 200)
    assert shape == (256, 192, 192) and len(corners) == 144
    boxes = set()
    for z, y, x in corners:
        assert y >= 16 and x >= 16 and y + 192 <= 1184 and x + 192 <= 1184 and z + 256 <= 1024
        for dz in (0, 255):
            for dy in (0, 191):
                for dx in (0, 191):
                    assert (z + dz, y + dy, x + dx) not in boxes
                    boxes.add((z + dz, y + dy, x + dx))
    c16, _ = bench.interior_subcubes((1024, 1200, 1200), 16)
    assert c16 == corners[:16]


def test_pair_kernels_sampled_gaussian():
    """Sampled-Gaussian runs: the FIR kernel stores the spatial sums of its
    run (+P) and the shared passes are named by the FWHM."""
    kernels = [(0.0, 0), (0.0, 3), (3.0, 0), (3.0, 3), (6.0, 0), (6.0, 7)]
    codes = [0, 2, 8, 7, 8, 7] + [0] * 58
    pk = bench.pair_kernels(_FakeSc, kernels, codes, sampled=True)
    assert pk == [("none", 8.125), ("k_smooth_z", 8.125), ("k_smooth_ws<sampled 3 px>+P", 16.125),
                  ("k_smooth_p<sampled 3 px>", 12.0), ("k_smooth_ws<sampled 6 px>+P", 16.125),
                  ("k_smooth_p<sampled 6 px>", 12.0)]
