"""CPU checks of bench.py's host-side helpers: kernel-name grouping of ncu
launch lists, the DRAM-traffic record, the roofline arithmetic of the dominant
smoothing kernel and of the Gaussian-fit histogram pass."""
import csv
import json
import os

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_kernel_key_grouping():
    k = bench.ncu_kernel_key
    assert k("void sc::k_smooth_ws<5, 5, 5, true, true, 32>(sc::SmoothArgs)") == "k_smooth_ws<5,5,5>"
    assert k("void sc::k_smooth_ws<1, 3, 3, true, false, 16>(sc::SmoothArgs)") == "k_smooth_ws<1,3,3>/16"
    assert k("void sc::k_smooth_tile<7, 9, 9, true>(sc::SmoothArgs)") == "k_smooth_tile<7,9,9>"
    assert k("void sc::k_smooth_z<4, 1, 1, 512>(sc::SmoothArgs)") == "k_smooth_z"
    assert k("sc::k_smooth_generic(sc::SmoothArgs)") == "k_smooth_generic"
    assert k("void sc::k_pass2(const float *, long long)") is None


def test_committed_traffic_record_matches_the_sources():
    """The bench uses profiles/smooth_traffic.json only while it matches the
    smoothing sources as they stand; a stale record reports traffic as null."""
    rec = json.load(open(os.path.join(ROOT, "profiles", "smooth_traffic.json")))
    if rec["source_sha256_16"] != bench.smooth_source_hash():
        assert bench.smooth_traffic_record() is None
        return
    assert bench.smooth_traffic_record() is not None
    for name, b in rec["kernels"].items():
        assert 7.5 < b < 13.0, (name, b)  # near the algorithmic bytes (8.125 full kernels, 12.125 shared pass)


def test_record_traffic_means(tmp_path, monkeypatch):
    """Two launches of one kernel (read + write in MB and GB), one of another,
    and a kernel that is not a smoothing kernel: mean bytes per voxel."""
    head = ["ID", "Process ID", "Process Name", "Host Name", "Kernel Name", "Context", "Stream", "Block Size",
            "Grid Size", "Device", "CC", "Section Name", "Metric Name", "Metric Unit", "Metric Value"]
    nv = bench.TRAFFIC_WORKLOAD_VOXELS

    def row(i, name, metric, unit, value):
        return [str(i), "1", "python", "h", name, "1", "7", "(512,1,1)", "(152,1,1)", "0", "10.3", "Command line",
                metric, unit, value]

    ws = "void sc::k_smooth_ws<5, 5, 5, true, true, 32>(sc::SmoothArgs)"
    z = "void sc::k_smooth_z<4, 1, 1, 512>(sc::SmoothArgs)"
    rows = [head,
            row(0, ws, "dram__bytes_read.sum", "Mbyte", f"{4.0 * nv / 1e6:,.6f}"),
            row(0, ws, "dram__bytes_write.sum", "Mbyte", f"{4.0 * nv / 1e6:,.6f}"),
            row(1, ws, "dram__bytes_read.sum", "Gbyte", f"{4.2 * nv / 1e9:.9f}"),
            row(1, ws, "dram__bytes_write.sum", "Gbyte", f"{4.0 * nv / 1e9:.9f}"),
            row(1, ws, "gpu__time_duration.sum", "usecond", "1000"),
            row(2, z, "dram__bytes_read.sum", "byte", str(int(4.1 * nv))),
            row(2, z, "dram__bytes_write.sum", "byte", str(int(3.9 * nv))),
            row(3, "void sc::k_pass2(const float *)", "dram__bytes_read.sum", "Mbyte", "537")]
    src = tmp_path / "t.csv"
    with open(src, "w", newline="") as f:
        csv.writer(f).writerows(rows)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "smooth_source_hash", lambda: "0123456789abcdef")
    assert bench.record_traffic(str(src), "cmd") == 0
    rec = json.load(open(tmp_path / "profiles" / "smooth_traffic.json"))
    assert rec["source_sha256_16"] == "0123456789abcdef" and rec["command"] == "cmd"
    assert rec["launches"] == {"k_smooth_ws<5,5,5>": 2, "k_smooth_z": 1}
    assert rec["kernels"]["k_smooth_ws<5,5,5>"] == pytest.approx(8.1, abs=1e-3)
    assert rec["kernels"]["k_smooth_z"] == pytest.approx(8.0, abs=1e-3)


class _FakeSc:
    SC_KERNEL_NONE, SC_KERNEL_IDENTITY, SC_KERNEL_Z, SC_KERNEL_WS32, SC_KERNEL_WS16 = 0, 1, 2, 3, 4
    SC_KERNEL_TILE, SC_KERNEL_GENERIC, SC_KERNEL_SHARED = 5, 6, 7

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


def test_gauss_hist_roofline():
    r = bench.gauss_hist_roofline({"ms_gauss_hist": 10.0, "gauss_hist_values": 1_500_000_000}, 6674.2, "measured")
    assert r["achieved"] == pytest.approx(4 * 1.5e9 / 10e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6674.2) and r["bound"] == "hbm"
    assert bench.gauss_hist_roofline({"ms_gauss_hist": 0.0, "gauss_hist_values": 0}, 6674.2, "measured") is None
