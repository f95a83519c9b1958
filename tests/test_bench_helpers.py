"""bench.py's line-building helpers, on the CPU with made-up counters: the
roofline objects carry the contract's fields and arithmetic, the peaks fall
back when no measured file exists, and committed DRAM traffic is reported
only while its kernel's source is unchanged."""
import hashlib
import json
import os
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

PEAKS = {"hbm_gbs": 7000.0, "bf16_tflops": 2000.0, "bf16_tflops_sustained": 1700.0, "kind": "measured"}


def _stats(**kw):
    base = dict(row_ors=1000, rows_changed=100, row_bytes=8192, gather_launches=10, ms_gather=2.0,
                tile_kstages=5000, tile_launches=4, ms_tile_products=1.0)
    base.update(kw)
    return types.SimpleNamespace(**base)


def _check_roofline(rf):
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in rf, k
    assert rf["frac"] == pytest.approx(rf["achieved"] / rf["peak"])


def test_gather_roofline_counts_algorithmic_bytes():
    st = _stats()
    rf = bench._roofline_gather(st, PEAKS, 12345)
    _check_roofline(rf)
    alg = (1000 + 2 * 100) * 8192
    assert rf["bound"] == "hbm" and rf["unit"] == "GB/s" and rf["peak"] == 7000.0
    assert rf["achieved"] == pytest.approx(alg / 2e-3 / 1e9)
    assert rf["algorithmic_bytes_per_launch"] == pytest.approx(alg / 10)
    assert rf["traffic"] is None  # no capture of a 12345-vertex workload


@pytest.mark.parametrize("fp4,nv,ratio,kind", [(False, False, 2.0, "kind::f8f6f4"), (True, False, 6.0, "kind::mxf4,"),
                                               (True, True, 6.0, "kind::mxf4nvf4")])
def test_tile_roofline_takes_the_format_peak(fp4, nv, ratio, kind):
    st = _stats()
    rf = bench._roofline_tiles(st, PEAKS, 12345, fp4=fp4, nv=nv)
    _check_roofline(rf)
    assert rf["bound"] == "tensor" and rf["unit"] == "TFLOP/s"
    assert rf["peak"] == pytest.approx(1700.0 * ratio)
    assert rf["achieved"] == pytest.approx(5000 * bench.TILE_FLOP_PER_KSTAGE / 1e-3 / 1e12)
    assert kind in rf["kernel"]


def test_peaks_fall_back_without_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    p = bench._peaks()
    assert p["kind"] == "fallback" and p["hbm_gbs"] == 6800.0 and p["bf16_tflops"] == 1900.0
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 7100, "bf16_tflops": 2100}))
    p = bench._peaks()
    assert p["kind"] == "measured" and p["hbm_gbs"] == 7100.0
    assert p["bf16_tflops_sustained"] == 2100.0  # the burst figure when no sustained one is given


def test_traffic_only_for_the_captured_source(tmp_path, monkeypatch):
    from paper_2103_14688_gb300 import build as B
    src = open(os.path.join(B.CSRC, "cfpq_tc.cu"), "rb").read()
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    rec = {"source_file": "cfpq_tc.cu", "kernel_source_sha1": hashlib.sha1(src).hexdigest(),
           "dram_bytes_per_launch": 123456789}
    (tmp_path / "profiles" / "k_x.json").write_text(json.dumps(rec))
    assert bench._traffic_from_profiles("k_x") == 123456789
    rec["kernel_source_sha1"] = "0" * 40  # taken on another version of the kernel
    (tmp_path / "profiles" / "k_x.json").write_text(json.dumps(rec))
    assert bench._traffic_from_profiles("k_x") is None
    assert bench._traffic_from_profiles("k_missing") is None


def test_committed_traffic_records_name_their_kernel_file():
    """Every committed traffic record names a kernel source file that exists,
    with a SHA-1 and a per-launch byte count (whether it is current is
    decided when the bench runs)."""
    from paper_2103_14688_gb300 import build as B
    recs = [f for f in os.listdir(os.path.join(ROOT, "profiles")) if f.endswith(".json")]
    assert recs
    for f in recs:
        d = json.load(open(os.path.join(ROOT, "profiles", f)))
        assert os.path.exists(os.path.join(B.CSRC, d.get("source_file", "cfpq_kernels.cu"))), f
        assert len(d["kernel_source_sha1"]) == 40 and d["dram_bytes_per_launch"] > 0, f


def test_dyck_config_names_the_workload():
    c = bench._dyck_config(65536, "flush")
    assert c["workload"] == "dyck4_zipf_n65536" and c["n"] == 65536 and c["rsm_states"] == 11
