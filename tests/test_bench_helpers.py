"""Host-side helpers of bench.py (CPU): the stored-capture lookup of the
roofline's DRAM traffic, and the algorithmic bytes of the HBM-bound stages."""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _fake_tree(tmp_path, source_text, workload="corehalo16m"):
    src_dir = tmp_path / "paper_2302_07567_gb300" / "csrc"
    src_dir.mkdir(parents=True)
    (src_dir / "adjoint.cu").write_text(source_text)
    (tmp_path / "profiles").mkdir()
    cap = {"workload": workload, "N": 1000,
           "kernels": {"k_adj_near": {"source": "adjoint.cu", "bytes": 5000.0,
                                      "source_sha256": hashlib.sha256(b"kernel v1").hexdigest()}}}
    (tmp_path / "profiles" / "dram_traffic_corehalo.json").write_text(json.dumps(cap))


def test_traffic_scales_a_current_capture(tmp_path, monkeypatch):
    _fake_tree(tmp_path, "kernel v1")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    b, basis = bench.traffic_of("adj_near", "corehalo16m", 4000)
    assert b == 20000.0 and "unchanged" in basis


def test_traffic_is_withheld_for_a_changed_source_or_another_workload(tmp_path, monkeypatch):
    _fake_tree(tmp_path, "kernel v2")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    b, basis = bench.traffic_of("adj_near", "corehalo16m", 4000)
    assert b is None and "changed" in basis
    b, basis = bench.traffic_of("adj_near", "gauss4k", 4000)
    assert b is None
    b, basis = bench.traffic_of("m2l", "corehalo16m", 4000)  # no capture of that kernel
    assert b is None


def test_hbm_bytes_grow_with_n():
    w = bench.WORKLOADS["corehalo16m"]
    small = bench.hbm_bytes({"kappa": 12}, w, 1 << 20)
    large = bench.hbm_bytes({"kappa": 16}, w, 1 << 24)
    assert set(small) == set(large) and all(v > 0 for v in small.values())
    assert all(large[k] > 8 * small[k] for k in small)
