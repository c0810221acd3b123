"""Host-side logic of bench.py (no GPU): the time-to-target model, peak
selection, the staleness rule of the committed DRAM-traffic figures, and the
many-chains size law."""
import hashlib
import json
import os

import pytest

import bench
from paper_2005_12338_gb300 import synth


def test_time_to_target_model():
    # two steps: fixed 1.0 s and 2.0 s, sampling 0.3 s over 300 pairs, stderr 1e-3 / sqrt(300)
    se = 1e-3 / 300 ** 0.5
    res = [(0.0, se, 1000.0, 300.0), (0.0, se, 2000.0, 300.0)]
    t = bench.time_to_target(res, 300, 1e-4)
    assert t["fixed_s"] == pytest.approx(1.5)
    assert t["per_pair_s"] == pytest.approx(1e-3)
    assert t["sd_per_pair"] == pytest.approx(1e-3)
    assert t["pairs_needed"] == pytest.approx(100.0)
    assert t["sampling_only_s"] == pytest.approx(0.1)
    assert t["seconds"] == pytest.approx(1.6)
    # a target already met still costs the minimum of two pairs
    assert bench.time_to_target(res, 300, 1.0)["pairs_needed"] == 2.0


def test_forms():
    assert bench.FORMS["plain"] == ("fp64", "fp64")
    assert bench.FORMS["chosen"] == ("bf16", "oz")
    assert set(bench.FORMS) == {"plain", "chosen", "df64"}


def test_traffic_figures_go_stale_with_their_source(tmp_path, monkeypatch):
    src_dir = tmp_path / "paper_2005_12338_gb300" / "csrc"
    src_dir.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    src = src_dir / "k.cu"
    src.write_text("kernel v1\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(
        {"plain/dd_spmm": {"source": "k.cu", "source_sha": sha, "bytes_per_launch": 123}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for("dd_spmm", "plain") == 123
    assert bench.traffic_for("dd_gemm", "plain") is None
    src.write_text("kernel v2\n")
    assert bench.traffic_for("dd_spmm", "plain") is None


def test_many_sizes():
    assert synth.many_sizes(1, 64, 256) == [64]
    sz = synth.many_sizes(16, 64, 256)
    assert sz[0] == 64 and sz[-1] == 256 and len(sz) == 16
    assert all(b > a for a, b in zip(sz, sz[1:]))


def test_committed_traffic_file_is_well_formed():
    d = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    for key, v in d.items():
        assert set(v) >= {"source", "source_sha", "bytes_per_launch"}, key
        assert os.path.exists(os.path.join(bench.ROOT, "paper_2005_12338_gb300", "csrc",
                                           v["source"])), key
