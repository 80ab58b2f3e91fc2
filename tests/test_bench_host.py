"""Host logic of bench.py: the algorithmic bytes behind the roofline numerator,
and the digest that ties a recorded ncu traffic figure to the kernel sources it
was measured on.  CPU only."""
import os
import shutil

import pytest

import bench


def test_pass_bytes_match_the_per_node_formulas():
    # 2187^2, 2 components, float32: the per-node counts 4ds+1, 2ds, 3ds, 6ds
    # with the exact half spectrum (1094 of 2187 frequencies along the last axis)
    n, d, s = 2187, 2, 4
    kb = bench.pass_bytes(n, d, s)
    nodes = n * n
    spec = 2 * s * d * 1094 * n
    assert kb["row_fwd"][1] == 3 * d * s * nodes + nodes + spec
    assert kb["col_green"][1] == 2 * spec
    assert kb["row_inv"][1] == spec + 2 * d * s * nodes
    assert kb["cg_update"][1] == 6 * d * s * nodes
    # the spectrum is ~d*s bytes per node: the half spectrum of a real field
    assert abs(spec / (d * s * nodes) - 1.0) < 1e-3
    mb = {k: v[1] / 1e6 for k, v in kb.items()}
    assert mb["row_fwd"] == pytest.approx(157.9, abs=0.1)
    assert mb["col_green"] == pytest.approx(76.6, abs=0.1)
    assert mb["row_inv"] == pytest.approx(114.8, abs=0.1)
    assert mb["cg_update"] == pytest.approx(229.6, abs=0.1)
    # profile indices of fh_profile: direction, Green, A p, update
    assert [kb[k][0] for k in ("row_fwd", "col_green", "row_inv", "cg_update")] == [0, 1, 2, 3]


def _write_traffic(root, rows):
    os.makedirs(os.path.join(root, "profiles"), exist_ok=True)
    with open(os.path.join(root, "profiles", "traffic_c2_2187_fp32.md"), "w") as f:
        f.write("| kernel | csrc digest | bytes |\n|---|---|---|\n")
        for k, dg, b in rows:
            f.write(f"| {k} | {dg} | {b} |\n")


def test_recorded_traffic_needs_the_current_digest(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "csrc_digest", lambda: "cafe0000cafe0000")
    _write_traffic(str(tmp_path), [("row_fwd", "cafe0000cafe0000", 123),
                                   ("col_green", "0123456789abcdef", 456),
                                   ("row_inv", "cafe0000cafe0000", "n/a")])
    assert bench.recorded_traffic("row_fwd") == 123
    assert bench.recorded_traffic("col_green") is None      # taken on other kernel sources
    assert bench.recorded_traffic("row_inv") is None        # not a number
    assert bench.recorded_traffic("cg_update") is None      # not recorded


def test_recorded_traffic_without_a_summary(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("row_fwd") is None


def test_digest_follows_every_kernel_source(tmp_path, monkeypatch):
    src = os.path.join(bench.ROOT, "paper_1004_1122_gb300", "csrc")
    dst = tmp_path / "paper_1004_1122_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES:
        shutil.copy(os.path.join(src, f), dst / f)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    d0 = bench.csrc_digest()
    assert d0 == bench.csrc_digest() and len(d0) == 16
    for f in bench.KERNEL_SOURCES:
        p = dst / f
        text = p.read_bytes()
        p.write_bytes(text + b"\n")
        assert bench.csrc_digest() != d0, f
        p.write_bytes(text)
    assert bench.csrc_digest() == d0
