"""bench.py's use of the committed ncu summaries: a measured count is used only
while the sources it was taken on are unchanged (comments aside), and the
roofline models' arithmetic."""
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _copy_tree(tmp_path):
    for d in ("profiles", os.path.join("paper_2111_03005_gb300", "csrc")):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d)
    return tmp_path


def test_committed_profiles_match_this_tree():
    # both summaries the bench lines use were taken on the sources as committed
    assert bench.traffic_from_profile("k_sortpair", "gnp_2p24") is not None
    assert bench.resident_inst_from_profile("gnp_small") is not None


def test_comment_edits_keep_a_profile_and_code_edits_void_it(tmp_path, monkeypatch):
    root = _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    base_traffic = bench.traffic_from_profile("k_sortpair", "gnp_2p24")
    base_inst = bench.resident_inst_from_profile("gnp_small")
    assert base_traffic and base_inst
    rc = root / "paper_2111_03005_gb300" / "csrc" / "round.cu"
    rs = root / "paper_2111_03005_gb300" / "csrc" / "resident.cu"
    rc.write_text(rc.read_text() + "\n// a comment changes no kernel\n\n")
    rs.write_text(rs.read_text() + "\n// nor here\n")
    assert bench.traffic_from_profile("k_sortpair", "gnp_2p24") == base_traffic
    assert bench.resident_inst_from_profile("gnp_small") == base_inst
    rc.write_text(rc.read_text() + "\nstatic int unused_variable_for_the_test = 1;\n")
    assert bench.traffic_from_profile("k_sortpair", "gnp_2p24") is None
    assert bench.resident_inst_from_profile("gnp_small") == base_inst   # resident.cu untouched
    rs.write_text(rs.read_text() + "\nstatic int another_unused_variable = 2;\n")
    assert bench.resident_inst_from_profile("gnp_small") is None


def test_missing_or_broken_summaries_give_none(tmp_path, monkeypatch):
    root = _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.traffic_from_profile("k_sortpair", "no_such_workload") is None
    (root / "profiles" / "inst_k_round_resident_gnp_small.txt").write_text("sources_sha256=x\n")
    assert bench.resident_inst_from_profile("gnp_small") is None


def test_algorithmic_bytes_per_stage():
    m, L = 1000, 500
    assert bench.algorithmic_bytes("permute", m, L, 4, 8, 0) == 12 * m + 4 * L + 16 * m
    assert bench.algorithmic_bytes("sortpair", m, L, 4, 8, 0) == 28 * m + 44 * L
    assert bench.algorithmic_bytes("group", m, L, 4, 8, 0) == 32 * L
    assert bench.algorithmic_bytes("resident", m, L, 4, 8, 0) == 0
    # the whole round: 220 bytes per switch at two positions per switch (the scans are per bucket)
    total = sum(bench.algorithmic_bytes(s, m, L, 0, 0, 0) for s in ("permute", "sortpair", "sources", "group", "wave1"))
    assert total / L == 220
