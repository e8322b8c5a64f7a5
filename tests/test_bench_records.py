"""The bench's use of the committed ncu record of the staged sweep (host logic, no GPU).

The record (DRAM bytes per pass, warp instructions per class) is reported only while it was
taken on the current source of the kernel: its hash must match the hash of the kernel's
layout, body and launcher in sweep.cu, and a change anywhere else in that file must not void
it.
"""
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_record_matches_the_current_kernel_source():
    h = bench._sweep_hash()
    assert h != "missing" and len(h) == 16
    with open(os.path.join(ROOT, "profiles", "k_sweep_tma_rmat22_dram.json")) as f:
        d = json.load(f)
    assert d["sweep_cu_sha256_16"] == h
    rec = bench._sweep_record()
    assert rec is not None and rec["warp_instructions_per_class"] > 0
    assert bench._traffic_per_pass() == float(d["dram_bytes_per_pass"])


def test_hash_covers_the_kernel_and_not_the_rest(monkeypatch, tmp_path):
    src = open(os.path.join(ROOT, "paper_2307_15969_gb300", "csrc", "sweep.cu")).read()
    base = bench._sweep_hash()

    def hash_of(text):
        d = tmp_path / "paper_2307_15969_gb300" / "csrc"
        d.mkdir(parents=True, exist_ok=True)
        (d / "sweep.cu").write_text(text)
        monkeypatch.setattr(bench, "ROOT", str(tmp_path))
        return bench._sweep_hash()

    # a function added after the launcher: same hash
    i = src.index("cudaError_t launch_sweep_tma(")
    j = src.index("\n}\n", i) + 3
    assert hash_of(src[:j] + "\n// another helper\nstatic int unrelated() { return 1; }\n" + src[j:]) == base
    # a change inside the kernel: another hash
    k = src.index("struct TmaLayout {")
    assert hash_of(src[:k + 20] + " " + src[k + 20:]) != base
    # a change inside the launcher: another hash
    assert hash_of(src[:i + 40] + " " + src[i + 40:]) != base
