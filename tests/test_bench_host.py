"""Host-side bookkeeping of bench.py and profiles/ (CPU, no GPU).

The JSON line's `traffic` fields come from ncu captures summarised under profiles/;
bench.py applies a capture's DRAM-to-algorithmic ratio only while the captured kernel's
definition is unchanged (a hash of its __global__ function's text).  These tests keep
that chain consistent.
"""
import glob
import os
import re

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("kind", sorted(bench.PROFILED_TRAFFIC))
def test_traffic_entries_name_existing_kernels_and_profiles(kind):
    e = bench.PROFILED_TRAFFIC[kind]
    assert os.path.exists(os.path.join(ROOT, e["source"])), e["source"]
    assert os.path.exists(os.path.join(ROOT, e["profile"])), e["profile"]
    assert bench._kernel_text(e["source"], e["kernel"]) is not None, e["kernel"]
    assert 0.0 < e["ratio"] < 1.5
    assert re.fullmatch(r"[0-9a-f]{16}", e["sha256"])
    assert e["sha256"] in open(os.path.join(ROOT, e["profile"])).read(), "profile records the hash"


def test_kernel_text_is_one_whole_definition():
    t = bench._kernel_text("paper_2502_06959_gb300/csrc/accum.cu", "finalize_kernel")
    assert t.startswith("__global__") and t.rstrip().endswith("}")
    assert t.count("{") == t.count("}")
    assert bench._kernel_text("paper_2502_06959_gb300/csrc/accum.cu", "no_such_kernel") is None


def test_traffic_is_gated_on_the_captured_kernel(monkeypatch):
    src, kern = "paper_2502_06959_gb300/csrc/accum.cu", "finalize_kernel"
    e = {"ratio": 0.9, "source": src, "kernel": kern, "sha256": bench._kernel_hash(src, kern),
         "profile": "profiles/none.md"}
    monkeypatch.setitem(bench.PROFILED_TRAFFIC, "probe", e)
    assert bench.traffic_per_launch("probe", 1000.0) == pytest.approx(900.0)
    # a changed kernel: no traffic figure
    monkeypatch.setitem(bench.PROFILED_TRAFFIC, "probe", dict(e, sha256="0" * 16))
    assert bench.traffic_per_launch("probe", 1000.0) is None
    assert bench.traffic_per_launch("no-such-kernel", 1000.0) is None


def test_profiles_name_their_commands_and_never_lock_clocks():
    files = sorted(glob.glob(os.path.join(ROOT, "profiles", "*")))
    assert files, "no profiles"
    for f in files:
        assert f.endswith((".md", ".txt")), f
        text = open(f).read()
        assert os.path.getsize(f) < 16 * 1024, f
        assert "Command" in text, f
        commands = re.sub(r"\\\n\s*", " ", text).splitlines()          # join continued lines
        ncu = [l for l in commands if re.match(r"\s*ncu\s", l)]
        assert ncu, f
        for l in ncu:
            assert "--clock-control none" in l, (f, l)
