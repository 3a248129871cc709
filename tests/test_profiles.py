"""The committed ncu summaries (profiles/*.md) that bench.py reads: each names
the ncu command that produced it (run on committed entry points, with the
clock control off), and the per-kernel summaries carry the DRAM traffic of a
full launch and the hash of the kernel sources they were taken on."""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))


def test_profiles_exist():
    names = {os.path.basename(p) for p in PROFILES}
    assert "launches_config1_n30.md" in names
    assert any(n.startswith("gate_tc_k5_c128_") for n in names)


@pytest.mark.parametrize("path", PROFILES, ids=[os.path.basename(p) for p in PROFILES])
def test_profile_names_its_command(path):
    text = open(path).read()
    cmds = [l.strip() for l in text.splitlines() if l.strip().startswith("ncu ")]
    assert cmds, "no ncu command"
    for c in cmds:
        assert "--clock-control none" in c
        assert "_work" not in c
        assert re.search(r"python bench\.py( |$)", c), c


@pytest.mark.parametrize("path", [p for p in PROFILES if not os.path.basename(p).startswith("launches_")],
                         ids=lambda p: os.path.basename(p))
def test_kernel_profile_fields(path):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    text = open(path).read()
    m = re.search(r"^traffic_bytes_per_launch_full: ([0-9.e+]+)", text, re.M)
    assert m and float(m.group(1)) > 0
    h = re.search(r"^source_sha256: ([0-9a-f]{16})$", text, re.M)
    assert h
    # the hash is of this kernel's sources (it may lag a later edit of them,
    # in which case bench.py reports no traffic for the kernel)
    name = re.match(r"(.+)_n\d+\.md$", os.path.basename(path)).group(1)
    assert len(bench.source_hash(name)) == 16
