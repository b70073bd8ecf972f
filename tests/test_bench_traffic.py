"""The bench line's `traffic` lookup (host only).

profiles/ncu_traffic.json records DRAM bytes per launch of the 2-D workload's level-0 kernels from a
committed ncu capture, with a hash of the sources of those kernels.  The bench reports an entry only
while that hash matches: a change to one of the hashed sources makes `traffic` null until the capture
is taken again, a change to any other source does not.
"""
import json
import os
import shutil

import pytest

import bench


def test_every_hashed_source_exists_and_the_table_names_its_workloads():
    with open(os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")) as fh:
        table = json.load(fh)
    for workload, files in bench.TRAFFIC_SOURCES.items():
        for fn in files:
            assert os.path.exists(os.path.join(bench.CSRC, fn)), fn
        assert workload in table["workloads"]
    for workload, ent in table["workloads"].items():
        assert workload in bench.TRAFFIC_SOURCES
        assert len(ent["sources_sha"]) == 16 and ent["kernels"]
        for kern in ent["kernels"].values():
            assert kern["dram_bytes_per_launch_full_size"] > 0


@pytest.fixture
def tree(tmp_path, monkeypatch):
    """A copy of the kernel sources and of the traffic table that the bench module reads instead."""
    csrc = tmp_path / "csrc"
    shutil.copytree(bench.CSRC, csrc, ignore=shutil.ignore_patterns("*.o", "_build"))
    (tmp_path / "profiles").mkdir()
    shutil.copy(os.path.join(bench.ROOT, "profiles", "ncu_traffic.json"), tmp_path / "profiles")
    monkeypatch.setattr(bench, "CSRC", str(csrc))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    table = json.loads((tmp_path / "profiles" / "ncu_traffic.json").read_text())
    ent = table["workloads"]["2d_1023_k7"]
    ent["sources_sha"] = bench.sources_sha("2d_1023_k7")  # the entry matches the copied sources
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(table))
    return csrc, ent


def test_lookup_follows_the_hashed_sources_only(tree):
    csrc, ent = tree
    kern, val = next(iter(ent["kernels"].items()))
    assert bench.ncu_traffic(kern) == val["dram_bytes_per_launch_full_size"]
    assert bench.ncu_traffic("no_such_kernel") is None
    assert bench.ncu_traffic(kern, "3d_255_var_k9") is None  # no capture recorded for that workload
    # a kernel source outside the hashed set changes: the entry stays valid
    with open(csrc / "sweep3d.cu", "a") as fh:
        fh.write("\n// edited\n")
    assert bench.ncu_traffic(kern) == val["dram_bytes_per_launch_full_size"]
    # one of the hashed sources changes: the entry is no longer reported
    with open(csrc / bench.TRAFFIC_SOURCES["2d_1023_k7"][0], "a") as fh:
        fh.write("\n// edited\n")
    assert bench.ncu_traffic(kern) is None
