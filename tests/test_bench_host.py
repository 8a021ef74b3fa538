"""Host-side logic of bench.py (no GPU): the traffic records, the bounded
oracle sample and the workload table."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_traffic_records_follow_the_kernel_sources(bench, tmp_path, monkeypatch):
    h = bench.kernel_source_hash()
    path = tmp_path / "traffic.txt"
    path.write_text("# comment: ignored\nkernel_source_hash: %s\n"
                    "workload: fss_160\ndram_bytes_per_launch: 2.5e9\n"
                    "workload: large_256\ndram_bytes_per_launch: 3.0e9\n" % h)
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(path))
    assert bench.load_traffic("fss_160") == 2.5e9
    assert bench.load_traffic("large_256") == 3.0e9
    assert bench.load_traffic("fss_60") is None                 # no record for it
    path.write_text("kernel_source_hash: %s\nworkload: fss_160\ndram_bytes_per_launch: 2.5e9\n" % ("0" * 16))
    assert bench.load_traffic("fss_160") is None                # taken on other kernel sources
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.txt"))
    assert bench.load_traffic("fss_160") is None


def test_oracle_sample_is_bounded(bench):
    for name, wl in bench.WORKLOADS.items():
        systems = bench.oracle_sample_systems(wl)
        assert systems, name
        for s in systems:
            assert s["nx"] * s["ny"] * s["nz"] <= bench.ORACLE_MAX_SITES, (name, s["nx"])
            assert s["lattice"] == wl["lattice"]
    big = bench.bounded_system(dict(lattice="D3Q19", nx=256, ny=256, nz=256, a=0.0))
    assert (big["nx"], big["ny"], big["nz"], big["a"]) == (64, 64, 64, 0.0)
    flat = bench.bounded_system(dict(lattice="D2Q9", nx=4096, ny=4096, nz=1))
    assert (flat["nx"], flat["ny"], flat["nz"]) == (512, 512, 1)
    small = dict(lattice="D3Q19", nx=16, ny=16, nz=16)
    assert bench.bounded_system(small) is small


def test_workload_table(bench):
    for name, wl in bench.WORKLOADS.items():
        assert wl["lattice"] in ("D2Q9", "D3Q19") and wl["precision"] in ("fp32", "fp64"), name
    assert bench.WORKLOADS["fss_160"]["precision"] == "fp32"
