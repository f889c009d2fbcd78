"""Host logic of bench.py that needs no GPU: the stored DRAM traffic figures are reported only for
the workload and the kernel sources they were captured on."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_host", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


def test_traffic_only_for_its_workload():
    b = _bench()
    for name, t in b.TRAFFIC.items():
        assert b.kernel_traffic(name, "uniform32") is None
        assert b.kernel_traffic(name, "uniform256") is None
        got = b.kernel_traffic(name, t["workload"])
        assert got in (None, t["bytes"])       # None once the kernel sources changed
    assert b.kernel_traffic("k_density<FP64>", "sedov128") is None


def test_traffic_null_after_a_source_change(monkeypatch):
    b = _bench()
    name = "k_forces_fp64"
    monkeypatch.setitem(b.TRAFFIC, name, dict(b.TRAFFIC[name], src_sha256="0" * 64))
    assert b.kernel_traffic(name, "sedov128") is None
