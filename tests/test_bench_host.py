"""Host logic of bench.py that its roofline figures depend on (no GPU)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1702_04487_gb300 import workloads as W  # noqa: E402


def test_algorithmic_bytes_follow_the_storage_layout():
    """Every stored population is read once and written once per update:
    2-D f[9] and g[5]; 3-D f[19] and g[7]; FP16 storage keeps g_0 in FP32."""
    f32, f16 = 4, 2
    assert bench.BYTES_PER_LUP["2d"] == 2 * (9 + 5) * f32
    assert bench.BYTES_PER_LUP["2d16"] == 2 * (9 * f16 + 4 * f16 + f32)
    assert bench.BYTES_PER_LUP["3d32"] == 2 * (19 + 7) * f32
    assert bench.BYTES_PER_LUP["3d16"] == 2 * (19 * f16 + 6 * f16 + f32)


def test_lattice_kinds():
    assert bench.lattice_kind(W.cfg1()) == "2d"
    assert bench.lattice_kind(dict(W.cfg1(), precision=1)) == "2d16"
    assert bench.lattice_kind(W.cfg4(precision=0, nx=8, ny=8, nz=8)) == "3d32"
    assert bench.lattice_kind(W.cfg4(precision=1, nx=8, ny=8, nz=8)) == "3d16"


@pytest.mark.parametrize("name", ["cfg2", "cfg2h", "big", "cfg3", "cfg4", "cfg4h", "e1"])
def test_every_workload_builds(name):
    ps, desc = bench.workload(name)
    assert ps and desc
    cells = sum(bench.cells_of(p) for p in ps)
    assert cells > 1_000_000  # larger than a toy: the bench lines are throughput lines
    if name.endswith("h"):
        assert all(p["precision"] == 1 for p in ps)


def test_traffic_records_are_reported_only_for_their_sources(monkeypatch):
    """A recorded ncu traffic figure is reported only at a recorded chunk and
    for the sources it was measured on; the current records lie near the
    algorithmic bytes (far above them would mean wasted re-reads)."""
    for name, rec in bench.NCU_TRAFFIC.items():
        ps, _ = bench.workload(name)
        for chunk, traffic in rec["bytes_per_step"].items():
            assert chunk in tuple(range(8, 129, 8)) + (160, 192, 256, 0, -1, -2, -3, -4, -5)
            got = bench.recorded_traffic(name, ps, [{"chunk": chunk}])
            if rec["kernel_sha"] == bench.kernel_hash(ps):
                assert got == traffic
                cells = sum(bench.cells_of(p) for p in ps)
                alg = bench.BYTES_PER_LUP[bench.lattice_kind(ps[0])] * cells
                assert 0.9 * alg < traffic < 1.2 * alg, (name, chunk, traffic / alg)
            else:
                assert got is None
        assert bench.recorded_traffic(name, ps, [{"chunk": 7}]) is None
        monkeypatch.setattr(bench, "kernel_hash", lambda params: "0" * 16)
        chunk = next(iter(rec["bytes_per_step"]))
        assert bench.recorded_traffic(name, ps, [{"chunk": chunk}]) is None
        monkeypatch.undo()
    assert bench.recorded_traffic("no-such-workload", W.cfg2_sweep(), [{"chunk": 64}]) is None
