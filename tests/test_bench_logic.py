"""Host logic of bench.py that the reported figures rest on (no GPU): the
DRAM-traffic stamp (the captured bytes are reported only for the captured
size and kernel sources, null otherwise), the step roofline's arithmetic
(the slower of the FP64 and HBM ceilings, algorithmic and executed FLOPs),
and the seeded ensemble of the batching workload."""
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


def test_traffic_only_for_the_captured_size_and_sources(bench, monkeypatch):
    sha = bench.sweep_src_sha256()
    assert len(sha) == 64
    monkeypatch.setattr(bench, "SWEEP_DRAM_CAPTURE", {"n": 256, "bytes": 1.25e9, "src_sha256": sha})
    assert bench.sweep_traffic(256) == 1.25e9
    assert bench.sweep_traffic(128) is None
    monkeypatch.setattr(bench, "SWEEP_DRAM_CAPTURE", {"n": 256, "bytes": 1.25e9, "src_sha256": "0" * 64})
    assert bench.sweep_traffic(256) is None


def test_step_roofline_takes_the_slower_ceiling(bench):
    peak = 1.25  # TFLOP/s
    value = 2.0e8
    r = bench.step_roofline(value, peak)
    alg = peak * 1e12 / bench.ALG_FLOPS_PER_CELL_UPDATE
    assert r["bound"] == "fp64" and r["fp64_rate"] == pytest.approx(alg)
    assert r["frac"] == pytest.approx(value / min(alg, r["hbm_rate"]))
    assert r["hbm_rate"] == pytest.approx(r["hbm_gbs"] * 1e9 / bench.STEP_BYTES_PER_CELL)
    assert r["hbm_frac"] == pytest.approx(value * bench.STEP_BYTES_PER_CELL / (r["hbm_gbs"] * 1e9))
    ex = r["executed"]
    exec_flops = 6 * bench.EXEC_FLOPS_PER_FACE + bench.EXEC_STAGE_FLOPS_PER_ZONE
    assert ex["flops_per_cell_update"] == pytest.approx(exec_flops)
    assert ex["frac"] == pytest.approx(value * exec_flops / (peak * 1e12))
    # the kernels execute fewer flops than the method's algorithmic count
    assert exec_flops < bench.ALG_FLOPS_PER_CELL_UPDATE
    # an FP64 peak high enough makes HBM the binding ceiling
    r2 = bench.step_roofline(value, 1e6)
    assert r2["bound"] == "hbm" and r2["frac"] == pytest.approx(value / r2["hbm_rate"])


def test_ensemble_is_seeded_and_prefix_stable(bench):
    e5, boxes5, st5 = bench.ensemble_boxes(5)
    e3, _, st3 = bench.ensemble_boxes(3)
    assert list(e5[:3]) == list(e3)
    assert set(int(e) for e in e5) <= {16, 24, 32, 48, 64, 96, 128}
    for b, st in zip(boxes5, st5):
        assert b["n"][0] == b["n"][1] == b["n"][2]
        assert tuple(st["length"]) == tuple(float(x) for x in b["length"])
    for a, b in zip(st3, st5[:3]):
        for k in ("W", "bx", "by", "bz"):
            assert (a[k] == b[k]).all()
