"""The oracle's instrumented FP64 operation counter (the algorithmic FLOPs of
a cell-update, used for the roofline): the counting build must give the
oracle's bits, its per-unit counts must equal hand counts of the formulas of
the simplest stages, and the figures the bench divides by must be the ones
the counter gives."""
import numpy as np
import pytest

from paper_1701_07452_gb300.initial_conditions import random_box, turbulence_box


def test_counting_build_gives_the_same_bits(oracle_mod):
    for prot in (0.0, 0.97):
        st = random_box((10, 8, 9), seed=17)
        runs = []
        for counting in (False, True):
            g = oracle_mod.Grid((10, 8, 9), st["length"], counting=counting)
            g.load_state(st)
            if prot:
                g.set_protection(prot, 0.0)
            g.advance(3)
            runs.append(g.read() + (g.counters(), g.dt()))
        for a, b in zip(*runs):
            if isinstance(a, np.ndarray):
                assert np.array_equal(a, b)
            else:
                assert a == b


def test_counts_of_the_simplest_stages(oracle_mod):
    """Hand counts of the printed formulas (Steps 4/11, 10, 3/9 and the
    reference EMF): constrained transport b - tau ((E+ - E)/da - (E+ - E)/db)
    is 7 operations a face; the update (((u - cx dF) - cy dG) - cz dH) is 9 a
    component, 45 a zone; a corner EMF is 18 (the eight candidate
    differences of both upwind sides, the quarter-weighted sum of the four
    face EMFs, the two quarter-weighted brackets and the two sums that join
    the three parts; the upwind choices are free); the reference EMF is 3
    divisions, 6 products and 3 differences -- except where the density is
    exactly 1, where the divisions are identity operations and are not
    counted."""
    st = turbulence_box((12, 12, 12), seed=2)   # density exactly 1 at load
    g = oracle_mod.Grid((12, 12, 12), st["length"], counting=True)
    g.load_state(st)
    oracle_mod.flop_reset()
    g.advance(1)
    first = oracle_mod.flop_report()
    oracle_mod.flop_reset()
    g.advance(1)
    second = oracle_mod.flop_report()
    per = {k: f / u for k, (f, u) in second.items() if u}
    assert per["ct"] == 7.0
    assert per["update"] == 45.0
    assert per["edge"] == 18.0
    assert per["eref"] == 12.0
    assert first["eref"][0] / first["eref"][1] == 9.0
    assert per["limit"] == 0.0          # minmod with beta = 1: comparisons only
    assert second["hll"] == (0, 0) and second["none"][0] == 0


def test_bench_divides_by_the_counted_figures(oracle_mod):
    """bench.py's algorithmic FLOPs per sweep face and per cell-update are the
    counter's (oracle/count_flops.py, on the bench workload's data at 64^3);
    a 32^3 count of the same data agrees within 1 %."""
    import bench
    from oracle import count_flops
    r = count_flops.count(32, 1)
    assert abs(r["flops_per_sweep_face"] / bench.ALG_FLOPS_PER_FACE - 1.0) < 0.01
    assert abs(r["flops_per_cell_update"] / bench.ALG_FLOPS_PER_CELL_UPDATE - 1.0) < 0.01


@pytest.mark.parametrize("n", [8])
def test_count_is_per_interior_unit(oracle_mod, n):
    """Every section's units grow with the box as its stage's index range
    does, so the per-unit means do not depend on the ghost-ring recompute:
    the per-face sweep count on two box sizes of the same kind of data agrees
    to 2 %."""
    from oracle import count_flops
    a = count_flops.count(n, 1)["flops_per_sweep_face"]
    b = count_flops.count(2 * n, 1)["flops_per_sweep_face"]
    assert abs(a / b - 1.0) < 0.02
