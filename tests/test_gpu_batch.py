"""Batching pattern: many independent boxes of uneven sizes advanced by one
persistent kernel with per-box dt (wb_batch_*), or by one launch per stage
(the staged form), compared with the single-box grid path, alone vs in the
mix, graph vs direct launch, persistent vs staged, after autotuning, and
with a barrier wait forced to run out (error status, context still usable);
every box of a mix against the FP64 oracle."""
import numpy as np
import pytest


pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_07452_gb300 import binding
    binding.lib()
    return binding


SIZES = [(8, 8, 8), (12, 10, 9), (16, 16, 16), (10, 14, 12), (6, 6, 6)]


def boxes_and_states(sizes, seed0=100):
    from paper_1701_07452_gb300.initial_conditions import random_box
    boxes, states = [], []
    for i, n in enumerate(sizes):
        st = random_box(n, seed=seed0 + i)
        boxes.append({"n": n, "length": st["length"]})
        states.append(st)
    return boxes, states


def test_batch_matches_single_box_grids(wb):
    boxes, states = boxes_and_states(SIZES)
    bt = wb.Batch(boxes)
    for i, st in enumerate(states):
        bt.load_state(i, st)
    bt.set_steps(-1, 4)
    bt.advance(4)
    for i, st in enumerate(states):
        g = wb.Grid(boxes[i]["n"], length=boxes[i]["length"])
        g.load_state(st)
        g.advance(4)
        # the stage arithmetic is explicitly rounded: the same bits as the grid
        for a, b in zip(bt.read(i), g.read()):
            assert np.array_equal(a, b), i
        c = bt.counters(i)
        assert c["steps"] == 4 and c["unphysical"] == 0
        assert abs(c["t"] - g.counters()["t"]) <= 1e-13 * c["t"]


@pytest.mark.parametrize("form", ["persistent", "staged"])
def test_alone_and_in_the_mix_are_bit_identical(wb, form):
    boxes, states = boxes_and_states(SIZES)
    mix = wb.Batch(boxes, work_budget=8 << 20)  # several workspace groups
    mix.set_form(form)
    assert mix.get_config()["groups"] > 1
    for i, st in enumerate(states):
        mix.load_state(i, st)
    mix.set_steps(-1, 3)
    mix.set_steps(1, 2)  # a box that stops early
    mix.advance(3)
    for i in (0, 1, 2):
        alone = wb.Batch([boxes[i]])
        alone.load_state(0, states[i])
        alone.set_steps(0, 2 if i == 1 else 3)
        alone.advance(3)
        for a, b in zip(alone.read(0), mix.read(i)):
            assert np.array_equal(a, b), i
    assert mix.counters(1)["steps"] == 2 and mix.counters(0)["steps"] == 3


def test_graph_direct_and_autotuned_runs_agree(wb):
    boxes, states = boxes_and_states(SIZES[:4], seed0=200)
    runs = []
    for mode in ("graph", "direct", "tuned", "staged", "staged_direct"):
        bt = wb.Batch(boxes)
        if mode.startswith("staged"):
            bt.set_form("staged")
        for i, st in enumerate(states):
            bt.load_state(i, st)
        if mode == "tuned":
            bt.set_steps(-1, 1000)
            bt.autotune(trial_steps=1)          # real steps, any configuration
            done = bt.counters(0)["steps"]
            assert done <= 30
            bt.set_steps(-1, 30 - done)
            bt.advance(30 - done)
        else:
            bt.set_steps(-1, 30)
            for _ in range(3):
                bt.advance(10, use_graph=mode in ("graph", "staged"))
        runs.append([bt.read(i) for i in range(len(boxes))])
        assert all(bt.counters(i)["steps"] == 30 for i in range(len(boxes)))
    for other in runs[1:]:
        for ra, rb in zip(runs[0], other):
            for a, b in zip(ra, rb):
                assert np.array_equal(a, b)


def test_barrier_timeout_returns_status_and_context_survives(wb):
    boxes, states = boxes_and_states(SIZES[:3], seed0=300)
    bt = wb.Batch(boxes)
    for i, st in enumerate(states):
        bt.load_state(i, st)
    bt.set_steps(-1, 2)
    bt.config(barrier_budget_cycles=1)     # every barrier wait runs out at once
    with pytest.raises(wb.WombatError) as ei:
        bt.advance(2, use_graph=False)
    assert ei.value.code == wb.WB_ERR_TIMEOUT
    # the context still works: a fresh batch advances normally
    ok = wb.Batch(boxes)
    for i, st in enumerate(states):
        ok.load_state(i, st)
    ok.set_steps(-1, 2)
    ok.advance(2)
    assert ok.counters(0)["steps"] == 2


def test_staged_stage_timer(wb):
    """The staged form times every stage but dt; its stage times add up to
    no more than the wall time of the advance."""
    import time
    boxes, states = boxes_and_states(SIZES[:3], seed0=400)
    bt = wb.Batch(boxes)
    bt.set_form("staged")
    for i, st in enumerate(states):
        bt.load_state(i, st)
    bt.set_steps(-1, 3)
    bt.stage_timer(True)
    t0 = time.perf_counter()
    bt.advance(3, use_graph=False)
    wall = time.perf_counter() - t0
    ms = bt.stage_times()
    assert len(ms) == 19 and ms["dt"] == 0.0
    assert ms["pred_sweeps"] > 0 and ms["corr_sweeps"] > 0 and ms["update"] > 0
    assert sum(ms.values()) <= wall * 1e3
    assert all(bt.counters(i)["steps"] == 3 for i in range(3))


def test_mixed_boundaries_both_forms(wb):
    """Periodic boxes (interior-only stages with images) and outflow boxes
    (ghost-ring regions, zero-gradient ghost fill) in one batch: each box
    gives its single grid's bits in both forms."""
    sizes = [(12, 10, 9), (10, 12, 8), (8, 8, 8)]
    bcs = [(0, 0, 0), (1, 1, 1), (0, 1, 0)]
    boxes, states = boxes_and_states(sizes, seed0=500)
    for b, bc in zip(boxes, bcs):
        b["bc"] = bc
    runs = []
    for form in ("persistent", "staged"):
        bt = wb.Batch(boxes)
        bt.set_form(form)
        for i, st in enumerate(states):
            bt.load_state(i, st)
        bt.set_steps(-1, 4)
        bt.advance(4)
        runs.append([bt.read(i) for i in range(len(boxes))])
    for i, (b, st) in enumerate(zip(boxes, states)):
        g = wb.Grid(b["n"], length=b["length"], bc=b["bc"])
        g.load_state(st)
        g.advance(4)
        for a, c, e in zip(runs[0][i], runs[1][i], g.read()):
            assert np.array_equal(a, c) and np.array_equal(a, e), i


@pytest.mark.parametrize("form", ["persistent", "staged"])
def test_batch_boxes_match_the_oracle(wb, oracle_mod, form):
    """Every box of an uneven mix (periodic and outflow, several workspace
    groups) against the FP64 oracle on the same seeded input: within 1e-11
    after one step and 1e-10 after ten, each box on its own CFL dt; totals of
    the periodic boxes to 1e-12."""
    from parity import state_err
    sizes = SIZES + [(20, 18, 16)]
    bcs = [(0, 0, 0), (1, 1, 1), (0, 0, 0), (0, 1, 0), (1, 0, 1), (0, 0, 0)]
    boxes, states = boxes_and_states(sizes, seed0=700)
    for b, bc in zip(boxes, bcs):
        b["bc"] = bc
    bt = wb.Batch(boxes, work_budget=8 << 20)
    bt.set_form(form)
    assert bt.get_config()["groups"] > 1
    for i, st in enumerate(states):
        bt.load_state(i, st)
    orc = []
    for b, st in zip(boxes, states):
        o = oracle_mod.Grid(b["n"], b["length"], bc=b["bc"])
        o.load_state(st)
        orc.append(o)
    t_o = [0.0] * len(orc)
    for steps, tol in ((1, 1e-11), (9, 1e-10)):
        bt.set_steps(-1, steps)
        bt.advance(steps)
        for i, o in enumerate(orc):
            t_o[i] += o.advance(steps)
            assert state_err(bt.read(i), o.read()) < tol, (i, steps)
            c = bt.counters(i)
            assert c["unphysical"] == 0 and c["steps"] == 1 + (steps == 9) * 9
            assert abs(c["t"] - t_o[i]) <= 1e-13 * t_o[i], i
    for i, o in enumerate(orc):
        if boxes[i]["bc"] != (0, 0, 0):
            continue
        g_tot = wb.Grid(boxes[i]["n"], length=boxes[i]["length"])
        U, bx, by, bz, _ = bt.read(i)
        g_tot.load(U, bx, by, bz)
        tg, to = g_tot.totals(), o.totals()
        scale = np.array([abs(to[0])] * 4 + [abs(to[4])] + [1.0] * 3)
        assert np.all(np.abs(tg - to) <= 1e-12 * np.maximum(scale, np.abs(to))), i
