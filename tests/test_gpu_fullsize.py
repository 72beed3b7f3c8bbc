"""Parity at the benchmark's full size: the 256^3 periodic turbulence box of
the bench (rho = 1, P = 1, solenoidal velocity modes 1 <= |k| <= 8 at rms
Mach 1, mean field along x at beta 100, 10 % field perturbation; seed 2),
single grid in the launch configuration bench.py times.

The oracle runs one full step of the whole box on the host cores (seconds),
so every zone is compared after one step, with the 1-step tolerance of the
parity tests.  Later steps are checked by what holds at any size: every
conserved total, div b at roundoff, and the CFL time step of the evolved
state against the oracle's dt of the same state.  The full 100 steps of the
box, every zone against the oracle, take about ten minutes of oracle time on
16 host cores and run when WB_FULLSIZE_LONG=1 is set."""
import os

import numpy as np
import pytest

from parity import TIGHT, state_err

pytestmark = pytest.mark.gpu

N = 256
SEED = 2


@pytest.fixture(scope="module")
def wb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_07452_gb300 import binding
    binding.lib()
    return binding


@pytest.fixture(scope="module")
def state():
    from paper_1701_07452_gb300.initial_conditions import turbulence_box
    return turbulence_box(N, SEED)


def test_full_size_one_step_every_zone(wb, oracle_mod, state):
    n = (N, N, N)
    g = wb.Grid(n, length=state["length"])
    g.load_state(state)
    o = oracle_mod.Grid(n, state["length"])
    o.load_state(state)
    d0 = o.dt()
    assert abs(g.dt() - d0) <= 1e-14 * d0
    g.advance(1)
    o.advance(1)
    assert state_err(g.read(), o.read()) < 1e-11
    assert abs(g.counters()["last_dt"] - d0) <= 1e-14 * d0


def test_full_size_ten_steps_properties(wb, oracle_mod, state):
    n = (N, N, N)
    g = wb.Grid(n, length=state["length"])
    g.load_state(state)
    U0, bx0, by0, bz0, _ = g.read()
    vol = float(np.prod([state["length"][a] / n[a] for a in range(3)]))
    scale = [np.abs(U0[c]).sum() * vol for c in range(5)]
    scale += [np.abs(b).sum() * vol for b in (bx0, by0, bz0)]
    bmax = max(np.abs(bx0).max(), np.abs(by0).max(), np.abs(bz0).max())
    t0 = g.totals()
    g.advance(10)
    t1 = g.totals()
    for c in range(8):
        assert abs(t1[c] - t0[c]) <= 1e-13 * scale[c], (c, t1[c], t0[c])
    assert g.divb_max() <= 1e-13 * bmax * N / state["length"][0]
    assert g.counters()["unphysical"] == 0 and g.counters()["floor_hits"] == 0
    # the dt the next step takes equals the oracle's dt of the same state
    U, bx, by, bz, _ = g.read()
    o = oracle_mod.Grid(n, state["length"])
    o.load(U, bx, by, bz)
    d_or = o.dt()
    assert abs(g.dt() - d_or) <= 1e-14 * d_or


def test_full_size_batch_equals_grid(wb, state):
    """The bench's box advanced through the batch path (staged form, the
    sweep inside the batch kernel) gives the single grid's bits."""
    n = (N, N, N)
    g = wb.Grid(n, length=state["length"])
    g.load_state(state)
    g.advance(2)
    bt = wb.Batch([{"n": n, "length": state["length"]}])
    bt.set_form("staged")
    bt.load_state(0, state)
    bt.set_steps(0, 2)
    bt.advance(2)
    for a, b in zip(bt.read(0), g.read()):
        assert np.array_equal(a, b)


@pytest.mark.skipif(os.environ.get("WB_FULLSIZE_LONG") != "1",
                    reason="about ten minutes of oracle time: set WB_FULLSIZE_LONG=1")
def test_full_size_hundred_steps_every_zone(wb, oracle_mod, state):
    """The bench's 256^3 box after 100 steps, every zone against the oracle
    at the 100-step tolerance (1e-8 per zone, under both guards), the time
    reached to 1e-11 and the conserved totals to 1e-12 of their scale."""
    n = (N, N, N)
    g = wb.Grid(n, length=state["length"])
    g.load_state(state)
    o = oracle_mod.Grid(n, state["length"])
    o.load_state(state)
    t_g = g.advance(100)
    t_o = o.advance(100)
    assert abs(t_g - t_o) <= 1e-11 * t_o
    gs, os_ = g.read(), o.read()
    err, err_tight = state_err(gs, os_), state_err(gs, os_, TIGHT)
    print(f"256^3 x 100 steps: max rel err {err:.3e} (guard 1e-3 of the box maximum), "
          f"{err_tight:.3e} (guard 1e-6); t = {t_g:.6f}")
    assert err < 1e-8 and err_tight < 1e-8
    tg, to = g.totals(), o.totals()
    scale = np.array([abs(to[0])] * 4 + [abs(to[4])] + [1.0] * 3)
    assert np.all(np.abs(tg - to) <= 1e-12 * np.maximum(scale, np.abs(to)))
    assert g.counters()["unphysical"] == 0
