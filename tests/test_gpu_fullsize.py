"""Parity at the benchmark's full size: the 256^3 periodic turbulence box of
the bench (rho = 1, P = 1, solenoidal velocity modes 1 <= |k| <= 8 at rms
Mach 1, mean field along x at beta 100, 10 % field perturbation; seed 2),
single grid in the launch configuration bench.py times.

The oracle runs one full step of the whole box on the host cores (seconds),
so every zone is compared after one step, with the 1-step tolerance of the
parity tests.  Later steps are checked by what holds at any size: every
conserved total, div b at roundoff, and the CFL time step of the evolved
state against the oracle's dt of the same state."""
import numpy as np
import pytest

from parity import state_err

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
