"""2D CTU+CT (Sec. "MHD in Two Dimensions") on the GPU: a box one zone thick
in z with periodic z is stored as one plane (z stride 0).  It must give
bit-for-bit the result of the full 3D layout of the same box (outflow z,
5 ghost layers), match the oracle, and run the Orszag-Tang vortex on the
paper's 192 x 192 grid conserving every total."""
import numpy as np
import pytest

from parity import state_err
from paper_1701_07452_gb300 import initial_conditions as ic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_07452_gb300 import binding
    binding.lib()
    return binding


def test_flat_layout_equals_3d_layout(wb):
    st = ic.random_box_2d(24, 16, seed=5)
    out = []
    for bc_z in (0, 1):   # periodic z: one plane; outflow z: the 3D layout
        g = wb.Grid((24, 16, 1), patches=(2, 2, 1), length=st["length"], bc=(0, 0, bc_z))
        g.load_state(st)
        g.advance(10)
        out.append((g.read(), g.counters(), g.nbytes))
    for a, b in zip(out[0][0], out[1][0]):
        assert np.array_equal(a, b)
    assert out[0][1]["t"] == out[1][1]["t"]
    assert out[0][2] * 4 < out[1][2]      # one plane instead of 11


def test_flat_layout_parity(wb, oracle_mod):
    st = ic.random_box_2d(24, 16, seed=6)
    g = wb.Grid((24, 16, 1), length=st["length"])
    g.load_state(st)
    o = oracle_mod.Grid((24, 16, 1), st["length"])
    o.load_state(st)
    g.advance(1)
    o.advance(1)
    assert state_err(g.read(), o.read()) < 1e-11
    g.advance(9)
    o.advance(9)
    assert state_err(g.read(), o.read()) < 1e-10
    st = ic.orszag_tang_box(32)
    g = wb.Grid((32, 32, 1), length=st["length"])
    g.load_state(st)
    o = oracle_mod.Grid((32, 32, 1), st["length"])
    o.load_state(st)
    g.advance(20)
    o.advance(20)
    assert state_err(g.read(), o.read()) < 1e-9


def test_orszag_tang_paper_grid(wb):
    n = 192
    st = ic.orszag_tang_box(n)
    g = wb.Grid((n, n, 1), length=st["length"])
    g.load_state(st)
    tot0 = g.totals()
    assert abs(g.advance(100000, t_end=0.5) - 0.5) < 1e-15
    tot = g.totals()
    for c in range(8):
        assert abs(tot[c] - tot0[c]) <= 1e-12 * max(abs(tot0[c]), tot0[0]), (c, tot[c], tot0[c])
    U, bx, by, bz, B = g.read()
    p = (2.0 / 3.0) * (U[4] - 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / U[0] - 0.5 * (B ** 2).sum(0))
    assert U[0].min() > 0.0 and p.min() > 0.0
    assert g.divb_max() < 1e-12
    c = g.counters()
    assert c["unphysical"] == 0 and c["floor_hits"] == 0
