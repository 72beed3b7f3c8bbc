"""GPU HLL fallback and protection floors (App. A) against the oracle.

The 1-2-3 double rarefaction and a 3D expansion box make a Roe-type flux meet
unphysical intermediate states: without protection both sides report an
unphysical state, with protection floors both stay positive, take HLL fluxes
on the same faces and agree zone by zone.  Floors that are never reached
change nothing; the default turbulence workload takes no HLL face."""
import numpy as np
import pytest

from parity import state_err

pytestmark = pytest.mark.gpu

PROT = dict(prot_rho=1e-3, prot_p=1e-4)


@pytest.fixture(scope="module")
def wb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_07452_gb300 import binding
    binding.lib()
    return binding


def double_rarefaction(n):
    W = np.zeros((5, 1, 1, n))
    x = (np.arange(n) + 0.5) / n
    W[0, 0, 0] = 1.0
    W[1, 0, 0] = np.where(x < 0.5, -2.0, 2.0)
    W[4, 0, 0] = 0.4
    return W, np.zeros((1, 1, n + 1)), np.zeros((1, 2, n)), np.zeros((2, 1, n))


def test_double_rarefaction_protected_parity(wb, oracle_mod):
    n = 128
    W, bx, by, bz = double_rarefaction(n)
    L = (1.0, 1e3, 1e3)
    kw = dict(gamma=1.4, bc=(1, 0, 0))
    g = wb.Grid((n, 1, 1), length=L, **kw, **PROT)
    g.load(W, bx, by, bz, primitive=True)
    o = oracle_mod.Grid((n, 1, 1), L, **kw)
    o.set_protection(PROT["prot_rho"], PROT["prot_p"])
    o.load_primitive(W, bx, by, bz)
    tg = g.advance(1000, t_end=0.15)
    to = o.advance(1000, t_end=0.15)
    assert abs(tg - 0.15) < 1e-14 and abs(to - 0.15) < 1e-14
    assert state_err(g.read(), o.read()) < 1e-9
    cg, co = g.counters(), o.counters()
    assert cg["unphysical"] == 0 and co[1] == 0
    assert cg["hll_faces"] == co[2] and co[2] > 0, (cg, co)
    U = g.read()[0][:, 0, 0]
    assert U[0].min() > 0.0


def test_double_rarefaction_unprotected_is_reported(wb, oracle_mod):
    n = 128
    W, bx, by, bz = double_rarefaction(n)
    g = wb.Grid((n, 1, 1), length=(1.0, 1e3, 1e3), gamma=1.4, bc=(1, 0, 0))
    g.load(W, bx, by, bz, primitive=True)
    with pytest.raises(wb.WombatError):
        g.advance(1000, t_end=0.15)


def test_expansion_box_protected_parity(wb, oracle_mod):
    from paper_1701_07452_gb300.initial_conditions import expansion_box
    n = 16
    st = expansion_box(n, 7)
    g = wb.Grid((n, n, n), length=st["length"], **PROT)
    g.load_state(st)
    o = oracle_mod.Grid((n, n, n), st["length"])
    o.set_protection(PROT["prot_rho"], PROT["prot_p"])
    o.load_state(st)
    for _ in range(4):
        g.advance(5)
        o.advance(5)
        assert state_err(g.read(), o.read()) < 1e-9
    cg, co = g.counters(), o.counters()
    assert cg["unphysical"] == 0 and co[1] == 0
    assert co[2] > 0 and abs(cg["hll_faces"] - co[2]) <= 0.01 * co[2], (cg, co)
    assert g.divb_max() < 1e-11


def test_expansion_box_batch_matches_grid(wb):
    from paper_1701_07452_gb300.initial_conditions import expansion_box
    st = [expansion_box(12, 11), expansion_box(16, 7)]
    boxes = [{"n": (12, 12, 12), "length": (1.0, 1.0, 1.0)},
             {"n": (16, 16, 16), "length": (1.0, 1.0, 1.0)}]
    bt = wb.Batch(boxes, **PROT)
    for i, s in enumerate(st):
        bt.load_state(i, s)
    bt.set_steps(-1, 12)
    bt.advance(12)
    # the staged form (general kernel variant with the protection test) gives
    # the persistent form's bits and HLL count
    bs = wb.Batch(boxes, **PROT)
    bs.set_form("staged")
    for i, s in enumerate(st):
        bs.load_state(i, s)
    bs.set_steps(-1, 12)
    bs.advance(12)
    for i, s in enumerate(st):
        g = wb.Grid(boxes[i]["n"], length=boxes[i]["length"], **PROT)
        g.load_state(s)
        g.advance(12)
        for a, b in zip(bt.read(i), g.read()):
            assert np.array_equal(a, b), i
        cb, cg = bt.counters(i), g.counters()
        assert cb["hll_faces"] == cg["hll_faces"] > 0 and cb["unphysical"] == 0
        for a, b in zip(bt.read(i), bs.read(i)):
            assert np.array_equal(a, b), i
        assert bs.counters(i)["hll_faces"] == cb["hll_faces"]


def test_unreached_floors_change_nothing(wb):
    from paper_1701_07452_gb300.initial_conditions import random_box
    st = random_box(12, seed=5)
    out = []
    for kw in ({}, dict(prot_rho=1e-9, prot_p=1e-9)):
        g = wb.Grid((12, 12, 12), length=st["length"], **kw)
        g.load_state(st)
        g.advance(3)
        out.append((g.read(), g.counters()))
    for a, b in zip(out[0][0], out[1][0]):
        assert np.array_equal(a, b)
    assert out[0][1]["hll_faces"] == out[1][1]["hll_faces"] == 0


def test_turbulence_takes_no_hll_face(wb):
    from paper_1701_07452_gb300.initial_conditions import turbulence_box
    st = turbulence_box(32, 2)
    g = wb.Grid((32, 32, 32), length=st["length"])
    g.load_state(st)
    g.advance(5)
    c = g.counters()
    assert c["hll_faces"] == 0 and c["unphysical"] == 0
