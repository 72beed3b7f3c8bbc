"""Validation problems of Sec. "Test Calculations" on the GPU path: parity with
the oracle on small boxes, then the properties that hold at any size
(exact-solution convergence, conservation, div b, positivity) at sizes the
oracle cannot run in a test, up to the paper's own blast-wave grid."""
import numpy as np
import pytest

from parity import rel_err, state_err, state_err_vec
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


def l1_vector_norm(a, b):
    dq = [np.abs(a[0][c] - b[0][c]).mean() for c in range(5)] + \
         [np.abs(a[4][c] - b[4][c]).mean() for c in range(3)]
    return float(np.sqrt(np.sum(np.square(dq))))


def test_cpaw_parity_and_convergence(wb, oracle_mod):
    n = 16
    st = ic.cpaw_box(n)
    g = wb.Grid((2 * n, n, n), length=st["length"])
    g.load_state(st)
    o = oracle_mod.Grid((2 * n, n, n), st["length"])
    o.load_state(st)
    assert abs(g.advance(100000, t_end=1.0) - 1.0) < 1e-13
    o.advance(100000, t_end=1.0)
    assert state_err(g.read(), o.read()) < 1e-9
    errs = []
    for n in (16, 32, 64):
        st = ic.cpaw_box(n)
        g = wb.Grid((2 * n, n, n), length=st["length"])
        g.load_state(st)
        s0 = g.read()
        g.advance(100000, t_end=1.0)
        errs.append(l1_vector_norm(g.read(), s0))
        assert g.counters()["unphysical"] == 0
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0, errs
    assert errs[2] < 0.002, errs


def test_field_loop(wb, oracle_mod):
    n = 32
    st = ic.field_loop_box(n)
    g = wb.Grid((2 * n, n, 1), length=st["length"])
    g.load_state(st)
    o = oracle_mod.Grid((2 * n, n, 1), st["length"])
    o.load_state(st)
    # 40 steps: later, where B_t crosses zero with a jump the two sides can
    # take different branches of the degenerate transverse direction
    # (beta = 1/sqrt2 below |B_t|^2 = 1e-24 ...) and then differ at 1e-4 of
    # the field scale
    g.advance(40)
    o.advance(40)
    assert state_err_vec(g.read(), o.read()) < 1e-8
    # the paper's grid, two periods
    n = 128
    st = ic.field_loop_box(n)
    g = wb.Grid((2 * n, n, 1), length=st["length"])
    g.load_state(st)
    em = [0.5 * float((g.read()[4] ** 2).sum())]
    for k in range(1, 9):
        g.advance(100000, t_end=0.25 * k)
        em.append(0.5 * float((g.read()[4] ** 2).sum()))
    assert all(em[i + 1] <= em[i] for i in range(8)), em
    assert em[-1] / em[0] > 0.536, em     # more than the oracle keeps at 128 x 64
    assert g.divb_max() < 1e-13


@pytest.mark.parametrize("name", ["briowu", "rj2a", "rj4a"])
def test_shock_tube_parity_and_convergence(wb, oracle_mod, name):
    sp = ic.SHOCK_TUBES[name]
    kw = dict(gamma=sp["gamma"], bc=(1, 0, 0))
    n = 128
    st = ic.shock_tube_1d(name, n)
    g = wb.Grid((n, 1, 1), length=st["length"], **kw)
    g.load_state(st)
    o = oracle_mod.Grid((n, 1, 1), st["length"], **kw)
    o.load_state(st)
    g.advance(100000, t_end=sp["t"])
    o.advance(100000, t_end=sp["t"])
    # v_z, B_z (and v_y, B_y in 4a) are zero or noise in exact arithmetic:
    # vector components are held to the vector's scale
    assert state_err_vec(g.read(), o.read()) < 1e-9
    rho = {}
    for n in (256, 512, 1024, 2048):
        st = ic.shock_tube_1d(name, n)
        g = wb.Grid((n, 1, 1), length=st["length"], **kw)
        g.load_state(st)
        g.advance(100000, t_end=sp["t"])
        rho[n] = g.read()[0][0, 0, 0]
        assert rho[n].min() > 0.0
    errs = [float(np.abs(rho[n] - rho[2048].reshape(n, -1).mean(axis=1)).mean()) for n in (256, 512, 1024)]
    assert errs[0] / errs[1] > 1.5 and errs[1] / errs[2] > 1.5, errs


def test_blast_wave_parity(wb, oracle_mod):
    # a milder blast (beta = 2 outside, P_in = 10), off-centre, agrees zone
    # by zone over its whole run.  (Centred, the mass flux on the symmetry
    # planes is rounding noise whose sign picks the upwind side of the corner
    # EMF, a choice that matters at the size of the local gradient.)
    st = ic.blast_box(16, 24, 16, b0=1.0, p_in=10.0, shift=(0.31, 0.17, 0.23))
    g = wb.Grid((16, 24, 16), length=st["length"])
    g.load_state(st)
    o = oracle_mod.Grid((16, 24, 16), st["length"])
    o.load_state(st)
    g.advance(100000, t_end=0.05)
    o.advance(100000, t_end=0.05)
    assert state_err_vec(g.read(), o.read()) < 1e-8
    # the paper's parameters (beta = 0.02, pressure floors reached): the
    # floored zones' pressure is the rounding of E - ke - B^2/2 and 1/a^2 of
    # their Roe states amplifies it, so zone-by-zone agreement holds for the
    # first step; floor hits and HLL faces agree over the run
    st = ic.blast_box(16, 24, 16)
    g = wb.Grid((16, 24, 16), length=st["length"], prot_rho=1e-3, prot_p=1e-3)
    g.load_state(st)
    o = oracle_mod.Grid((16, 24, 16), st["length"])
    o.set_protection(1e-3, 1e-3)
    o.load_state(st)
    dt1 = o.dt()
    g.advance(1)
    o.advance(1)
    assert state_err_vec(g.read(), o.read()) < 1e-10
    g.advance(100000, t_end=0.02)
    o.advance(100000, t_end=0.02 - dt1)
    cg, co = g.counters(), o.counters()
    assert cg["floor_hits"] == co[0] > 0 and cg["hll_faces"] == co[2] > 0


def test_blast_wave_paper_grid(wb):
    """200 x 300 x 200 zones to t = 0.02 (Sec. "MHD Blast Wave")."""
    st = ic.blast_box(200, 300, 200)
    g = wb.Grid((200, 300, 200), length=st["length"], prot_rho=1e-3, prot_p=1e-3)
    g.load_state(st)
    tot0 = g.totals()
    assert abs(g.advance(100000, t_end=0.02) - 0.02) < 1e-15
    tot = g.totals()
    for c in (0, 1, 2, 3, 5, 6, 7):
        assert abs(tot[c] - tot0[c]) <= 1e-11 * max(abs(tot0[c]), tot0[0]), c
    U, bx, by, bz, B = g.read()
    p = (2.0 / 3.0) * (U[4] - 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / U[0] - 0.5 * (B ** 2).sum(0))
    assert U[0].min() > 0.0 and p.min() > 0.0
    assert g.divb_max() < 1e-9
    c = g.counters()
    assert c["unphysical"] == 0


@pytest.mark.parametrize("name", ["rj2a", "rj4a"])
def test_rotated_shock_tube_3d(wb, oracle_mod, name):
    """RJ95 2a / 4a in 3D (Sec. "RJ95 2a", "RJ95 4a"): the tube on a cube of
    128 zones a side, its normal along (1, 1, 1)/sqrt 3, equally inclined to
    the three primary planes (reading R27), outflow on every axis, face field
    from an edge potential (div b = 0).  On a 24^3 cube the GPU follows the
    oracle zone by zone (vector components held to their vector's scale, as
    for the 1D tubes).  At 128^3 and the paper's end time the density along
    the main diagonal, sampled at s = n . (x - centre), must agree with the
    1D driver's 2048-zone solution as closely as the 1D driver at 128 zones
    does (L1 within 1.5x of it over |s| <= 0.45, where no wave has met the
    outflow faces); div b stays at rounding level and pressure positive.
    The parity part adds a uniform transverse velocity (0.1 e2 + 0.3 e3) to
    both states: with the paper's states the velocity is exactly zero on one
    or both sides, the mass flux ahead of each front is rounding noise, and
    its sign picks the upwind side of the corner EMF differently on the two
    implementations (the tie rule of the upwinded EMF)."""
    import math
    import test_oracle_validation as tov
    sp = ic.SHOCK_TUBES[name]
    kw = dict(gamma=sp["gamma"], bc=(1, 1, 1))
    n = 24
    st = ic.shock_tube_rotated(name, n, boost=(0.1, 0.3))
    g = wb.Grid((n, n, n), length=st["length"], **kw)
    g.load_state(st)
    o = oracle_mod.Grid((n, n, n), st["length"], **kw)
    o.load_state(st)
    g.advance(100000, t_end=0.3 * sp["t"])
    o.advance(100000, t_end=0.3 * sp["t"])
    assert state_err_vec(g.read(), o.read()) < 1e-9
    n = 128
    st = ic.shock_tube_rotated(name, n)
    g = wb.Grid((n, n, n), length=st["length"], **kw)
    g.load_state(st)
    assert abs(g.advance(100000, t_end=sp["t"]) - sp["t"]) < 1e-13
    c = g.counters()
    assert c["unphysical"] == 0 and c["floor_hits"] == 0
    U, bx, by, bz, B = g.read()
    bmax = max(np.abs(b).max() for b in (bx, by, bz))
    div = np.diff(bx, axis=2) + np.diff(by, axis=1) + np.diff(bz, axis=0)
    assert np.abs(div[1:-1, 1:-1, 1:-1]).max() <= 1e-12 * bmax
    idx = np.arange(n)
    rho3 = U[0][idx, idx, idx]
    s3 = math.sqrt(3.0) * ((idx + 0.5) / n - 0.5)
    ref, _ = tov.run_line(oracle_mod, name, 2048)
    x1 = (np.arange(2048) + 0.5) / 2048 - 0.5
    coarse, _ = tov.run_line(oracle_mod, name, n)
    xc = (np.arange(n) + 0.5) / n - 0.5
    m, mc = np.abs(s3) <= 0.45, np.abs(xc) <= 0.45
    err3 = float(np.abs(rho3[m] - np.interp(s3[m], x1, ref[:, 0])).mean())
    err1 = float(np.abs(coarse[mc, 0] - np.interp(xc[mc], x1, ref[:, 0])).mean())
    assert err3 < 1.5 * err1, (err3, err1)
