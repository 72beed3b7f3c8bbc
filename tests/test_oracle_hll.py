"""Pins of the oracle's HLL flux and protection floor (App. A: the HLL flux
with speeds b+ and b-, switched on where the protection floor is exceeded).

What fixes the oracle here, independent of its own code:
  * consistency: the HLL flux of a uniform state is the flux of that state
    (the printed numerator, with +b- F(q_R), fails this; reading R22);
  * upwinding: with all signal speeds of one sign the HLL flux is the flux of
    the upwind zone alone, whatever the downwind state;
  * the Einfeldt 1-2-3 double rarefaction (Toro's test 2): a Roe-type flux
    produces negative densities or pressures there (the failure the paper's
    protection floor exists for); with protection the run stays positive and
    converges to the exact Euler solution (tests/exact_riemann.py, pinned to
    Toro's printed star values);
  * an all-HLL run of the Sod problem converges to the exact solution;
  * floors that are never reached leave the scheme bit-identical.
"""
import numpy as np
import pytest

import exact_riemann

GAMMA = 5.0 / 3.0


def pencil(states, b):
    cells = np.array(states, dtype=np.float64)
    return cells, np.full(cells.shape[0] + 1, float(b))


def cons(rho, vn, vt1, vt2, p, bn, bt1, bt2, gamma=GAMMA):
    e = p / (gamma - 1.0) + 0.5 * rho * (vn * vn + vt1 * vt1 + vt2 * vt2) + \
        0.5 * (bn * bn + bt1 * bt1 + bt2 * bt2)
    return [rho, rho * vn, rho * vt1, rho * vt2, e, bn, bt1, bt2]


def test_hll_flux_of_uniform_state_is_its_flux(oracle_mod):
    q = cons(1.3, 0.4, -0.2, 0.1, 0.9, 0.6, 0.3, -0.5)
    cells, bf = pencil([q] * 8, 0.6)
    tvd, nh0 = oracle_mod.flux_pencil(cells, bf, 0.3, 1.7, GAMMA, with_hll=True)
    hll, nh = oracle_mod.flux_pencil(cells, bf, 0.3, 1.7, GAMMA, prot_rho=1e30, with_hll=True)
    assert nh0 == 0 and nh == 5          # faces 2..6 of 8 cells
    # the MHDTVD flux of a uniform state is F(q) (all alpha_k = 0)
    for f in range(2, 7):
        assert np.allclose(hll[f], tvd[f], rtol=2e-15, atol=2e-15), (hll[f], tvd[f])
    # mass flux = rho vn exactly as a number the test knows
    assert abs(hll[4][0] - 1.3 * 0.4) <= 1e-15


@pytest.mark.parametrize("direction", [1.0, -1.0])
def test_hll_upwinds_supersonic_flow(oracle_mod, direction):
    # |vn| = 6 exceeds every fast speed (< 2.2 here) on both sides
    qa = cons(1.0, 6.0 * direction, 0.3, 0.0, 1.0, 0.5, 0.8, 0.2)
    qb = cons(0.4, 6.0 * direction, -0.5, 0.1, 0.3, 0.5, -0.3, 0.6)
    qc = cons(2.0, 6.0 * direction, 0.1, 0.9, 3.0, 0.5, 0.0, -0.7)
    up_state = qa if direction > 0 else qb
    cells, bf = pencil([qa, qa, qa, qb, qb, qb], 0.5)
    hll, _ = oracle_mod.flux_pencil(cells, bf, 0.01, 50.0, GAMMA, prot_rho=1e30, with_hll=True)
    ref_cells, rbf = pencil([up_state] * 6, 0.5)
    ref = oracle_mod.flux_pencil(ref_cells, rbf, 0.01, 50.0, GAMMA)
    assert np.allclose(hll[3], ref[3], rtol=4e-16 * 8, atol=1e-15)
    # the downwind state does not enter
    cells2 = cells.copy()
    if direction > 0:
        cells2[3:] = qc
    else:
        cells2[:3] = qc
    hll2, _ = oracle_mod.flux_pencil(cells2, bf, 0.01, 50.0, GAMMA, prot_rho=1e30, with_hll=True)
    assert np.allclose(hll2[3], ref[3], rtol=4e-16 * 8, atol=1e-15)


def riemann_run(oracle_mod, n, W_left, W_right, t_end, prot=None, gamma=1.4):
    W = np.zeros((5, 1, 1, n))
    x = (np.arange(n) + 0.5) / n
    for c, (a, b) in enumerate(zip(W_left, W_right)):
        W[c, 0, 0] = np.where(x < 0.5, a, b)
    g = oracle_mod.Grid((n, 1, 1), (1.0, 1e3, 1e3), gamma=gamma, bc=(1, 0, 0))
    if prot is not None:
        g.set_protection(*prot)
    g.load_primitive(W, np.zeros((1, 1, n + 1)), np.zeros((1, 2, n)), np.zeros((2, 1, n)))
    g.advance(100000, t_end=t_end)
    U = g.read()[0][:, 0, 0]
    rho = U[0]
    p = (gamma - 1.0) * (U[4] - 0.5 * U[1] ** 2 / rho)
    return x, rho, p, g.counters()


def test_double_rarefaction_needs_protection(oracle_mod):
    left, right = (1.0, -2.0, 0.0, 0.0, 0.4), (1.0, 2.0, 0.0, 0.0, 0.4)
    with pytest.raises(RuntimeError):
        riemann_run(oracle_mod, 100, left, right, 0.15)
    errs = []
    for n in (100, 200, 400):
        x, rho, p, cnt = riemann_run(oracle_mod, n, left, right, 0.15, prot=(1e-3, 1e-4))
        assert cnt[1] == 0 and cnt[2] > 0, cnt
        assert rho.min() > 0.0 and p.min() > 0.0
        ex = exact_riemann.sample(x, 0.15, 0.5, 1.0, -2.0, 0.4, 1.0, 2.0, 0.4, 1.4)
        errs.append(float(np.abs(rho - ex[0]).mean()))
    assert errs[0] < 0.012 and errs[2] < 0.0045, errs
    assert errs[1] < errs[0] / 1.4 and errs[2] < errs[1] / 1.4, errs


def test_all_hll_sod_converges(oracle_mod):
    errs = []
    for n in (100, 200, 400):
        x, rho, p, cnt = riemann_run(oracle_mod, n, (1.0, 0, 0, 0, 1.0), (0.125, 0, 0, 0, 0.1),
                                     0.2, prot=(1e30, 0.0))
        assert cnt[2] > 0
        ex = exact_riemann.sample(x, 0.2, 0.5, 1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4)
        errs.append(float(np.abs(rho - ex[0]).mean()))
    # first-order HLL: converges, more diffusive than the MHDTVD run of the
    # same problem (test_oracle_physics: 0.006 at n = 100)
    assert 0.008 < errs[0] < 0.025 and errs[2] < 0.009, errs
    assert errs[1] < errs[0] / 1.4 and errs[2] < errs[1] / 1.4, errs


def test_unreached_protection_is_bit_identical(oracle_mod):
    from paper_1701_07452_gb300.initial_conditions import random_box
    st = random_box(8, 3)
    out = []
    for prot in (None, (1e-9, 1e-9)):
        g = oracle_mod.Grid((8, 8, 8), st["length"])
        if prot:
            g.set_protection(*prot)
        g.load_state(st)
        g.advance(2)
        out.append((g.read(), g.counters()))
    for a, b in zip(out[0][0], out[1][0]):
        assert np.array_equal(a, b)
    assert out[0][1] == out[1][1] == (0, 0, 0)
