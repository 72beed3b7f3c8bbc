"""Validation problems of Sec. "Test Calculations" on the oracle.

Pins of the oracle that do not come from its own code:
  * circularly polarised Alfven wave: an exact nonlinear solution that returns
    to its initial state after one period; the L1 error vector converges;
  * field-loop advection: constrained transport keeps div b at round-off for
    a discontinuous field, and the loop's magnetic energy only decays;
  * RJ95 2a, RJ95 4a, Brio & Wu: solutions converge to a 2048-zone solution
    of the independent 1D driver (as the paper compares Brio & Wu with a
    finer run), and the 3D CTU+CT path with x-only data equals the 1D driver;
  * magnetised blast wave: mass, momentum and face field are conserved,
    div b stays at round-off and the state stays physical.
"""
import numpy as np
import pytest

from paper_1701_07452_gb300 import initial_conditions as ic


def l1_vector_norm(a, b):
    """Norm of the L1 error vector (Sec. "Linear Wave Convergence") over the
    conserved variables and the zone field."""
    Ua, Ba = a[0], a[4]
    Ub, Bb = b[0], b[4]
    dq = [np.abs(Ua[c] - Ub[c]).mean() for c in range(5)] + \
         [np.abs(Ba[c] - Bb[c]).mean() for c in range(3)]
    return float(np.sqrt(np.sum(np.square(dq))))


def cpaw_error(oracle_mod, n):
    st = ic.cpaw_box(n)
    g = oracle_mod.Grid((2 * n, n, n), st["length"])
    g.load_state(st)
    s0 = g.read()
    t = g.advance(100000, t_end=1.0)
    assert abs(t - 1.0) < 1e-13
    assert g.counters() == (0, 0, 0)
    return l1_vector_norm(g.read(), s0)


def test_cpaw_returns_after_one_period(oracle_mod):
    errs = [cpaw_error(oracle_mod, n) for n in (8, 16, 32)]
    assert errs[2] < 0.008, errs
    assert errs[0] / errs[1] > 2.5 and errs[1] / errs[2] > 3.0, errs


def test_field_loop_keeps_div_b_and_decays(oracle_mod):
    n = 32
    st = ic.field_loop_box(n)
    g = oracle_mod.Grid((2 * n, n, 1), st["length"])
    g.load_state(st)
    B0 = g.read()[4]
    em = [0.5 * float((B0 ** 2).sum())]
    for _ in range(8):  # two periods (t = 2), as in the paper
        g.advance(100000, t_end=0.25)
        em.append(0.5 * float((g.read()[4] ** 2).sum()))
    U, bx, by, bz, B = g.read()
    assert g.divb_max() < 1e-14
    assert all(em[i + 1] <= em[i] for i in range(len(em) - 1)), em
    assert 0.15 < em[-1] / em[0] < 0.35, em
    # B_z and v_z stay small against the loop field (the RJ95 degenerate
    # eigenvector convention couples the two transverse directions where B = 0)
    assert np.abs(bz).max() < 1e-3 * np.abs(B).max()
    assert g.counters() == (0, 0, 0)


def shock_line(name, n):
    st = ic.SHOCK_TUBES[name]
    W = ic.shock_tube_1d(name, n)["W"][:, 0, 0]
    g = st["gamma"]
    rho, vx, vy, vz, p = W
    by = np.where((np.arange(n) + 0.5) / n < 0.5, st["left"][4], st["right"][4])
    bz = np.where((np.arange(n) + 0.5) / n < 0.5, st["left"][5], st["right"][5])
    bx = st["bx"]
    q = np.empty((n, 8))
    q[:, 0] = rho
    q[:, 1], q[:, 2], q[:, 3] = rho * vx, rho * vy, rho * vz
    q[:, 4] = p / (g - 1.0) + 0.5 * rho * (vx ** 2 + vy ** 2 + vz ** 2) + 0.5 * (bx ** 2 + by ** 2 + bz ** 2)
    q[:, 5], q[:, 6], q[:, 7] = bx, by, bz
    return q


def cfl_dt_1d(q, gamma, dx, cfl=0.8):
    rho = q[:, 0]
    b2 = q[:, 5] ** 2 + q[:, 6] ** 2 + q[:, 7] ** 2
    p = (gamma - 1.0) * (q[:, 4] - 0.5 * (q[:, 1] ** 2 + q[:, 2] ** 2 + q[:, 3] ** 2) / rho - 0.5 * b2)
    a2 = gamma * p / rho
    s = a2 + b2 / rho
    cf = np.sqrt(0.5 * (s + np.sqrt(np.maximum(s * s - 4.0 * a2 * q[:, 5] ** 2 / rho, 0.0))))
    return cfl * dx / np.max(np.abs(q[:, 1] / rho) + cf)


def run_line(oracle_mod, name, n, dts=None):
    st = ic.SHOCK_TUBES[name]
    q = shock_line(name, n)
    t, dx, used = 0.0, 1.0 / n, []
    while t < st["t"] * (1.0 - 1e-14):
        dt = dts[len(used)] if dts is not None else min(cfl_dt_1d(q, st["gamma"], dx), st["t"] - t)
        q = oracle_mod.step_1d(q, st["bx"], dt, dx, st["gamma"], outflow=True)
        used.append(dt)
        t += dt
    return q, used


@pytest.mark.parametrize("name", ["briowu", "rj2a", "rj4a"])
def test_shock_tube_self_convergence(oracle_mod, name):
    ref, _ = run_line(oracle_mod, name, 2048)
    errs = []
    for n in (128, 256, 512):
        q, _ = run_line(oracle_mod, name, n)
        assert q[:, 0].min() > 0.0
        r = ref[:, 0].reshape(n, -1).mean(axis=1)
        errs.append(float(np.abs(q[:, 0] - r).mean()))
    assert errs[0] < 0.012 and errs[2] < 0.004, errs
    assert errs[0] / errs[1] > 1.5 and errs[1] / errs[2] > 1.5, errs


def test_shock_tube_3d_path_equals_1d_driver(oracle_mod):
    name, n = "briowu", 64
    st = ic.SHOCK_TUBES[name]
    q1, dts = run_line(oracle_mod, name, n)
    s = ic.shock_tube_1d(name, n)
    g = oracle_mod.Grid((n, 1, 1), s["length"], gamma=st["gamma"], bc=(1, 0, 0))
    g.load_state(s)
    for dt in dts:
        assert g.step(dt) == 0
    U, bx, by, bz, B = g.read()
    q3 = np.stack([U[0, 0, 0], U[1, 0, 0], U[2, 0, 0], U[3, 0, 0], U[4, 0, 0],
                   B[0, 0, 0], B[1, 0, 0], B[2, 0, 0]], axis=1)
    scale = np.abs(q1).max(axis=0) + 1e-300
    assert (np.abs(q3 - q1) / scale).max() < 1e-12


def test_blast_wave_conserves_and_stays_physical(oracle_mod):
    st = ic.blast_box(16, 24, 16)
    g = oracle_mod.Grid((16, 24, 16), st["length"])
    g.set_protection(1e-3, 1e-3)
    g.load_state(st)
    tot0 = g.totals()
    t = g.advance(100000, t_end=0.02)
    assert abs(t - 0.02) < 1e-15
    tot = g.totals()
    for c in (0, 1, 2, 3, 5, 6, 7):
        assert abs(tot[c] - tot0[c]) <= 1e-12 * max(abs(tot0[c]), tot0[0]), (c, tot[c], tot0[c])
    U, bx, by, bz, B = g.read()
    p = (2.0 / 3.0) * (U[4] - 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / U[0] - 0.5 * (B ** 2).sum(0))
    assert U[0].min() > 0.0 and p.min() > 0.0
    assert g.divb_max() < 1e-12
    floors, unphysical, hll = g.counters()
    assert unphysical == 0 and hll > 0
