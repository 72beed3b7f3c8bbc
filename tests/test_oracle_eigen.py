"""Pins of the oracle's interface eigen-system (App. A: R_k, alpha_k from the
Cargo & Gallice type Roe average; Sec. 3: eigenvalues a_1..a_7 and c_f, c_s,
c_a) against facts that do not come from the oracle itself:
  * L R = I (left and right eigenvectors are dual bases);
  * the Roe property  sum_k a_k alpha_k R_k = F(q_R) - F(q_L)  for equal
    normal field, with F written out from the paper's flux vector (Sec. 3);
  * at equal states, R_k is an eigenvector of the flux Jacobian obtained by
    complex-step differentiation of that flux vector, with eigenvalue a_k;
  * the paper's linear-wave background (Sec. "Linear Wave Convergence")
    gives c_f = 2, c_a = 1, c_s = 1/2 exactly.
"""
import json
import math
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def cons(rho, v, p, B, gam):
    E = p / (gam - 1) + 0.5 * rho * np.dot(v, v) + 0.5 * np.dot(B, B)
    return np.array([rho, rho * v[0], rho * v[1], rho * v[2], E, B[0], B[1], B[2]])


def flux_paper(q, gam):
    """Sec. 3 flux vector F (7 non-trivial comps, system order)."""
    rho, mn, mt1, mt2, E, bn, bt1, bt2 = q
    vn, vt1, vt2 = mn / rho, mt1 / rho, mt2 / rho
    P = (gam - 1) * (E - 0.5 * rho * (vn * vn + vt1 * vt1 + vt2 * vt2)
                     - 0.5 * (bn * bn + bt1 * bt1 + bt2 * bt2))
    Ps = P + 0.5 * (bn * bn + bt1 * bt1 + bt2 * bt2)
    return np.array([rho * vn, rho * vn * vn + Ps - bn * bn, rho * vn * vt1 - bn * bt1,
                     rho * vn * vt2 - bn * bt2, bt1 * vn - bn * vt1, bt2 * vn - bn * vt2,
                     (E + Ps) * vn - bn * (bn * vn + bt1 * vt1 + bt2 * vt2)])


def to_sys(q):
    return np.array([q[0], q[1], q[2], q[3], q[6], q[7], q[4]])


def from_sys(u, bn):
    return np.array([u[0], u[1], u[2], u[3], u[6], bn, u[4], u[5]])


def jacobian(q, gam):
    """Complex-step Jacobian dF/dU of the 7-variable system (B_n fixed)."""
    u0 = to_sys(q).astype(complex)
    J = np.zeros((7, 7))
    h = 1e-30
    for m in range(7):
        u = u0.copy()
        u[m] += 1j * h
        J[:, m] = flux_paper(from_sys(u, q[5]), gam).imag / h
    return J


def random_pair(rng, gam, b, degenerate=None):
    qs = []
    for _ in range(2):
        rho = math.exp(rng.normal())
        v = rng.normal(size=3)
        p = math.exp(rng.normal())
        bt = rng.normal(size=2)
        if degenerate == "bt0":
            bt = bt * 1e-9
        qs.append(cons(rho, v, p, np.array([b, bt[0], bt[1]]), gam))
    return qs


@pytest.mark.parametrize("gam", [5.0 / 3.0, 1.4, 2.0])
def test_left_right_duality_and_roe_property(oracle_mod, gam):
    rng = np.random.default_rng(11)
    for t in range(300):
        b = 0.0 if t % 6 == 0 else rng.normal()
        qL, qR = random_pair(rng, gam, b, "bt0" if t % 5 == 0 else None)
        lam, alpha, R, L = oracle_mod.face_eigen(qL, qR, b, gam)
        assert np.abs(L @ R - np.eye(7)).max() < 1e-12
        dF = flux_paper(qR, gam) - flux_paper(qL, gam)
        roe = R @ (lam * alpha)
        assert np.abs(roe - dF).max() <= 1e-12 * max(1.0, np.abs(dF).max())


def test_eigenvectors_of_flux_jacobian(oracle_mod):
    rng = np.random.default_rng(12)
    for t in range(100):
        gam = [5.0 / 3.0, 1.4][t % 2]
        b = rng.normal()
        q, _ = random_pair(rng, gam, b)
        lam, alpha, R, L = oracle_mod.face_eigen(q, q, b, gam)
        assert np.all(alpha == 0.0)
        J = jacobian(q, gam)
        scale = np.abs(J).max()
        for k in range(7):
            res = J @ R[:, k] - lam[k] * R[:, k]
            assert np.abs(res).max() <= 1e-12 * scale * max(1.0, np.abs(R[:, k]).max())
        # eigenvalues are those of the Jacobian (numpy's general solver)
        ev = np.sort(np.linalg.eigvals(J).real)
        assert np.allclose(np.sort(lam), ev, rtol=1e-9, atol=1e-9 * scale)


def test_linear_wave_background_speeds(oracle_mod):
    with open(os.path.join(GOLD, "linear_wave_background.json")) as f:
        g = json.load(f)
    gam, rho, p = g["gamma"], g["rho"], g["P"]
    B = np.array(g["B"])
    v = np.array([g["vx"], 0.0, 0.0])
    q = cons(rho, v, p, B, gam)
    lam, _, _, _ = oracle_mod.face_eigen(q, q, B[0], gam)
    expect = np.array(g["eigenvalues_vx_plus"])
    assert np.allclose(lam, expect, rtol=0, atol=2e-15)


def test_degenerate_states_stay_complete(oracle_mod):
    """B = 0 (hydro), B_t = 0 with a = c_a (triple degeneracy) and B_n = 0."""
    gam = 5.0 / 3.0
    cases = [
        (cons(1.0, np.zeros(3), 0.6, np.zeros(3), gam), 0.0),
        (cons(1.0, np.array([0.3, 0, 0]), 0.6, np.array([1.0, 0, 0]), gam), 1.0),  # a = ca = 1
        (cons(2.0, np.array([0.3, 0.1, 0]), 1.0, np.array([0.0, 0.4, -0.2]), gam), 0.0),
    ]
    for q, b in cases:
        lam, alpha, R, L = oracle_mod.face_eigen(q, q, b, gam)
        assert np.abs(L @ R - np.eye(7)).max() < 1e-12
        J = jacobian(q, gam)
        for k in range(7):
            res = J @ R[:, k] - lam[k] * R[:, k]
            assert np.abs(res).max() < 1e-11
