"""Linear-wave initial data of the paper's convergence tests (Sec. 'Linear Wave
Convergence'): background rho = 1, P = 3/5, gamma = 5/3, B = (1, sqrt 2, 1/2),
v_1 = 1 (or a background at rest, v = 0, as in the oblique setup the paper
takes from GS08), amplitude A0 = 1e-6 times a right eigenvector of the flux
Jacobian.
The eigenvector comes from numpy's eigen-solver applied to the complex-step
Jacobian of the paper's flux vector (Sec. 3), not from the oracle."""
import math

import numpy as np

GAMMA = 5.0 / 3.0
RHO, PRES, A0 = 1.0, 0.6, 1e-6
B_WAVE = np.array([1.0, math.sqrt(2.0), 0.5])
V_WAVE = np.array([1.0, 0.0, 0.0])
MODES = {"fast": 6, "alfven": 5, "slow": 4, "entropy": 3}  # index in ascending eigenvalues


def _flux(u, bn, gam):
    rho, mn, mt1, mt2, bt1, bt2, E = u
    vn, vt1, vt2 = mn / rho, mt1 / rho, mt2 / rho
    P = (gam - 1) * (E - 0.5 * rho * (vn * vn + vt1 * vt1 + vt2 * vt2)
                     - 0.5 * (bn * bn + bt1 * bt1 + bt2 * bt2))
    Ps = P + 0.5 * (bn * bn + bt1 * bt1 + bt2 * bt2)
    return np.array([mn, mn * vn + Ps - bn * bn, mn * vt1 - bn * bt1, mn * vt2 - bn * bt2,
                     bt1 * vn - bn * vt1, bt2 * vn - bn * vt2,
                     (E + Ps) * vn - bn * (bn * vn + bt1 * vt1 + bt2 * vt2)])


def background_u(v=None):
    v = V_WAVE if v is None else np.asarray(v, float)
    B = B_WAVE
    E = PRES / (GAMMA - 1) + 0.5 * RHO * v @ v + 0.5 * B @ B
    return np.array([RHO, RHO * v[0], RHO * v[1], RHO * v[2], B[1], B[2], E])


def eigenmode(mode, v=None):
    """(lambda, r) for the wave-frame 7-variable system (rho, M1, M2, M3, B2, B3, E)."""
    u0 = background_u(v).astype(complex)
    J = np.zeros((7, 7))
    for m in range(7):
        u = u0.copy()
        u[m] += 1e-30j
        J[:, m] = _flux(u, B_WAVE[0], GAMMA).imag / 1e-30
    w, V = np.linalg.eig(J)
    order = np.argsort(w.real)
    k = order[MODES[mode]]
    r = V[:, k].real
    r = r / np.abs(r).max()
    return float(w[k].real), r


def state_1d(mode, n):
    """x-only wave in an n x 1 x 1 box of length 1 (conserved U and faces)."""
    lam, r = eigenmode(mode)
    u0 = background_u()
    x = (np.arange(n) + 0.5) / n
    c = np.cos(2 * math.pi * x)
    q = u0[:, None] + A0 * r[:, None] * c[None, :]
    U = np.zeros((5, 1, 1, n))
    U[0, 0, 0], U[1, 0, 0], U[2, 0, 0], U[3, 0, 0], U[4, 0, 0] = q[0], q[1], q[2], q[3], q[6]
    bx = np.full((1, 1, n + 1), B_WAVE[0])
    by = np.zeros((1, 2, n)); by[0, 0] = q[4]; by[0, 1] = q[4]
    bz = np.zeros((2, 1, n)); bz[0, 0] = q[5]; bz[1, 0] = q[5]
    return lam, U, bx, by, bz


def frame(kvec):
    e1 = np.asarray(kvec, float) / np.linalg.norm(kvec)
    e2 = np.array([-e1[1], e1[0], 0.0]); e2 /= np.linalg.norm(e2)
    e3 = np.cross(e1, e2)
    return e1, e2, e3


def state_oblique(mode, n, kvec=(1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0), length=(3.0, 1.5, 1.5),
                  v=None):
    """Oblique wave on a 2n x n x n grid of size (3, 3/2, 3/2), wave vector k
    (wavelength 1); face b = uniform mean + curl of an edge potential.  v: the
    wave-frame background velocity (default (1, 0, 0); (0, 0, 0) at rest)."""
    lam, r = eigenmode(mode, v)
    e1, e2, e3 = frame(kvec)
    nx, ny, nz = 2 * n, n, n
    dx, dy, dz = length[0] / nx, length[1] / ny, length[2] / nz
    R = np.stack([e1, e2, e3], axis=1)   # wave frame -> grid
    u0 = background_u(v)
    rho_b, m_b, e_b = u0[0], R @ u0[1:4], u0[6]
    Bbar = R @ B_WAVE
    dm = R @ r[1:4]
    dBw = np.array([0.0, r[4], r[5]])
    def phase(x, y, z):
        return 2 * math.pi * (e1[0] * x + e1[1] * y + e1[2] * z)
    zc = (np.arange(nz) + 0.5) * dz
    yc = (np.arange(ny) + 0.5) * dy
    xc = (np.arange(nx) + 0.5) * dx
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    c = np.cos(phase(X, Y, Z))
    U = np.zeros((5, nz, ny, nx))
    U[0] = rho_b + A0 * r[0] * c
    for d in range(3):
        U[1 + d] = m_b[d] + A0 * dm[d] * c
    U[4] = e_b + A0 * r[6] * c
    # vector potential (wave frame) A = A0 (0, r_B3, -r_B2) sin(2 pi x1) / (2 pi)
    aw = A0 * np.array([0.0, dBw[2], -dBw[1]]) / (2 * math.pi)
    ag = R @ aw
    xf = np.arange(nx) * dx; yf = np.arange(ny) * dy; zf = np.arange(nz) * dz
    def edge(comp, xs, ys, zs):
        Zz, Yy, Xx = np.meshgrid(zs, ys, xs, indexing="ij")
        return ag[comp] * np.sin(phase(Xx, Yy, Zz))
    Ax = edge(0, xc, yf, zf)
    Ay = edge(1, xf, yc, zf)
    Az = edge(2, xf, yf, zc)
    from paper_1701_07452_gb300.initial_conditions import curl_faces
    bx, by, bz = curl_faces(Ax, Ay, Az, dx, dy, dz)
    bx = bx + Bbar[0]; by = by + Bbar[1]; bz = bz + Bbar[2]
    return lam, U, bx, by, bz


def l1_error(U, U0, B, B0):
    """Norm of the L1 error vector over the 8 zone variables."""
    errs = [np.abs(U[c] - U0[c]).mean() for c in range(5)]
    errs += [np.abs(B[c] - B0[c]).mean() for c in range(3)]
    return math.sqrt(sum(e * e for e in errs))
