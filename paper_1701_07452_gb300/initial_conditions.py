"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no arithmetic of the MHD step itself: it returns primitive
zone data (rho, vx, vy, vz, P) and face-centred magnetic fields built as the
discrete curl of an edge-centred vector potential (so div b = 0 to rounding).
Each consumer converts primitives to conserved variables on its own side.

Workloads (the paper's performance runs do not state their initial data, so
these stand in for them):
  * ``random_box``      -- rho = 1 + 0.1 U(-1,1), P = 0.6, v_d ~ U(-0.1, 0.1),
    b = (1/sqrt(4 pi)) x^ + curl A, A_d ~ 0.05 U(-1,1) per edge, dx = 1.
  * ``turbulence_box``  -- rho = 1, P = 1, random-phase solenoidal velocity
    modes 1 <= |k| <= 8 with amplitude ~ |k|^-2 (shell spectrum ~ k^-2) at
    rms Mach 1, mean field along x at plasma beta 100, plus curl of a random
    vector potential (1 <= |k| <= 4) at 10 % of the mean field, L = 1.  The
    mode table depends on the seed only, never on N.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["random_box", "turbulence_box", "turbulence_box_device", "expansion_box", "mode_table",
           "curl_faces", "cpaw_box", "field_loop_box", "shock_tube_1d", "blast_box", "SHOCK_TUBES",
           "orszag_tang_box", "random_box_2d", "shock_tube_rotated", "curl_faces_open", "State"]


class State(dict):
    """W[5][nz][ny][nx] = (rho, vx, vy, vz, P); bx[nz][ny][nx+1], by, bz."""


def curl_faces(Ax, Ay, Az, dx, dy, dz):
    """Face fields b = curl A from periodic edge-centred potentials.

    Ax[k, j, i] sits on the x-edge at ((i+1/2)dx, j dy, k dz), Ay on
    (i dx, (j+1/2)dy, k dz), Az on (i dx, j dy, (k+1/2) dz); all periodic.
    Returns bx[nz][ny][nx+1], by[nz][ny+1][nx], bz[nz+1][ny][nx] where face
    index f is the low face of zone f and the last face repeats face 0.
    """
    # b_x at (i dx, (j+1/2) dy, (k+1/2) dz)
    bx = (np.roll(Az, -1, axis=1) - Az) / dy - (np.roll(Ay, -1, axis=0) - Ay) / dz
    by = (np.roll(Ax, -1, axis=0) - Ax) / dz - (np.roll(Az, -1, axis=2) - Az) / dx
    bz = (np.roll(Ay, -1, axis=2) - Ay) / dx - (np.roll(Ax, -1, axis=1) - Ax) / dy
    bx = np.concatenate([bx, bx[:, :, :1]], axis=2)
    by = np.concatenate([by, by[:, :1, :]], axis=1)
    bz = np.concatenate([bz, bz[:1, :, :]], axis=0)
    return bx, by, bz


def random_box(n, seed, b0=1.0 / math.sqrt(4.0 * math.pi), a_amp=0.05):
    """Config-1-style box: n^3 zones, dx = 1 (L = n), every value from one seed."""
    if np.isscalar(n):
        n = (int(n),) * 3
    nx, ny, nz = n
    rng = np.random.default_rng(seed)
    shape = (nz, ny, nx)
    W = np.empty((5,) + shape)
    W[0] = 1.0 + 0.1 * rng.uniform(-1.0, 1.0, shape)
    W[1] = rng.uniform(-0.1, 0.1, shape)
    W[2] = rng.uniform(-0.1, 0.1, shape)
    W[3] = rng.uniform(-0.1, 0.1, shape)
    W[4] = 0.6
    Ax = a_amp * rng.uniform(-1.0, 1.0, shape)
    Ay = a_amp * rng.uniform(-1.0, 1.0, shape)
    Az = a_amp * rng.uniform(-1.0, 1.0, shape)
    bx, by, bz = curl_faces(Ax, Ay, Az, 1.0, 1.0, 1.0)
    bx = bx + b0
    return State(W=W, bx=bx, by=by, bz=bz, length=(float(nx), float(ny), float(nz)))


def expansion_box(n, seed, speed=2.0, gamma=5.0 / 3.0):
    """Strong 3D expansion on a periodic unit box: v_x = -speed on the low
    half and +speed on the high half (a double rarefaction at the middle, a
    collision at the wrap, Mach ~2.4 each way), transverse shear
    0.3 sin(2 pi x), 5 % random noise, P = 0.4, field (0.3, 0.2, 0.1) plus
    the curl of a random edge potential.  A Roe-type flux meets unphysical
    intermediate states here; the input for the protection-floor path."""
    n = int(n)
    rng = np.random.default_rng(seed)
    shape = (n, n, n)
    x = (np.arange(n) + 0.5) / n
    W = np.empty((5,) + shape)
    W[0] = 1.0 + 0.05 * rng.uniform(-1.0, 1.0, shape)
    W[1] = np.where(x[None, None, :] < 0.5, -speed, speed) + 0.05 * rng.uniform(-1.0, 1.0, shape)
    W[2] = 0.3 * np.sin(2.0 * np.pi * x)[:, None, None] + 0.05 * rng.uniform(-1.0, 1.0, shape)
    W[3] = 0.3 * np.sin(2.0 * np.pi * x)[None, :, None] + 0.05 * rng.uniform(-1.0, 1.0, shape)
    W[4] = 0.4
    A = [0.02 / n * rng.uniform(-1.0, 1.0, shape) for _ in range(3)]
    bx, by, bz = curl_faces(*A, 1.0 / n, 1.0 / n, 1.0 / n)
    return State(W=W, bx=bx + 0.3, by=by + 0.2, bz=bz + 0.1, length=(1.0, 1.0, 1.0))


# Rotated frame of the oblique tests (Sec. "Linear Wave Convergence", 3D): the
# wave normal n = (1, 2, 2)/3 makes every box of shape (3, 3/2, 3/2) with
# 2N x N x N zones periodic for one wavelength 1 along n.
OBLIQUE_N = np.array([1.0, 2.0, 2.0]) / 3.0
OBLIQUE_E2 = np.array([-2.0, 1.0, 0.0]) / math.sqrt(5.0)
OBLIQUE_E3 = np.cross(OBLIQUE_N, OBLIQUE_E2)


def _oblique_coords(n):
    """Zone-centre and edge-centre coordinates x1 = n . x of a 2N x N x N box
    of size (3, 3/2, 3/2); edges as in curl_faces."""
    nx, ny, nz = 2 * n, n, n
    d = 1.5 / n
    i = np.arange(nx)[None, None, :]
    j = np.arange(ny)[None, :, None]
    k = np.arange(nz)[:, None, None]
    nv = OBLIQUE_N

    def x1(xo, yo, zo):
        return nv[0] * (i + xo) * d + nv[1] * (j + yo) * d + nv[2] * (k + zo) * d

    return (nx, ny, nz), d, x1(0.5, 0.5, 0.5), x1(0.5, 0.0, 0.0), x1(0.0, 0.5, 0.0), x1(0.0, 0.0, 0.5)


def _oblique_state(n, rho, p, v_of, b_par, a2_of, a3_of):
    """State of a 2N x N x N oblique box whose fields depend on x1 = n . x
    only: v(x1) in grid axes, B = b_par n + curl(A2(x1) e2 + A3(x1) e3)."""
    shape, d, xc, xex, xey, xez = _oblique_coords(n)
    W = np.empty((5,) + shape[::-1])
    W[0] = rho(xc)
    v = v_of(xc)
    W[1], W[2], W[3] = v[0], v[1], v[2]
    W[4] = p(xc)
    e2, e3 = OBLIQUE_E2, OBLIQUE_E3
    A = []
    for ax, xe in enumerate((xex, xey, xez)):
        A.append(a2_of(xe) * e2[ax] + a3_of(xe) * e3[ax])
    bx, by, bz = curl_faces(A[0], A[1], A[2], d, d, d)
    bx = bx + b_par * OBLIQUE_N[0]
    by = by + b_par * OBLIQUE_N[1]
    bz = bz + b_par * OBLIQUE_N[2]
    return State(W=W, bx=bx, by=by, bz=bz, length=(3.0, 1.5, 1.5))


def cpaw_box(n, amp=0.1, p=0.1):
    """Circularly polarised Alfven wave (Sec. "Circularly Polarized Alfven
    Wave"), an exact nonlinear solution: rho = 1, P = 0.1, v_par = 0,
    B_par = 1, v_2 = B_2 = amp sin(2 pi x1), v_3 = B_3 = amp cos(2 pi x1), on
    the oblique 2N x N x N box of size (3, 3/2, 3/2).  With v_perp = B_perp the
    wave moves along -n at the Alfven speed 1 and returns after t = 1."""
    tp = 2.0 * math.pi
    e2, e3 = OBLIQUE_E2, OBLIQUE_E3

    def v_of(x1):
        s, c = amp * np.sin(tp * x1), amp * np.cos(tp * x1)
        return [s * e2[a] + c * e3[a] for a in range(3)]

    return _oblique_state(n, lambda x: np.ones_like(x), lambda x: np.full_like(x, p), v_of, 1.0,
                          lambda x: amp * np.sin(tp * x) / tp, lambda x: amp * np.cos(tp * x) / tp)


def field_loop_box(n, amp=1e-3, r0=0.3, v=(2.0, 0.5)):
    """Advection of a weak field loop (Sec. "Advection of a Field Loop"), 2D:
    a 2N x N x 1 periodic box [-1, 1] x [-1/2, 1/2] (thin in z), rho = 1,
    P = 1, v = (2, 0.5, 0), A_z = max(amp (r0 - r), 0) at zone corners."""
    nx, ny = 2 * n, n
    dx = 2.0 / nx
    x = -1.0 + np.arange(nx) * dx
    y = -0.5 + np.arange(ny) * dx
    r = np.sqrt(x[None, :] ** 2 + y[:, None] ** 2)
    Az = np.maximum(amp * (r0 - r), 0.0)[None, :, :]
    zero = np.zeros((1, ny, nx))
    dz = 1e3
    bx, by, bz = curl_faces(zero, zero, Az, dx, dx, dz)
    W = np.empty((5, 1, ny, nx))
    W[0] = 1.0
    W[1] = v[0]
    W[2] = v[1]
    W[3] = 0.0
    W[4] = 1.0
    return State(W=W, bx=bx, by=by, bz=bz, length=(2.0, 1.0, dz))


def orszag_tang_box(n, v0=1.0):
    """Orszag-Tang vortex (Sec. "Orszag-Tang Vortex"), 2D: periodic unit box
    [-1/2, 1/2]^2 with n x n x 1 zones (thin in z), rho = 25/(36 pi),
    P = 5/(12 pi), v = v0 (-sin 2 pi y, sin 2 pi x, 0), field from the corner
    potential A_z = B0 [cos(4 pi x)/2 + cos(2 pi y)] / (2 pi), B0 = 1/sqrt(4 pi)."""
    d = 1.0 / n
    xc = -0.5 + (np.arange(n) + 0.5) * d
    x = -0.5 + np.arange(n) * d
    b0 = 1.0 / math.sqrt(4.0 * math.pi)
    Az = b0 * (np.cos(4.0 * math.pi * x)[None, :] / 2.0 + np.cos(2.0 * math.pi * x)[:, None]) / (2.0 * math.pi)
    zero = np.zeros((1, n, n))
    dz = 1e3
    bx, by, bz = curl_faces(zero, zero, Az[None, :, :], d, d, dz)
    W = np.empty((5, 1, n, n))
    W[0] = 25.0 / (36.0 * math.pi)
    W[1] = -v0 * np.sin(2.0 * math.pi * xc)[None, :, None]
    W[2] = v0 * np.sin(2.0 * math.pi * xc)[None, None, :]
    W[3] = 0.0
    W[4] = 5.0 / (12.0 * math.pi)
    return State(W=W, bx=bx, by=by, bz=bz, length=(1.0, 1.0, dz))


def random_box_2d(nx, ny, seed):
    """2.5D random box, one zone thick in z: every field, v_z and B_z
    included, varies in x and y only (dx = 1)."""
    rng = np.random.default_rng(seed)
    shape = (1, ny, nx)
    W = np.empty((5,) + shape)
    W[0] = 1.0 + 0.1 * rng.uniform(-1.0, 1.0, shape)
    for c in (1, 2, 3):
        W[c] = rng.uniform(-0.2, 0.2, shape)
    W[4] = 0.6 + 0.05 * rng.uniform(-1.0, 1.0, shape)
    A = [0.05 * rng.uniform(-1.0, 1.0, shape) for _ in range(3)]
    bx, by, bz = curl_faces(A[0], A[1], A[2], 1.0, 1.0, 1.0)
    return State(W=W, bx=bx + 0.3, by=by + 0.2, bz=bz + 0.25, length=(float(nx), float(ny), 1.0))


# Shock-tube states (rho, vx, vy, vz, By, Bz, P) and the normal field Bx
# (Secs. "RJ95 2a", "RJ95 4a", "Brio & Wu Shock-tube").
_S4PI = math.sqrt(4.0 * math.pi)
SHOCK_TUBES = {
    # the printed 2a left state lists six numbers for seven variables; the
    # missing one is v_z = 0.5 of the RJ95 problem it reproduces
    "rj2a": dict(left=(1.08, 1.2, 0.01, 0.5, 3.6 / _S4PI, 2.0 / _S4PI, 0.95),
                 right=(1.0, 0.0, 0.0, 0.0, 4.0 / _S4PI, 2.0 / _S4PI, 1.0),
                 bx=2.0 / _S4PI, gamma=5.0 / 3.0, t=0.2),
    "rj4a": dict(left=(1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 1.0),
                 right=(0.2, 0.0, 0.0, 0.0, 0.0, 0.0, 0.1),
                 bx=1.0, gamma=5.0 / 3.0, t=0.15),
    "briowu": dict(left=(1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 1.0),
                   right=(0.125, 0.0, 0.0, 0.0, -1.0, 0.0, 0.1),
                   bx=0.75, gamma=2.0, t=0.08),
}


def shock_tube_1d(name, n):
    """n x 1 x 1 box on [0, 1] (outflow along x, thin in y and z) with the
    named shock-tube states on either side of x = 1/2."""
    st = SHOCK_TUBES[name]
    x = (np.arange(n) + 0.5) / n
    left = x < 0.5
    W = np.empty((5, 1, 1, n))
    for c, idx in enumerate((0, 1, 2, 3, 6)):
        W[c, 0, 0] = np.where(left, st["left"][idx], st["right"][idx])
    by_z = np.where(left, st["left"][4], st["right"][4])
    bz_z = np.where(left, st["left"][5], st["right"][5])
    bx = np.full((1, 1, n + 1), st["bx"])
    by = np.repeat(by_z[None, None, :], 2, axis=1)
    bz = np.repeat(bz_z[None, None, :], 2, axis=0)
    return State(W=W, bx=bx, by=by, bz=bz, length=(1.0, 1e3, 1e3))


ROTATED_N = np.array([1.0, 1.0, 1.0]) / math.sqrt(3.0)
ROTATED_E2 = np.array([-1.0, 1.0, 0.0]) / math.sqrt(2.0)
ROTATED_E3 = np.cross(ROTATED_N, ROTATED_E2)


def curl_faces_open(Ax, Ay, Az, dx, dy, dz):
    """Face fields b = curl A of a non-periodic box from edge potentials that
    include the high edges: Ax[nz+1][ny+1][nx] on ((i+1/2)dx, j dy, k dz),
    Ay[nz+1][ny][nx+1] on (i dx, (j+1/2)dy, k dz), Az[nz][ny+1][nx+1] on
    (i dx, j dy, (k+1/2)dz).  Returns bx[nz][ny][nx+1], by[nz][ny+1][nx],
    bz[nz+1][ny][nx] with every face of the box, so that each zone's
    discrete div b is zero to rounding."""
    bx = (Az[:, 1:, :] - Az[:, :-1, :]) / dy - (Ay[1:, :, :] - Ay[:-1, :, :]) / dz
    by = (Ax[1:, :, :] - Ax[:-1, :, :]) / dz - (Az[:, :, 1:] - Az[:, :, :-1]) / dx
    bz = (Ay[:, :, 1:] - Ay[:, :, :-1]) / dx - (Ax[:, 1:, :] - Ax[:, :-1, :]) / dy
    return bx, by, bz


def shock_tube_rotated(name, n, boost=(0.0, 0.0)):
    """The named shock tube in an n^3 cube of side 1 (outflow on every axis)
    with its normal along n = (1, 1, 1)/sqrt 3, equally inclined to the three
    primary planes (Sec. "RJ95 2a" tilts the normal out of all of them), the
    discontinuity on the plane through the box centre.  The
    1D states (rho, v_n, v_t2, v_t3, B_t2, B_t3, P), B_n, are laid out in the
    frame (n, e2, e3); the field is B_n n + curl(G3(s) e2 - G2(s) e3) with
    s = n . (x - centre) and G2, G3 the continuous piecewise-linear integrals
    of B_t2, B_t3, evaluated on the edges (div b = 0 to rounding).  boost =
    (V2, V3) adds the uniform velocity V2 e2 + V3 e3 to both states (MHD is
    Galilean invariant: the solution is the same, its transverse velocity
    shifted by the boost)."""
    st = SHOCK_TUBES[name]
    d = 1.0 / n
    e1, e2, e3 = ROTATED_N, ROTATED_E2, ROTATED_E3
    L, R = st["left"], st["right"]

    def coords(xo, yo, zo, sx, sy, sz):
        i = (np.arange(sx) + xo)[None, None, :] * d - 0.5
        j = (np.arange(sy) + yo)[None, :, None] * d - 0.5
        k = (np.arange(sz) + zo)[:, None, None] * d - 0.5
        return i, j, k

    x, y, z = coords(0.5, 0.5, 0.5, n, n, n)
    sc = e1[0] * x + e1[1] * y + e1[2] * z
    left = sc < 0.0
    W = np.empty((5, n, n, n))
    W[0] = np.where(left, L[0], R[0])
    vn = np.where(left, L[1], R[1])
    v2 = np.where(left, L[2], R[2]) + boost[0]
    v3 = np.where(left, L[3], R[3]) + boost[1]
    for a in range(3):
        W[1 + a] = vn * e1[a] + v2 * e2[a] + v3 * e3[a]
    W[4] = np.where(left, L[6], R[6])

    def G(sv, bl, br):   # integral of a field that is bl for s < 0, br for s > 0
        return np.where(sv < 0.0, bl * sv, br * sv)

    bn = st["bx"]

    def potential(comp, xo, yo, zo, sx, sy, sz):
        xx, yy, zz = coords(xo, yo, zo, sx, sy, sz)
        sv = e1[0] * xx + e1[1] * yy + e1[2] * zz
        pos = (xx, yy, zz)
        # (bn/2) (n x r) + G3(s) e2 - G2(s) e3
        cross = 0.5 * bn * (e1[(comp + 1) % 3] * pos[(comp + 2) % 3] - e1[(comp + 2) % 3] * pos[(comp + 1) % 3])
        return cross + G(sv, L[5], R[5]) * e2[comp] - G(sv, L[4], R[4]) * e3[comp]

    Ax = potential(0, 0.5, 0.0, 0.0, n, n + 1, n + 1)
    Ay = potential(1, 0.0, 0.5, 0.0, n + 1, n, n + 1)
    Az = potential(2, 0.0, 0.0, 0.5, n + 1, n + 1, n)
    bx, by, bz = curl_faces_open(Ax, Ay, Az, d, d, d)
    return State(W=W, bx=bx, by=by, bz=bz, length=(1.0, 1.0, 1.0))


def blast_box(nx, ny, nz, b0=10.0, p_in=100.0, r0=0.125, shift=(0.0, 0.0, 0.0)):
    """Magnetised strong blast wave (Sec. "MHD Blast Wave"): periodic box of
    size (1, 3/2, 1) with nx x ny x nz zones, rho = 1 at rest,
    B = (b0/sqrt2, b0/sqrt2, 0), P = 1 except P = p_in within r0 of the
    centre.  shift moves the centre by that many zones per axis (an exactly
    centred blast has symmetry planes on faces, where the mass flux is zero
    in exact arithmetic)."""
    L = (1.0, 1.5, 1.0)
    d = [L[0] / nx, L[1] / ny, L[2] / nz]
    x = (np.arange(nx) + 0.5 - shift[0]) * d[0] - 0.5 * L[0]
    y = (np.arange(ny) + 0.5 - shift[1]) * d[1] - 0.5 * L[1]
    z = (np.arange(nz) + 0.5 - shift[2]) * d[2] - 0.5 * L[2]
    r = np.sqrt(x[None, None, :] ** 2 + y[None, :, None] ** 2 + z[:, None, None] ** 2)
    W = np.zeros((5, nz, ny, nx))
    W[0] = 1.0
    W[4] = np.where(r < r0, p_in, 1.0)
    bx = np.full((nz, ny, nx + 1), b0 / math.sqrt(2.0))
    by = np.full((nz, ny + 1, nx), b0 / math.sqrt(2.0))
    bz = np.zeros((nz + 1, ny, nx))
    return State(W=W, bx=bx, by=by, bz=bz, length=L)


def mode_table(seed, kmin, kmax, slope=-2.0):
    """Random-phase solenoidal modes: integer k in a half space with
    kmin <= |k| <= kmax, unit amplitude direction perpendicular to k, scale
    |k|^slope, uniform phase.  Returns (k[m,3], a[m,3], phase[m])."""
    rng = np.random.default_rng(seed)
    ks, amps, phs = [], [], []
    for kz in range(-kmax, kmax + 1):
        for ky in range(-kmax, kmax + 1):
            for kx in range(-kmax, kmax + 1):
                kk = math.sqrt(kx * kx + ky * ky + kz * kz)
                if kk < kmin or kk > kmax:
                    continue
                if not (kx > 0 or (kx == 0 and ky > 0) or (kx == 0 and ky == 0 and kz > 0)):
                    continue
                k = np.array([kx, ky, kz], dtype=np.float64)
                g = rng.normal(size=3)
                g -= k * (g @ k) / (k @ k)
                nrm = np.linalg.norm(g)
                if nrm == 0.0:
                    g = np.cross(k, [1.0, 0.3, 0.1]); nrm = np.linalg.norm(g)
                ks.append(k)
                amps.append(g / nrm * kk ** slope)
                phs.append(rng.uniform(0.0, 2.0 * math.pi))
    return np.array(ks), np.array(amps), np.array(phs)


def _eval_modes(k, a, ph, n, offsets, L=1.0):
    """f_c(x) = sum_m a[m,c] cos(2 pi k_m . x / L + ph_m) on a periodic grid,
    x_d = (i + offsets[d]) L / n_d, by separable small-band sums."""
    nx, ny, nz = n
    kmax = int(np.abs(k).max())
    nk = 2 * kmax + 1
    out = []
    ex = np.exp(2j * math.pi * np.outer((np.arange(nx) + offsets[0]) / nx, np.arange(-kmax, kmax + 1)))
    ey = np.exp(2j * math.pi * np.outer((np.arange(ny) + offsets[1]) / ny, np.arange(-kmax, kmax + 1)))
    ez = np.exp(2j * math.pi * np.outer((np.arange(nz) + offsets[2]) / nz, np.arange(-kmax, kmax + 1)))
    idx = (k.astype(int) + kmax)
    for c in range(a.shape[1]):
        C = np.zeros((nk, nk, nk), dtype=np.complex128)  # [kz, ky, kx]
        np.add.at(C, (idx[:, 2], idx[:, 1], idx[:, 0]), a[:, c] * np.exp(1j * ph))
        T1 = C @ ex.T                                   # [kz, ky, x]
        T2 = np.einsum("yb,zbx->zyx", ey, T1)            # [kz, y, x]
        f = (ez @ T2.reshape(nk, ny * nx)).real.reshape(nz, ny, nx)
        out.append(f)
    return out


def turbulence_box(n, seed, gamma=5.0 / 3.0, beta=100.0, mach=1.0, db_frac=0.1):
    """Config-2-style turbulence box on the unit cube (same modes for every n)."""
    if np.isscalar(n):
        n = (int(n),) * 3
    nx, ny, nz = n
    rho0, p0 = 1.0, 1.0
    cs = math.sqrt(gamma * p0 / rho0)
    kv, av, pv = mode_table(seed, 1, 8, slope=-2.0)
    # rms |v| of a sum of cosines over the periodic box: sqrt(sum |a|^2 / 2)
    vscale = mach * cs / math.sqrt(0.5 * float(np.sum(av * av)))
    vx, vy, vz = _eval_modes(kv, av * vscale, pv, n, (0.5, 0.5, 0.5))
    B0 = math.sqrt(2.0 * p0 / beta)
    kb, ab, pb = mode_table(seed + 7919, 1, 4, slope=-2.0)
    # |curl(a cos(2 pi k.x + p))| = 2 pi |k| |a| for a perpendicular to k
    kn = np.linalg.norm(kb, axis=1)
    brms = math.sqrt(0.5 * float(np.sum((2.0 * math.pi * kn[:, None] * ab) ** 2)))
    ab = ab * (db_frac * B0 / brms)
    Ax = _eval_modes(kb, ab[:, 0:1], pb, n, (0.5, 0.0, 0.0))[0]
    Ay = _eval_modes(kb, ab[:, 1:2], pb, n, (0.0, 0.5, 0.0))[0]
    Az = _eval_modes(kb, ab[:, 2:3], pb, n, (0.0, 0.0, 0.5))[0]
    bx, by, bz = curl_faces(Ax, Ay, Az, 1.0 / nx, 1.0 / ny, 1.0 / nz)
    bx = bx + B0
    W = np.empty((5, nz, ny, nx))
    W[0] = rho0
    W[1], W[2], W[3] = vx, vy, vz
    W[4] = p0
    return State(W=W, bx=bx, by=by, bz=bz, length=(1.0, 1.0, 1.0))


def _eval_modes_torch(k, a, ph, n, offsets, device):
    """_eval_modes with torch on a device (large grids); returns tensors."""
    import torch
    nx, ny, nz = n
    kmax = int(np.abs(k).max())
    nk = 2 * kmax + 1
    kr = torch.arange(-kmax, kmax + 1, dtype=torch.float64, device=device)
    def basis(m, off):
        x = (torch.arange(m, dtype=torch.float64, device=device) + off) / m
        return torch.exp(2j * math.pi * torch.outer(x, kr).to(torch.complex128))
    ex, ey, ez = basis(nx, offsets[0]), basis(ny, offsets[1]), basis(nz, offsets[2])
    idx = k.astype(int) + kmax
    out = []
    for c in range(a.shape[1]):
        C = np.zeros((nk, nk, nk), dtype=np.complex128)
        np.add.at(C, (idx[:, 2], idx[:, 1], idx[:, 0]), a[:, c] * np.exp(1j * ph))
        Ct = torch.from_numpy(C).to(device)
        T1 = Ct @ ex.T                                  # [kz, ky, x]
        T2 = torch.einsum("yb,zbx->zyx", ey, T1)         # [kz, y, x]
        f = (ez @ T2.reshape(nk, ny * nx)).real.reshape(nz, ny, nx).contiguous()
        out.append(f)
    return out


def _curl_faces_torch(Ax, Ay, Az, dx, dy, dz):
    import torch
    bx = (torch.roll(Az, -1, 1) - Az) / dy - (torch.roll(Ay, -1, 0) - Ay) / dz
    by = (torch.roll(Ax, -1, 0) - Ax) / dz - (torch.roll(Az, -1, 2) - Az) / dx
    bz = (torch.roll(Ay, -1, 2) - Ay) / dx - (torch.roll(Ax, -1, 1) - Ax) / dy
    bx = torch.cat([bx, bx[:, :, :1]], dim=2).contiguous()
    by = torch.cat([by, by[:, :1, :]], dim=1).contiguous()
    bz = torch.cat([bz, bz[:1, :, :]], dim=0).contiguous()
    return bx, by, bz


def turbulence_box_device(n, seed, device, gamma=5.0 / 3.0, beta=100.0, mach=1.0, db_frac=0.1):
    """turbulence_box evaluated with torch on ``device`` (same mode table and
    scaling; values agree with the NumPy version to rounding).  Returns a
    State whose arrays are device tensors."""
    import torch
    if np.isscalar(n):
        n = (int(n),) * 3
    nx, ny, nz = n
    rho0, p0 = 1.0, 1.0
    cs = math.sqrt(gamma * p0 / rho0)
    kv, av, pv = mode_table(seed, 1, 8, slope=-2.0)
    vscale = mach * cs / math.sqrt(0.5 * float(np.sum(av * av)))
    vx, vy, vz = _eval_modes_torch(kv, av * vscale, pv, n, (0.5, 0.5, 0.5), device)
    B0 = math.sqrt(2.0 * p0 / beta)
    kb, ab, pb = mode_table(seed + 7919, 1, 4, slope=-2.0)
    kn = np.linalg.norm(kb, axis=1)
    brms = math.sqrt(0.5 * float(np.sum((2.0 * math.pi * kn[:, None] * ab) ** 2)))
    ab = ab * (db_frac * B0 / brms)
    Ax = _eval_modes_torch(kb, ab[:, 0:1], pb, n, (0.5, 0.0, 0.0), device)[0]
    Ay = _eval_modes_torch(kb, ab[:, 1:2], pb, n, (0.0, 0.5, 0.0), device)[0]
    Az = _eval_modes_torch(kb, ab[:, 2:3], pb, n, (0.0, 0.0, 0.5), device)[0]
    bx, by, bz = _curl_faces_torch(Ax, Ay, Az, 1.0 / nx, 1.0 / ny, 1.0 / nz)
    del Ax, Ay, Az
    bx = bx + B0
    W = torch.empty((5, nz, ny, nx), dtype=torch.float64, device=device)
    W[0] = rho0
    W[1], W[2], W[3] = vx, vy, vz
    W[4] = p0
    return State(W=W, bx=bx, by=by, bz=bz, length=(1.0, 1.0, 1.0))
