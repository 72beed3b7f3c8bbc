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
           "curl_faces", "State"]


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
