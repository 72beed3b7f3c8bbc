"""TEST INFRASTRUCTURE ONLY: ctypes front end of the plain FP64 CPU oracle.

The oracle (``mhd_oracle.cpp``) restates the WOMBAT per-patch ideal-MHD step
(Mendygral et al. 2017, arXiv:1701.07452: App. A MHDTVD flux inside the 3D
CTU+CT integrator, Sec. "MHD in Three Dimensions", Steps 1-11) in plain C++
built without multiply-add contraction.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use
it.  It shares no code with the CUDA path in ``paper_1701_07452_gb300``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mhd_oracle.cpp")
_HDR = os.path.join(_HERE, "mhd_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libmhd_oracle.so")
_LIB_COUNT = os.path.join(_BUILD, "libmhd_oracle_count.so")
_CNT_HDR = os.path.join(_HERE, "flop_count.h")
_lock = threading.Lock()
_libs = {}

DEFAULT_EPS = (0.1, 0.0, 0.1, 0.0, 0.1, 0.0, 0.1)


def build(force: bool = False, count: bool = False) -> str:
    """Compile the oracle with g++ (-O2 -ffp-contract=off -fopenmp).  With
    count=True, the single-threaded operation-counting build
    (-DORACLE_COUNT_FLOPS, flop_count.h): the same results, plus per-section
    FP64 operation counts."""
    os.makedirs(_BUILD, exist_ok=True)
    target = _LIB_COUNT if count else _LIB
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR), os.path.getmtime(_CNT_HDR))
    if not force and os.path.exists(target) and os.path.getmtime(target) >= newest:
        return target
    tmp = target + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c++17"]
    cmd += ["-DORACLE_COUNT_FLOPS", "-Wno-unknown-pragmas"] if count else ["-fopenmp"]
    cmd += ["-o", tmp, _SRC]
    subprocess.check_call(cmd)
    os.replace(tmp, target)
    return target


def lib(count: bool = False):
    with _lock:
        if count not in _libs:
            path = build(count=count)
            L = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            L.or_create.restype = ctypes.c_void_p
            L.or_create.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 5 + [ip, dp] + \
                [ctypes.c_double] * 3
            L.or_destroy.argtypes = [ctypes.c_void_p]
            L.or_load.argtypes = [ctypes.c_void_p, dp, dp, dp, dp]
            L.or_load_primitive.argtypes = [ctypes.c_void_p, dp, dp, dp, dp]
            L.or_read.argtypes = [ctypes.c_void_p, dp, dp, dp, dp, dp]
            L.or_compute_dt.restype = ctypes.c_double
            L.or_compute_dt.argtypes = [ctypes.c_void_p]
            L.or_step.argtypes = [ctypes.c_void_p, ctypes.c_double]
            L.or_totals.argtypes = [ctypes.c_void_p, dp]
            L.or_divb_max.restype = ctypes.c_double
            L.or_divb_max.argtypes = [ctypes.c_void_p]
            L.or_counters.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong)]
            L.or_set_threads.argtypes = [ctypes.c_int]
            L.or_stage.restype = ctypes.c_longlong
            L.or_stage.argtypes = [ctypes.c_void_p, ctypes.c_int, dp, ctypes.c_longlong]
            L.or_face_eigen.argtypes = [dp, dp, ctypes.c_double, ctypes.c_double, dp, dp, dp, dp]
            L.or_set_protection.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double]
            L.or_set_source_scale.argtypes = [ctypes.c_void_p, ctypes.c_double]
            L.or_flux_pencil.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, dp, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, dp]
            L.or_step_1d.argtypes = [ctypes.c_int, dp, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, dp, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_int]
            llp = ctypes.POINTER(ctypes.c_longlong)
            L.or_flop_report.argtypes = [llp, llp, ctypes.c_int]
            L.or_flop_reset.argtypes = []
            _libs[count] = L
    return _libs[count]


# sections of the counting build, in the order of flop_count.h
FLOP_SECTIONS = ("none", "cell", "face", "hll", "limit", "emit", "eref", "edge", "ct", "trans",
                 "erefh", "update", "final", "dt")


def flop_report():
    """{section: (operations, units)} of the counting build since the last
    flop_reset()."""
    L = lib(count=True)
    n = len(FLOP_SECTIONS)
    f = (ctypes.c_longlong * n)()
    u = (ctypes.c_longlong * n)()
    got = L.or_flop_report(f, u, n)
    assert got == n, got
    return {name: (int(f[i]), int(u[i])) for i, name in enumerate(FLOP_SECTIONS)}


def flop_reset():
    lib(count=True).or_flop_reset()


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def set_threads(n: int) -> int:
    return lib().or_set_threads(int(n))


class Grid:
    """One periodic/outflow box evolved by the oracle (single grid, 5 ghosts)."""

    def __init__(self, n, length, gamma=5.0 / 3.0, cfl=0.8, bc=(0, 0, 0), eps=DEFAULT_EPS,
                 sweby=1.0, rho_floor=1e-20, p_floor=1e-20, dt_lag=False, counting=False):
        """counting=True runs the grid in the operation-counting build."""
        self._L = lib(count=counting)
        self.dt_lag = bool(dt_lag)
        self._lag_dt = None   # lagged dt: CFL dt of the previous step's start state
        self.n = tuple(int(x) for x in n)
        self.length = tuple(float(x) for x in length)
        self.gamma = float(gamma)
        bcs = (ctypes.c_int * 3)(*[int(b) for b in bc])
        epsa = np.ascontiguousarray(eps, dtype=np.float64)
        self._h = self._L.or_create(*self.n, *self.length, self.gamma, float(cfl), bcs, _p(epsa),
                                  float(sweby), float(rho_floor), float(p_floor))
        if not self._h:
            raise ValueError("oracle: invalid grid description")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.or_destroy(h)
            self._h = None

    def load(self, U, bx, by, bz):
        nx, ny, nz = self.n
        U = np.ascontiguousarray(U, dtype=np.float64)
        bx = np.ascontiguousarray(bx, dtype=np.float64)
        by = np.ascontiguousarray(by, dtype=np.float64)
        bz = np.ascontiguousarray(bz, dtype=np.float64)
        assert U.shape == (5, nz, ny, nx)
        assert bx.shape == (nz, ny, nx + 1) and by.shape == (nz, ny + 1, nx)
        assert bz.shape == (nz + 1, ny, nx)
        rc = self._L.or_load(self._h, _p(U), _p(bx), _p(by), _p(bz))
        if rc:
            raise RuntimeError(f"oracle load failed rc={rc}")
        self._lag_dt = None

    def load_primitive(self, W, bx, by, bz):
        nx, ny, nz = self.n
        W = np.ascontiguousarray(W, dtype=np.float64)
        assert W.shape == (5, nz, ny, nx)
        bx = np.ascontiguousarray(bx, dtype=np.float64)
        by = np.ascontiguousarray(by, dtype=np.float64)
        bz = np.ascontiguousarray(bz, dtype=np.float64)
        rc = self._L.or_load_primitive(self._h, _p(W), _p(bx), _p(by), _p(bz))
        if rc:
            raise RuntimeError(f"oracle load failed rc={rc}")
        self._lag_dt = None

    def load_state(self, st):
        self.load_primitive(st["W"], st["bx"], st["by"], st["bz"])

    def read(self):
        nx, ny, nz = self.n
        U = np.empty((5, nz, ny, nx))
        bx = np.empty((nz, ny, nx + 1))
        by = np.empty((nz, ny + 1, nx))
        bz = np.empty((nz + 1, ny, nx))
        B = np.empty((3, nz, ny, nx))
        self._L.or_read(self._h, _p(U), _p(bx), _p(by), _p(bz), _p(B))
        return U, bx, by, bz, B

    def dt(self) -> float:
        return self._L.or_compute_dt(self._h)

    def step(self, dt: float) -> int:
        return self._L.or_step(self._h, float(dt))

    def advance(self, nsteps: int, t_end: float | None = None, dt: float | None = None):
        """nsteps CFL (or fixed-dt) steps; stops at t_end (measured from this
        call) if given.  With dt_lag each step takes the CFL dt of the previous
        step's start state (the first two steps after a load both take the
        loaded state's).  Returns t."""
        t = 0.0
        for _ in range(int(nsteps)):
            if dt is not None:
                h = float(dt)
            else:
                h = self.dt()
                if self.dt_lag:
                    h_now = h
                    if self._lag_dt is not None:
                        h = self._lag_dt
            last = False
            if t_end is not None:
                rem = t_end - t
                if not rem > 0.0:
                    break
                # the step that reaches t_end lands on it and leaves no
                # sliver below 1e-10 of a step
                if h >= rem * (1.0 - 1e-10):
                    h, last = rem, True
            rc = self.step(h)
            if rc:
                raise RuntimeError(f"oracle step returned {rc}")
            if dt is None and self.dt_lag:
                self._lag_dt = h_now
            t = t_end if last else t + h
        return t

    def totals(self):
        out = np.zeros(8)
        self._L.or_totals(self._h, _p(out))
        return out

    def divb_max(self) -> float:
        return self._L.or_divb_max(self._h)

    def counters(self):
        """(floor hits, unphysical zones, HLL faces) over all steps."""
        out = (ctypes.c_longlong * 3)()
        self._L.or_counters(self._h, out)
        return int(out[0]), int(out[1]), int(out[2])

    def set_protection(self, prot_rho: float = 0.0, prot_p: float = 0.0):
        """Protection floors of App. A (faces next to a zone below them use HLL)."""
        if self._L.or_set_protection(self._h, float(prot_rho), float(prot_p)):
            raise ValueError("oracle: invalid protection floors")

    def set_source_scale(self, s: float):
        """Test ablation: multiply the div B source of Steps 5 and 7 by s."""
        if self._L.or_set_source_scale(self._h, float(s)):
            raise ValueError("oracle: invalid source scale")

    def stage(self, which: int):
        nx, ny, nz = self.n
        cap = 8 * (nx + 1) * (ny + 1) * (nz + 1)
        out = np.empty(cap)
        w = self._L.or_stage(self._h, int(which), _p(out), cap)
        return out[:w]


def face_eigen(qL, qR, b, gamma):
    qL = np.ascontiguousarray(qL, dtype=np.float64)
    qR = np.ascontiguousarray(qR, dtype=np.float64)
    lam = np.empty(7); alpha = np.empty(7); R = np.empty(49); L = np.empty(49)
    rc = lib().or_face_eigen(_p(qL), _p(qR), float(b), float(gamma), _p(lam), _p(alpha), _p(R), _p(L))
    if rc:
        raise ValueError("unphysical Roe state")
    return lam, alpha, R.reshape(7, 7), L.reshape(7, 7)


def flux_pencil(cells, bface, dtdx, dx_over_2dt, gamma, eps=DEFAULT_EPS, sweby=1.0,
                prot_rho=0.0, prot_p=0.0, with_hll=False):
    """Face fluxes of one pencil; with_hll also returns the number of output
    faces that took the HLL flux."""
    cells = np.ascontiguousarray(cells, dtype=np.float64)
    bface = np.ascontiguousarray(bface, dtype=np.float64)
    n = cells.shape[0]
    out = np.full((n + 1, 7), np.nan)
    epsa = np.ascontiguousarray(eps, dtype=np.float64)
    nh = lib().or_flux_pencil(n, _p(cells), _p(bface), float(dtdx), float(dx_over_2dt),
                              float(gamma), _p(epsa), float(sweby), float(prot_rho),
                              float(prot_p), _p(out))
    if nh < 0:
        raise ValueError("flux pencil: invalid arguments")
    return (out, nh) if with_hll else out


def step_1d(q, b, dt, dx, gamma, eps=DEFAULT_EPS, sweby=1.0, prot_rho=0.0, prot_p=0.0,
            outflow=False, with_hll=False):
    """One 1D step (periodic or zero-gradient ends); with_hll also returns the
    number of faces that took the HLL flux."""
    q = np.ascontiguousarray(q, dtype=np.float64).copy()
    epsa = np.ascontiguousarray(eps, dtype=np.float64)
    nh = lib().or_step_1d(q.shape[0], _p(q), float(b), float(dt), float(dx), float(gamma),
                          _p(epsa), float(sweby), float(prot_rho), float(prot_p), int(outflow))
    if nh < 0:
        raise ValueError("1d step: invalid arguments")
    return (q, nh) if with_hll else q
