"""Thin ctypes binding of ``libwombat_gb300.so`` (C ABI in include/wombat.h).

Argument marshalling only: every step of the MHD update runs in the
library's CUDA kernels.  PyTorch provides the device workspace (a uint8
tensor the caller owns) and the CUDA stream.  There is no CPU fallback: if
the library cannot be built or loaded, or no CUDA device is present, the
calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

WB_OK, WB_ERR_INVALID, WB_ERR_NOMEM, WB_ERR_CUDA, WB_ERR_UNPHYSICAL, WB_ERR_TIMEOUT = range(6)
WB_BC_PERIODIC, WB_BC_OUTFLOW = 0, 1
DEFAULT_EPS = (0.1, 0.0, 0.1, 0.0, 0.1, 0.0, 0.1)

EXPORTED = (
    "wb_desc_default", "wb_grid_bytes", "wb_grid_create", "wb_grid_destroy", "wb_load_state",
    "wb_load_primitive", "wb_compute_dt", "wb_advance", "wb_read_state", "wb_conserved_totals",
    "wb_divb_max", "wb_counters", "wb_last_error", "wb_debug_stage", "wb_measure_fp64_peak",
    "wb_profile_sweeps", "wb_profile_read", "wb_step_noalloc", "wb_noalloc_last_error",
    "wb_selftest_math", "wb_selftest_bits", "wb_batch_bytes", "wb_batch_create", "wb_batch_destroy", "wb_batch_load",
    "wb_batch_set_steps", "wb_batch_advance", "wb_batch_read", "wb_batch_counters",
    "wb_batch_autotune", "wb_batch_config", "wb_batch_get_config", "wb_batch_last_error",
    "wb_pool_bytes", "wb_pool_create", "wb_pool_admit", "wb_pool_release", "wb_pool_free_bytes",
    "wb_batch_steps_left", "wb_batch_stage_timer", "wb_batch_stage_times", "wb_batch_set_form",
    "wb_batch_get_form", "wb_check_flags", "wb_check_selftest",
)

BATCH_FORMS = {"persistent": 0, "staged": 1}


class WbDesc(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int * 3),
        ("patches", ctypes.c_int * 3),
        ("length", ctypes.c_double * 3),
        ("gamma", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("bc", ctypes.c_int * 3),
        ("eps", ctypes.c_double * 7),
        ("sweby_beta", ctypes.c_double),
        ("rho_floor", ctypes.c_double),
        ("p_floor", ctypes.c_double),
        ("batch_patches", ctypes.c_int),
        ("prot_rho", ctypes.c_double),
        ("prot_p", ctypes.c_double),
        ("dt_lag", ctypes.c_int),
        ("keep_stages", ctypes.c_int),
    ]


class WbCounters(ctypes.Structure):
    _fields_ = [
        ("steps", ctypes.c_longlong),
        ("floor_hits", ctypes.c_longlong),
        ("unphysical", ctypes.c_longlong),
        ("t", ctypes.c_double),
        ("last_dt", ctypes.c_double),
        ("hll_faces", ctypes.c_longlong),
    ]


class WombatError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"wombat error {code}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return os.path.join(_build.OUT, "checked", "libwombat_gb300.so") if _checked() else _build.LIB


def _checked() -> bool:
    """WOMBAT_CHECKED=1 in the environment loads the index-checked build."""
    return os.environ.get("WOMBAT_CHECKED", "") == "1"


def lib(build: bool = True):
    """Load (building first if needed) the CUDA library.  Raises if absent."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build(checked=_checked()) if build else library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"libwombat_gb300.so not found at {path}")
            L = ctypes.CDLL(path)
            vp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
            L.wb_desc_default.argtypes = [ctypes.POINTER(WbDesc), ctypes.c_int, ctypes.c_int, ctypes.c_int]
            L.wb_desc_default.restype = None
            L.wb_grid_bytes.argtypes = [ctypes.POINTER(WbDesc), ctypes.POINTER(ctypes.c_size_t)]
            L.wb_grid_create.argtypes = [ctypes.POINTER(WbDesc), vp, ctypes.c_size_t, vp,
                                         ctypes.POINTER(vp)]
            L.wb_grid_destroy.argtypes = [vp]
            L.wb_load_state.argtypes = [vp, vp, vp, vp, vp, ctypes.c_int]
            L.wb_load_primitive.argtypes = [vp, vp, vp, vp, vp, ctypes.c_int]
            L.wb_compute_dt.argtypes = [vp, dp]
            L.wb_advance.argtypes = [vp, ctypes.c_int, ctypes.c_double, dp]
            L.wb_read_state.argtypes = [vp, vp, vp, vp, vp, vp, ctypes.c_int]
            L.wb_conserved_totals.argtypes = [vp, dp]
            L.wb_divb_max.argtypes = [vp, dp]
            L.wb_counters.argtypes = [vp, ctypes.POINTER(WbCounters)]
            L.wb_last_error.argtypes = [vp]
            L.wb_last_error.restype = ctypes.c_char_p
            L.wb_debug_stage.argtypes = [vp, ctypes.c_int, dp, ctypes.c_longlong,
                                         ctypes.POINTER(ctypes.c_longlong)]
            L.wb_measure_fp64_peak.argtypes = [vp, dp]
            L.wb_profile_sweeps.argtypes = [vp, ctypes.c_int]
            L.wb_profile_read.argtypes = [vp, dp, ctypes.POINTER(ctypes.c_longlong)]
            L.wb_step_noalloc.argtypes = [ctypes.POINTER(WbDesc)] + [vp] * 10
            L.wb_selftest_math.argtypes = [vp, ctypes.c_int, dp]
            L.wb_selftest_bits.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong)]
            L.wb_batch_bytes.argtypes = [ctypes.c_int, ctypes.POINTER(WbDesc), ctypes.c_size_t,
                                         ctypes.POINTER(ctypes.c_size_t)]
            L.wb_batch_create.argtypes = [ctypes.c_int, ctypes.POINTER(WbDesc), ctypes.c_size_t, vp,
                                          ctypes.c_size_t, vp, ctypes.POINTER(vp)]
            L.wb_batch_destroy.argtypes = [vp]
            L.wb_batch_load.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp, ctypes.c_int, ctypes.c_int]
            L.wb_batch_set_steps.argtypes = [vp, ctypes.c_int, ctypes.c_int]
            L.wb_batch_advance.argtypes = [vp, ctypes.c_int, ctypes.c_int]
            L.wb_batch_read.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp, vp, ctypes.c_int]
            L.wb_batch_counters.argtypes = [vp, ctypes.c_int, ctypes.POINTER(WbCounters)]
            L.wb_batch_autotune.argtypes = [vp, ctypes.c_int, dp]
            L.wb_batch_config.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_longlong]
            L.wb_batch_stage_timer.argtypes = [vp, ctypes.c_int]
            L.wb_batch_stage_times.argtypes = [vp, dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
            L.wb_batch_get_config.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                              ctypes.POINTER(ctypes.c_int)]
            L.wb_check_flags.argtypes = [ctypes.POINTER(ctypes.c_uint)]
            L.wb_check_selftest.argtypes = [ctypes.POINTER(ctypes.c_int)]
            L.wb_batch_set_form.argtypes = [vp, ctypes.c_int]
            L.wb_batch_get_form.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
            L.wb_batch_last_error.argtypes = [vp]
            L.wb_batch_last_error.restype = ctypes.c_char_p
            L.wb_pool_bytes.argtypes = [ctypes.c_size_t, ctypes.c_size_t, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_size_t)]
            L.wb_pool_create.argtypes = [ctypes.POINTER(WbDesc), ctypes.c_size_t, ctypes.c_size_t, ctypes.c_int,
                                         ctypes.c_int, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)]
            L.wb_pool_admit.argtypes = [vp, ctypes.POINTER(WbDesc), ctypes.POINTER(ctypes.c_int)]
            L.wb_pool_release.argtypes = [vp, ctypes.c_int]
            L.wb_pool_free_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]
            L.wb_batch_steps_left.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
            L.wb_noalloc_last_error.argtypes = []
            L.wb_noalloc_last_error.restype = ctypes.c_char_p
            _lib = L
    return _lib


def make_desc(n, patches=(1, 1, 1), length=None, gamma=5.0 / 3.0, cfl=0.8, bc=(0, 0, 0),
              eps=DEFAULT_EPS, sweby=1.0, rho_floor=1e-20, p_floor=1e-20, batch_patches=0,
              prot_rho=0.0, prot_p=0.0, dt_lag=False, keep_stages=False):
    d = WbDesc()
    lib().wb_desc_default(ctypes.byref(d), int(n[0]), int(n[1]), int(n[2]))
    for a in range(3):
        d.patches[a] = int(patches[a])
        d.length[a] = float(length[a] if length is not None else n[a])
        d.bc[a] = int(bc[a])
    for k in range(7):
        d.eps[k] = float(eps[k])
    d.gamma, d.cfl, d.sweby_beta = float(gamma), float(cfl), float(sweby)
    d.rho_floor, d.p_floor = float(rho_floor), float(p_floor)
    d.batch_patches = int(batch_patches)
    d.prot_rho, d.prot_p = float(prot_rho), float(prot_p)
    d.dt_lag = int(bool(dt_lag))
    d.keep_stages = int(bool(keep_stages))
    return d


def grid_bytes(desc: WbDesc) -> int:
    out = ctypes.c_size_t(0)
    rc = lib().wb_grid_bytes(ctypes.byref(desc), ctypes.byref(out))
    if rc:
        raise WombatError(rc, "invalid descriptor")
    return int(out.value)


def _ptr(a):
    """Raw pointer of a numpy array or a torch tensor."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


class Grid:
    """A grid of patches advanced on the current CUDA device.

    The device workspace is a torch uint8 tensor owned by this object (the
    caller side of the C ABI); the stream is torch's current stream unless
    one is given."""

    def __init__(self, n, patches=(1, 1, 1), length=None, stream=None, **kw):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("wombat: a CUDA device is required (no CPU fallback)")
        self.n = tuple(int(x) for x in n)
        self.desc = make_desc(self.n, patches, length, **kw)
        self.nbytes = grid_bytes(self.desc)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.workspace = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        rc = lib().wb_grid_create(ctypes.byref(self.desc), ctypes.c_void_p(self.workspace.data_ptr()),
                                  ctypes.c_size_t(self.nbytes), ctypes.c_void_p(self.stream.cuda_stream),
                                  ctypes.byref(h))
        if rc:
            raise WombatError(rc, "grid create failed")
        self._h = h

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().wb_grid_destroy(h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc:
            msg = lib().wb_last_error(self._h)
            raise WombatError(rc, msg.decode() if msg else "")

    # -- load / read -------------------------------------------------------
    def _prep(self, a, shape, on_device):
        if on_device:
            assert tuple(a.shape) == shape and a.is_contiguous()
            return a
        a = np.ascontiguousarray(a, dtype=np.float64)
        assert a.shape == shape, (a.shape, shape)
        return a

    def _shapes(self):
        nx, ny, nz = self.n
        return (5, nz, ny, nx), (nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)

    def load(self, U, bx, by, bz, on_device=False, primitive=False):
        sU, sx, sy, sz = self._shapes()
        arrs = [self._prep(U, sU, on_device), self._prep(bx, sx, on_device),
                self._prep(by, sy, on_device), self._prep(bz, sz, on_device)]
        fn = lib().wb_load_primitive if primitive else lib().wb_load_state
        self._check(fn(self._h, *[ctypes.c_void_p(_ptr(a)) for a in arrs], int(bool(on_device))))

    def load_state(self, st):
        """Load a dict with primitive W and faces (see initial_conditions)."""
        self.load(st["W"], st["bx"], st["by"], st["bz"], primitive=True)

    def read(self, on_device=False, out=None):
        sU, sx, sy, sz = self._shapes()
        nx, ny, nz = self.n
        if out is None:
            if on_device:
                import torch
                kw = dict(dtype=torch.float64, device=self.device)
                out = (torch.empty(sU, **kw), torch.empty(sx, **kw), torch.empty(sy, **kw),
                       torch.empty(sz, **kw), torch.empty((3, nz, ny, nx), **kw))
            else:
                out = (np.empty(sU), np.empty(sx), np.empty(sy), np.empty(sz), np.empty((3, nz, ny, nx)))
        self._check(lib().wb_read_state(self._h, *[ctypes.c_void_p(_ptr(a)) for a in out],
                                        int(bool(on_device))))
        return out

    # -- stepping ----------------------------------------------------------
    def dt(self) -> float:
        out = ctypes.c_double(0.0)
        self._check(lib().wb_compute_dt(self._h, ctypes.byref(out)))
        return out.value

    def advance(self, nsteps: int, t_end: float = 0.0, sync: bool = True):
        """Enqueue nsteps steps; with sync, wait and return the time since load."""
        if sync:
            t = ctypes.c_double(0.0)
            self._check(lib().wb_advance(self._h, int(nsteps), float(t_end), ctypes.byref(t)))
            return t.value
        self._check(lib().wb_advance(self._h, int(nsteps), float(t_end), None))
        return None

    def totals(self):
        out = np.zeros(8)
        self._check(lib().wb_conserved_totals(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def divb_max(self) -> float:
        out = ctypes.c_double(0.0)
        self._check(lib().wb_divb_max(self._h, ctypes.byref(out)))
        return out.value

    def counters(self):
        c = WbCounters()
        self._check(lib().wb_counters(self._h, ctypes.byref(c)))
        return {"steps": c.steps, "floor_hits": c.floor_hits, "unphysical": c.unphysical,
                "t": c.t, "last_dt": c.last_dt, "hll_faces": c.hll_faces}

    def profile_sweeps(self, enable: bool):
        self._check(lib().wb_profile_sweeps(self._h, int(bool(enable))))

    def profile_read(self):
        ms = ctypes.c_double(0.0)
        n = ctypes.c_longlong(0)
        self._check(lib().wb_profile_read(self._h, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def selftest_math(self, n: int = 1 << 20):
        out = np.zeros(2)
        self._check(lib().wb_selftest_math(self._h, int(n), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return float(out[0]), float(out[1])

    BITS_TESTS = ("zero", "twice", "order_less", "rate_key", "pos", "neg", "normal_pos", "abs_less",
                  "minmod", "half", "fabs", "flip", "le_nonneg", "below_floor", "finite")

    def selftest_bits(self, n: int = 1 << 22):
        """Mismatches of each integer-pipe helper against its FP64 definition."""
        out = np.zeros(len(self.BITS_TESTS), dtype=np.int64)
        self._check(lib().wb_selftest_bits(self._h, int(n), out.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong))))
        return dict(zip(self.BITS_TESTS, (int(x) for x in out)))

    def stage(self, which: int):
        nx, ny, nz = self.n
        cap = 8 * (nx + 1) * (ny + 1) * (nz + 1)
        out = np.empty(cap)
        w = ctypes.c_longlong(0)
        self._check(lib().wb_debug_stage(self._h, int(which), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         cap, ctypes.byref(w)))
        return out[: w.value]


class Batch:
    """Many independent single-patch boxes advanced together, by one
    persistent kernel or by one launch per stage (set_form), each with its own
    dt (wb_batch_* of the C ABI).  boxes: list of dicts with keys n, length
    and optional bc; physics keywords are shared by every box."""

    def __init__(self, boxes, work_budget=0, stream=None, **kw):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("wombat: a CUDA device is required (no CPU fallback)")
        self.phys_kw = kw
        self.nbox = len(boxes)
        self.n = [tuple(int(x) for x in b["n"]) for b in boxes]
        arr = (WbDesc * self.nbox)()
        for i, b in enumerate(boxes):
            d = make_desc(b["n"], (1, 1, 1), b.get("length"), bc=b.get("bc", (0, 0, 0)), **kw)
            arr[i] = d
        self._descs = arr
        nbytes = ctypes.c_size_t(0)
        rc = lib().wb_batch_bytes(self.nbox, arr, ctypes.c_size_t(int(work_budget)), ctypes.byref(nbytes))
        if rc:
            raise WombatError(rc, "invalid batch description")
        self.nbytes = int(nbytes.value)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.workspace = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        rc = lib().wb_batch_create(self.nbox, arr, ctypes.c_size_t(int(work_budget)),
                                   ctypes.c_void_p(self.workspace.data_ptr()), ctypes.c_size_t(self.nbytes),
                                   ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if rc:
            raise WombatError(rc, "batch create failed")
        self._h = h

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().wb_batch_destroy(h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc:
            msg = lib().wb_batch_last_error(self._h)
            raise WombatError(rc, msg.decode() if msg else "")

    def load(self, box, U, bx, by, bz, primitive=False, on_device=False):
        arrs = [U, bx, by, bz]
        if not on_device:
            arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in arrs]
        self._check(lib().wb_batch_load(self._h, int(box), *[ctypes.c_void_p(_ptr(a)) for a in arrs],
                                        int(bool(on_device)), int(bool(primitive))))

    def load_state(self, box, st):
        self.load(box, st["W"], st["bx"], st["by"], st["bz"], primitive=True)

    def set_steps(self, box, nsteps):
        self._check(lib().wb_batch_set_steps(self._h, int(box), int(nsteps)))

    def advance(self, nsteps, use_graph=True):
        self._check(lib().wb_batch_advance(self._h, int(nsteps), int(bool(use_graph))))

    def read(self, box):
        nx, ny, nz = self.n[box]
        return self._read(box, nx, ny, nz)

    def _read(self, box, nx, ny, nz):
        out = (np.empty((5, nz, ny, nx)), np.empty((nz, ny, nx + 1)), np.empty((nz, ny + 1, nx)),
               np.empty((nz + 1, ny, nx)), np.empty((3, nz, ny, nx)))
        self._check(lib().wb_batch_read(self._h, int(box), *[ctypes.c_void_p(_ptr(a)) for a in out], 0))
        return out

    def counters(self, box):
        c = WbCounters()
        self._check(lib().wb_batch_counters(self._h, int(box), ctypes.byref(c)))
        return {"steps": c.steps, "floor_hits": c.floor_hits, "unphysical": c.unphysical,
                "t": c.t, "last_dt": c.last_dt, "hll_faces": c.hll_faces}

    def autotune(self, trial_steps=1):
        ms = ctypes.c_double(0.0)
        self._check(lib().wb_batch_autotune(self._h, int(trial_steps), ctypes.byref(ms)))
        return ms.value

    def config(self, seg_len=0, blocks_per_sm=0, barrier_budget_cycles=0):
        self._check(lib().wb_batch_config(self._h, int(seg_len), int(blocks_per_sm),
                                          ctypes.c_longlong(int(barrier_budget_cycles))))

    def stage_timer(self, on=True):
        self._check(lib().wb_batch_stage_timer(self._h, int(bool(on))))

    def stage_times(self):
        """Accumulated milliseconds per stage (see wb_batch_stage_times)."""
        ms = (ctypes.c_double * 32)()
        cnt = ctypes.c_int(0)
        self._check(lib().wb_batch_stage_times(self._h, ms, 32, ctypes.byref(cnt)))
        names = ["dt", "pred_sweeps", "eref", "wrap_fp", "edges_pred", "wrap_edges", "ct_half",
                 "wrap_bh", "transverse", "wrap_qh", "corr_sweeps", "wrap_fc", "eref_half",
                 "wrap_erefh", "edges_corr", "wrap_edgesh", "ct_final", "update", "halo"]
        return {names[i] if i < len(names) else str(i): ms[i] for i in range(cnt.value)}

    def set_form(self, form):
        """"persistent" (one cooperative launch per advance) or "staged" (one
        launch per stage); results are identical."""
        self._check(lib().wb_batch_set_form(self._h, BATCH_FORMS[form]))

    def get_config(self):
        a, b, c = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        self._check(lib().wb_batch_get_config(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        f = ctypes.c_int(0)
        self._check(lib().wb_batch_get_form(self._h, ctypes.byref(f)))
        form = {v: k for k, v in BATCH_FORMS.items()}[f.value]
        return {"seg_len": a.value, "blocks_per_sm": b.value, "groups": c.value, "form": form}


class Pool(Batch):
    """A batch whose boxes join and leave between launches (wb_pool_*): the
    state region is the HBM budget of resident runs."""

    def __init__(self, state_bytes, work_bytes, max_boxes=256, max_n=256, stream=None, **kw):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("wombat: a CUDA device is required (no CPU fallback)")
        self.phys_kw = kw
        self.physics = make_desc((8, 8, 8), **kw)
        self.max_boxes = int(max_boxes)
        nbytes = ctypes.c_size_t(0)
        rc = lib().wb_pool_bytes(ctypes.c_size_t(int(state_bytes)), ctypes.c_size_t(int(work_bytes)),
                                 self.max_boxes, int(max_n), ctypes.byref(nbytes))
        if rc:
            raise WombatError(rc, "invalid pool description")
        self.nbytes = int(nbytes.value)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.workspace = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        rc = lib().wb_pool_create(ctypes.byref(self.physics), ctypes.c_size_t(int(state_bytes)),
                                  ctypes.c_size_t(int(work_bytes)), self.max_boxes, int(max_n),
                                  ctypes.c_void_p(self.workspace.data_ptr()), ctypes.c_size_t(self.nbytes),
                                  ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if rc:
            raise WombatError(rc, "pool create failed")
        self._h = h
        self.n = {}

    def admit(self, n, length=None, bc=(0, 0, 0)):
        """Slot of a newly admitted box, or None when it does not fit now."""
        d = make_desc(n, (1, 1, 1), length, bc=bc, **self.phys_kw)
        slot = ctypes.c_int(-1)
        rc = lib().wb_pool_admit(self._h, ctypes.byref(d), ctypes.byref(slot))
        if rc == WB_ERR_NOMEM:
            return None
        self._check(rc)
        self.n[slot.value] = tuple(int(x) for x in n)
        return slot.value

    def release(self, box):
        self._check(lib().wb_pool_release(self._h, int(box)))
        self.n.pop(box, None)

    def steps_left(self):
        out = (ctypes.c_int * self.max_boxes)()
        self._check(lib().wb_batch_steps_left(self._h, out))
        return list(out)

    def free_bytes(self):
        a, b = ctypes.c_size_t(0), ctypes.c_size_t(0)
        self._check(lib().wb_pool_free_bytes(self._h, ctypes.byref(a), ctypes.byref(b)))
        return int(a.value), int(b.value)


def step_noalloc(desc: WbDesc, U, bx, by, bz, U_out, bx_out, by_out, bz_out, dt_out=None,
                 stream=None):
    """One step of a small single box through wb_step_noalloc (device tensors
    in and out; no device memory is allocated by the library)."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    args = [U, bx, by, bz, U_out, bx_out, by_out, bz_out, dt_out]
    rc = lib().wb_step_noalloc(ctypes.byref(desc), *[ctypes.c_void_p(_ptr(a)) for a in args],
                               ctypes.c_void_p(s.cuda_stream))
    if rc:
        raise WombatError(rc, lib().wb_noalloc_last_error().decode())


def check_flags() -> int:
    """Check words of the index-checked build (0: no bad index since the last
    call).  Raises in an unchecked build."""
    out = ctypes.c_uint(0)
    rc = lib().wb_check_flags(ctypes.byref(out))
    if rc:
        raise WombatError(rc, "not the checked build (set WOMBAT_CHECKED=1)")
    return int(out.value)


def check_selftest() -> bool:
    """The checked build flags an out-of-range index formed by a probe kernel."""
    out = ctypes.c_int(0)
    rc = lib().wb_check_selftest(ctypes.byref(out))
    if rc:
        raise WombatError(rc, "not the checked build (set WOMBAT_CHECKED=1)")
    return bool(out.value)


def measure_fp64_peak(stream=None) -> float:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    out = ctypes.c_double(0.0)
    rc = lib().wb_measure_fp64_peak(ctypes.c_void_p(s.cuda_stream), ctypes.byref(out))
    if rc:
        raise WombatError(rc, "fp64 probe failed")
    return out.value
