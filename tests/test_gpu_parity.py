"""GPU path (C ABI libwombat_gb300.so) against the FP64 oracle on the same
seeded inputs.  Tolerances (per zone, relative, guarded): 1e-11 after one
step, 1e-8 after 100 steps; conserved totals 1e-12; patch decomposition and
halo indexing bit-exact against the single-grid run."""
import numpy as np
import pytest

from parity import TIGHT, rel_err, state_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_07452_gb300 import binding
    binding.lib()
    return binding


def make_pair(wb, oracle_mod, st, n, patches=(1, 1, 1), **kw):
    g = wb.Grid(n, patches=patches, length=st["length"], **kw)
    g.load_state(st)
    o = oracle_mod.Grid(n, st["length"], **{k: v for k, v in kw.items()
                                            if k not in ("batch_patches", "keep_stages")})
    o.load_state(st)
    return g, o


def test_load_and_dt_match(wb, oracle_mod):
    from paper_1701_07452_gb300.initial_conditions import random_box
    st = random_box(12, seed=3)
    g, o = make_pair(wb, oracle_mod, st, (12, 12, 12))
    assert state_err(g.read(), o.read()) < 1e-14
    assert abs(g.dt() - o.dt()) <= 1e-14 * o.dt()


def test_stage_parity_one_step(wb, oracle_mod):
    from paper_1701_07452_gb300.initial_conditions import random_box
    st = random_box((13, 11, 12), seed=5)
    n = (13, 11, 12)
    g, o = make_pair(wb, oracle_mod, st, n, keep_stages=True)
    dt = o.dt()
    g.advance(1)
    assert o.step(dt) == 0
    for which in range(12):
        a, b = g.stage(which), o.stage(which)
        assert a.shape == b.shape, which
        err = rel_err(a, b)
        assert err < 1e-11, (which, err)
    assert state_err(g.read(), o.read()) < 1e-11
    assert state_err(g.read(), o.read(), TIGHT) < 1e-11


@pytest.mark.parametrize("n,steps,tol", [((32, 32, 32), 10, 1e-10), ((24, 20, 16), 1, 1e-11)])
def test_random_box_parity(wb, oracle_mod, n, steps, tol):
    from paper_1701_07452_gb300.initial_conditions import random_box
    st = random_box(n, seed=1)
    g, o = make_pair(wb, oracle_mod, st, n)
    t_g = g.advance(steps)
    t_o = o.advance(steps)
    assert abs(t_g - t_o) <= 1e-13 * t_o
    assert state_err(g.read(), o.read()) < tol
    # under the tight guard: 1e-11 after one step, 1e-8 after ten
    assert state_err(g.read(), o.read(), TIGHT) < (1e-11 if steps == 1 else 1e-8)
    tg, to = g.totals(), o.totals()
    scale = np.array([abs(to[0]), abs(to[0]), abs(to[0]), abs(to[0]), abs(to[4]), 1, 1, 1])
    assert np.all(np.abs(tg - to) <= 1e-12 * np.maximum(scale, np.abs(to)))
    assert g.counters()["unphysical"] == 0


@pytest.mark.parametrize("eps,sweby", [
    ((0.1, 0.05, 0.1, 0.02, 0.1, 0.05, 0.1), 1.0),   # every wave with an entropy fix: generic sweep
    ((0.1, 0.0, 0.1, 0.0, 0.1, 0.0, 0.1), 1.5),      # the default eps_k, SWEBY beta = 1.5
    ((0.0,) * 7, 2.0),                                # no entropy fix, SWEBY beta = 2
    ((0.25, 0.0, 0.25, 0.0, 0.25, 0.0, 0.25), 1.0),   # a wide band on the fast and slow waves
])
def test_entropy_fix_and_limiter_parity(wb, oracle_mod, eps, sweby):
    """The App. A flux with other entropy-fix parameters eps_k (the sweep
    specialised for eps = 0 on the Alfven and entropy waves, and the generic
    one, whose beta_k takes the Q_k band test on every wave) and other SWEBY
    beta, against the oracle: 1e-11 after one step, 1e-10 after ten; a batch
    box with the same parameters gives the grid's bits."""
    from paper_1701_07452_gb300.initial_conditions import random_box
    n = (24, 20, 16)
    st = random_box(n, seed=7)
    for steps, tol in ((1, 1e-11), (10, 1e-10)):
        g, o = make_pair(wb, oracle_mod, st, n, eps=eps, sweby=sweby)
        t_g = g.advance(steps)
        t_o = o.advance(steps)
        assert abs(t_g - t_o) <= 1e-13 * t_o
        err = state_err(g.read(), o.read())
        assert err < tol, (steps, err)
    bt = wb.Batch([{"n": n, "length": st["length"]}], eps=eps, sweby=sweby)
    bt.load_state(0, st)
    bt.set_steps(-1, 10)
    bt.advance(10)
    for a, b in zip(bt.read(0), g.read()):
        assert np.array_equal(a, b)


def test_turbulence_parity_100_steps(wb, oracle_mod):
    from paper_1701_07452_gb300.initial_conditions import turbulence_box
    n = (24, 24, 24)
    st = turbulence_box(n, seed=2)
    g, o = make_pair(wb, oracle_mod, st, n)
    g.advance(100)
    o.advance(100)
    assert state_err(g.read(), o.read()) < 1e-8
    assert state_err(g.read(), o.read(), TIGHT) < 1e-8


def test_turbulence_parity_100_steps_balanced_sweep(wb, oracle_mod):
    """100 steps of the turbulence data at 64^3, where every sweep launch runs
    the balanced form (equal runs of 32-pencil-group faces per resident warp,
    the form the 256^3 bench box takes), against the oracle at 1e-8; totals
    to 1e-12 of their scale."""
    from paper_1701_07452_gb300.initial_conditions import turbulence_box
    n = (64, 64, 64)
    st = turbulence_box(n, seed=2)
    g, o = make_pair(wb, oracle_mod, st, n)
    t_g = g.advance(100)
    t_o = o.advance(100)
    assert abs(t_g - t_o) <= 1e-11 * t_o
    assert state_err(g.read(), o.read()) < 1e-8
    assert state_err(g.read(), o.read(), TIGHT) < 1e-8
    tg, to = g.totals(), o.totals()
    scale = np.array([abs(to[0])] * 4 + [abs(to[4])] + [1.0] * 3)
    assert np.all(np.abs(tg - to) <= 1e-12 * np.maximum(scale, np.abs(to)))
    assert g.counters()["unphysical"] == 0


@pytest.mark.parametrize("n,patches,batch", [(32, (2, 2, 2), 5), (32, (4, 2, 1), 5), (32, (8, 8, 8), 5),
                                              (64, (2, 2, 2), 3), (48, (3, 1, 2), 0), (32, (2, 2, 2), 0),
                                              (32, (4, 2, 1), 0)])
def test_patches_bit_exact(wb, n, patches, batch):
    """Patch decomposition changes the pencil-segment layout of the sweeps and
    how ghost values arise (recomputed rings when patches go through the
    pipeline in batches, neighbour images when all are resident, batch 0);
    every zone must still match the single grid bit for bit."""
    from paper_1701_07452_gb300.initial_conditions import random_box
    n = (n, n, n)
    st = random_box(n, seed=7)
    ref = wb.Grid(n, length=st["length"])
    ref.load_state(st)
    ref.advance(3)
    pg = wb.Grid(n, patches=patches, length=st["length"], batch_patches=batch)
    pg.load_state(st)
    pg.advance(3)
    for a, b in zip(ref.read(), pg.read()):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("patches,batch,bc", [((2, 2, 2), 0, (1, 1, 1)), ((4, 2, 1), 3, (1, 0, 1)),
                                              ((2, 1, 2), 2, (0, 1, 1))])
def test_patches_bit_exact_outflow(wb, patches, batch, bc):
    """Patched grids with outflow axes (the ghost rings recomputed at every
    stage; resident or pipelined patches): the last patch along an outflow
    axis takes its high boundary face as the zero-gradient copy when it
    averages the zone field (Step 11), the inner patches their neighbour's
    owned face; every zone must match the single grid bit for bit."""
    from paper_1701_07452_gb300.initial_conditions import random_box
    n = (32, 32, 32)
    st = random_box(n, seed=9)
    ref = wb.Grid(n, length=st["length"], bc=bc)
    ref.load_state(st)
    ref.advance(3)
    pg = wb.Grid(n, patches=patches, length=st["length"], bc=bc, batch_patches=batch)
    pg.load_state(st)
    pg.advance(3)
    for a, b in zip(ref.read(), pg.read()):
        assert np.array_equal(a, b)


def test_balanced_sweep_split(wb, oracle_mod):
    """Boxes large enough that every sweep launch hands each resident warp an
    equal run of (slot, 32-pencil group, face) units (dozens of units per warp
    on a 152-SM GPU at 4 resident 64-thread blocks per SM), with a ragged last
    group of pencils: one step against the oracle, and 2^3 resident patches
    against the single grid bit for bit (the runs then span slots)."""
    from paper_1701_07452_gb300.initial_conditions import turbulence_box
    n = (150, 136, 144)   # z sweep: 20400 pencils, the last group holds 16
    st = turbulence_box(n, seed=11)
    g, o = make_pair(wb, oracle_mod, st, n)
    g.advance(1)
    o.advance(1)
    assert state_err(g.read(), o.read()) < 1e-11
    n = (140, 140, 140)   # 4900 pencils per patch, the last group holds 4
    st = turbulence_box(n, seed=12)
    ref = wb.Grid(n, length=st["length"])
    ref.load_state(st)
    ref.advance(2)
    pg = wb.Grid(n, patches=(2, 2, 2), length=st["length"], batch_patches=0)
    pg.load_state(st)
    pg.advance(2)
    for a, b in zip(ref.read(), pg.read()):
        assert np.array_equal(a, b)


def test_uniform_state_bit_exact(wb):
    n = (10, 9, 8)
    W = np.zeros((5, n[2], n[1], n[0]))
    W[0], W[1], W[2], W[3], W[4] = 1.3, 0.2, -0.1, 0.05, 0.7
    bx = np.full((n[2], n[1], n[0] + 1), 0.4)
    by = np.full((n[2], n[1] + 1, n[0]), -0.3)
    bz = np.full((n[2] + 1, n[1], n[0]), 0.25)
    g = wb.Grid(n, length=(1.0, 1.0, 1.0))
    g.load(W, bx, by, bz, primitive=True)
    before = g.read()
    g.advance(5)
    after = g.read()
    for a, b in zip(before, after):
        assert np.array_equal(a, b)


def test_divb_and_conservation(wb):
    from paper_1701_07452_gb300.initial_conditions import turbulence_box
    n = (32, 32, 32)
    st = turbulence_box(n, seed=2)
    g = wb.Grid(n, length=st["length"])
    g.load_state(st)
    t0 = g.totals()
    U0 = g.read()[0]
    bmax = max(np.abs(st["bx"]).max(), np.abs(st["by"]).max(), np.abs(st["bz"]).max())
    for steps in (1, 9, 90):
        g.advance(steps)
        assert g.divb_max() <= 1e-13 * bmax * n[0]
    t1 = g.totals()
    mom_scale = np.abs(U0[1:4]).sum(axis=0).sum() / U0[0].size
    scale = np.array([abs(t0[0]), mom_scale, mom_scale, mom_scale, abs(t0[4]), bmax, bmax, bmax])
    assert np.all(np.abs(t1 - t0) <= 1e-13 * scale)


def test_outflow_sod_parity(wb, oracle_mod):
    n = (64, 1, 1)
    W = np.zeros((5, 1, 1, 64))
    x = (np.arange(64) + 0.5) / 64
    W[0, 0, 0] = np.where(x < 0.5, 1.0, 0.125)
    W[4, 0, 0] = np.where(x < 0.5, 1.0, 0.1)
    bx = np.zeros((1, 1, 65)); by = np.zeros((1, 2, 64)); bz = np.zeros((2, 1, 64))
    kw = dict(gamma=1.4, bc=(1, 0, 0))
    L = (1.0, 1e3, 1e3)
    g = wb.Grid(n, length=L, **kw)
    g.load(W, bx, by, bz, primitive=True)
    o = oracle_mod.Grid(n, L, **kw)
    o.load_primitive(W, bx, by, bz)
    tg = g.advance(1000, t_end=0.1)
    to = o.advance(1000, t_end=0.1)
    assert abs(tg - 0.1) < 1e-14 and abs(to - 0.1) < 1e-14
    assert state_err(g.read(), o.read()) < 1e-9


def test_fp64_reciprocal_helpers_match_cuda(wb):
    """The sweep's reciprocal / rsqrt (PTX approximation + third-order
    correction) agree with CUDA's division and rsqrt to ~1 ulp over 600 decades."""
    g = wb.Grid((8, 8, 8))
    e_rcp, e_rsq = g.selftest_math(1 << 22)
    assert e_rcp < 4.5e-16, e_rcp
    assert e_rsq < 4.5e-16, e_rsq


def test_integer_pipe_helpers_match_fp64_definitions(wb):
    """Every bit-pattern helper that stands in for an FP64 compare, a sign
    operation or a power-of-two scaling (zero and sign tests, orders, minmod,
    the signal-rate max key, halving and exact doubling) agrees with its FP64
    definition on all pairs of 16 special values and on 4M random bit patterns
    (NaN, infinities, subnormals and signed zeros included)."""
    g = wb.Grid((8, 8, 8))
    bad = g.selftest_bits(1 << 22)
    assert len(bad) == 15
    assert not {k: v for k, v in bad.items() if v}


def test_lagged_dt_parity(wb, oracle_mod):
    from paper_1701_07452_gb300.initial_conditions import random_box
    st = random_box(12, seed=21)
    g, o = make_pair(wb, oracle_mod, st, (12, 12, 12), dt_lag=True)
    d0 = o.dt()
    g.advance(2)
    o.advance(2)
    assert abs(g.counters()["last_dt"] - d0) <= 1e-14 * d0
    g.advance(18)
    o.advance(18)
    assert state_err(g.read(), o.read()) < 1e-10


def test_device_totals_match_exact_sums(wb):
    """The device's compensated totals against exactly rounded sums (math.fsum)
    of the state read back: rho, M, E over zones, b over the owned (low) faces."""
    import math
    from paper_1701_07452_gb300.initial_conditions import random_box
    n = (20, 18, 16)
    st = random_box(n, seed=31)
    g = wb.Grid(n, length=st["length"])
    g.load_state(st)
    g.advance(3)
    U, bx, by, bz, _ = g.read()
    vol = float(np.prod([st["length"][a] / n[a] for a in range(3)]))
    exact = [math.fsum(U[c].ravel()) * vol for c in range(5)]
    exact += [math.fsum(bx[:, :, :-1].ravel()) * vol, math.fsum(by[:, :-1, :].ravel()) * vol,
              math.fsum(bz[:-1].ravel()) * vol]
    scale = [math.fsum(np.abs(U[c]).ravel()) * vol for c in range(5)]
    scale += [math.fsum(np.abs(bx).ravel()) * vol, math.fsum(np.abs(by).ravel()) * vol,
              math.fsum(np.abs(bz).ravel()) * vol]
    tot = g.totals()
    for c in range(8):
        assert abs(tot[c] - exact[c]) <= 1e-15 * scale[c], (c, tot[c], exact[c])
    assert np.array_equal(g.totals(), tot)   # fixed-order reduction: the same bits again


def test_pinned_host_buffers_round_trip(wb):
    """Page-locked host arrays are read and written in place by the kernels;
    the result equals the staged path (ordinary host memory) bit for bit."""
    torch = pytest.importorskip("torch")
    from paper_1701_07452_gb300.initial_conditions import random_box
    n = (16, 12, 10)
    st = random_box(n, seed=32)
    g = wb.Grid(n, length=st["length"])
    g.load_state(st)
    g.advance(2)
    plain = g.read()
    pinned = [torch.empty(a.shape, dtype=torch.float64, pin_memory=True) for a in plain]
    g.read(out=tuple(p.numpy() for p in pinned))
    for a, p in zip(plain, pinned):
        assert np.array_equal(a, p.numpy())
    # load from the pinned copy, step both, compare
    h = wb.Grid(n, length=st["length"])
    h.load(*(p.numpy() for p in pinned[:4]))
    k = wb.Grid(n, length=st["length"])
    k.load(*plain[:4])
    h.advance(2)
    k.advance(2)
    for a, b in zip(h.read(), k.read()):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("case", ["late_max", "near_ties", "out_of_range"])
def test_screened_cfl_rate_finds_the_exact_max(wb, oracle_mod, case):
    """The CFL reduction screens zones with an FP32 estimate and evaluates the
    FP64 rate only where a zone could hold the maximum; dt must equal the
    oracle's (the max over every zone) whatever the data: the largest zone
    last in memory, near-ties below the FP32 resolution, and values outside
    the FP32 screen's range."""
    n = (24, 20, 16)
    W = np.zeros((5, n[2], n[1], n[0]))
    W[0], W[1], W[2], W[3], W[4] = 1.0, 0.3, -0.2, 0.1, 0.6
    bx = np.full((n[2], n[1], n[0] + 1), 0.4)
    by = np.full((n[2], n[1] + 1, n[0]), -0.3)
    bz = np.full((n[2] + 1, n[1], n[0]), 0.25)
    rng = np.random.default_rng(11)
    if case == "late_max":
        W[1] += 0.01 * rng.uniform(-1, 1, W[1].shape)
        W[1][-1, -1, -1] = 0.5              # fastest zone: the last one stored
    elif case == "near_ties":
        W[1] *= 1.0 + 1e-9 * rng.uniform(-1, 1, W[1].shape)   # below FP32 resolution
    else:
        W[0][n[2] // 2, 3, 5] = 1e-25       # density far below the screen's range
        W[4][0, 0, 0] = 1e-30
    L = (1.0, 1.0, 1.0)
    g = wb.Grid(n, length=L)
    g.load(W, bx, by, bz, primitive=True)
    o = oracle_mod.Grid(n, L)
    o.load_primitive(W, bx, by, bz)
    dg, do = g.dt(), o.dt()
    assert abs(dg - do) <= 1e-14 * do, (dg, do)


@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 0, 1), (1, 1, 1)])
def test_checkpoint_resume_bit_exact(wb, bc):
    """wb_read_state / wb_load_state are the checkpoint: 10 steps equal 5
    steps, a read to host, a fresh grid loaded from it, and 5 more steps,
    bit for bit (the loaded state's dt is the one the running grid takes).
    On outflow axes the zone field of the last zone averages the boundary
    face as the ghost fill leaves it, so a load of the read faces gives the
    same zone field."""
    from paper_1701_07452_gb300.initial_conditions import turbulence_box
    n = (24, 20, 16)
    st = turbulence_box(n, seed=8)
    a = wb.Grid(n, length=st["length"], bc=bc)
    a.load_state(st)
    a.advance(10)
    b = wb.Grid(n, length=st["length"], bc=bc)
    b.load_state(st)
    b.advance(5)
    U, bx, by, bz, _ = b.read()
    c = wb.Grid(n, length=st["length"], bc=bc)
    c.load(U, bx, by, bz)
    c.advance(5)
    for x, y in zip(a.read(), c.read()):
        assert np.array_equal(x, y)


def test_reused_workspace_arrays(wb):
    """The default workspace reuses the predictor arrays for the corrector
    stages (54 arrays a zone instead of 81); the step is the same bit for bit,
    and the overwritten predictor fluxes are not offered for dumping."""
    from paper_1701_07452_gb300.initial_conditions import turbulence_box
    n = (20, 18, 16)
    st = turbulence_box(n, seed=13)
    keep = wb.Grid(n, length=st["length"], keep_stages=True)
    lean = wb.Grid(n, length=st["length"])
    assert lean.nbytes < keep.nbytes
    for g in (keep, lean):
        g.load_state(st)
        g.advance(3)
    for a, b in zip(keep.read(), lean.read()):
        assert np.array_equal(a, b)
    with pytest.raises(wb.WombatError):
        lean.stage(0)
    assert np.array_equal(keep.stage(4), lean.stage(4))


def test_ghost_poison_beyond_dependency_radius(wb):
    """Halo indexing: on a box periodic on every axis (interior-only stages with
    periodic images between them) a step reads the loaded ghost zones only to
    depth 2.  NaN written into the state's ghost zones at depth 3 to 5 after
    the load (every zone field and face field; the storage is padded by 5
    zones per side, [field][z][y][x], state first in the workspace) must leave
    the step's result bit-identical and every counter clean."""
    import torch
    from paper_1701_07452_gb300.initial_conditions import turbulence_box
    n = (20, 18, 16)
    st = turbulence_box(n, seed=21)
    clean = wb.Grid(n, length=st["length"])
    clean.load_state(st)
    clean.advance(1)
    g = wb.Grid(n, length=st["length"])
    g.load_state(st)
    torch.cuda.synchronize()
    NG = 5
    pd = [x + 2 * NG for x in n]
    V = pd[0] * pd[1] * pd[2]
    mem = g.workspace.view(torch.float64)
    idx = [torch.arange(p, device=mem.device) - NG for p in pd]
    k, j, i = torch.meshgrid(idx[2], idx[1], idx[0], indexing="ij")

    def depth(x, m):
        return torch.clamp(torch.maximum(-x, x - (m - 1)), min=0)

    d = torch.maximum(torch.maximum(depth(i, n[0]), depth(j, n[1])), depth(k, n[2]))
    mask = (d >= 3).reshape(-1)
    assert int(mask.sum()) > 0
    for field in range(11):
        view = mem[field * V:(field + 1) * V]
        view[mask] = float("nan")
    g.advance(1)
    for a, b in zip(clean.read(), g.read()):
        assert np.array_equal(a, b)
    c = g.counters()
    assert c["unphysical"] == 0 and c["floor_hits"] == 0
    assert np.isfinite(g.totals()).all()
