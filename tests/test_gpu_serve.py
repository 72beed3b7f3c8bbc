"""Serving pattern on the GPU: runs that arrive while others are resident are
admitted as memory frees up, share launches, and each result is bit-identical
to the same run served alone, under either tick policy and either batch
form, and within tolerance of the FP64 oracle run of the same request."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_07452_gb300 import binding, serve
    binding.lib()
    return binding, serve


def requests():
    from paper_1701_07452_gb300 import serve
    from paper_1701_07452_gb300.initial_conditions import random_box, turbulence_box
    spec = [((12, 12, 12), 7, 0.00), ((16, 12, 10), 5, 0.00), ((10, 10, 10), 9, 0.02),
            ((14, 14, 14), 4, 0.04), ((8, 16, 12), 6, 0.05)]
    out = []
    for i, (n, steps, t) in enumerate(spec):
        st = turbulence_box(n, seed=50 + i) if i % 2 else random_box(n, seed=60 + i)
        out.append(serve.Request(i, t, n, steps, st, st["length"]))
    return out


@pytest.mark.parametrize("policy", ["fair", "srpt"])
def test_served_results_equal_alone_results(mods, policy):
    binding, serve = mods
    reqs = requests()
    # the state budget holds about two of these boxes at a time
    per = max(11 * 8 * (n[0] + 10) * (n[1] + 10) * (n[2] + 10) for n in [r.n for r in reqs])
    srv = serve.Server(state_bytes=2 * per + 4096, work_bytes=64 << 20, max_boxes=8, max_n=32,
                       tick_steps=2, keep_results=True, policy=policy, tick_cells=2 * 14 ** 3)
    recs = srv.run(reqs)
    assert len(recs) == len(reqs)
    assert any(r.admitted > r.arrival + 1e-6 for r in recs), "budget never delayed an admission"
    for r, rec in zip(reqs, recs):
        # alone in the other batch form for the fair policy: forms give the same bits
        alone = serve.Server(state_bytes=per + 4096, work_bytes=64 << 20, max_boxes=2, max_n=32,
                             tick_steps=3, keep_results=True,
                             form="persistent" if policy == "fair" else "staged")
        (arec,) = alone.run([serve.Request(r.rid, 0.0, r.n, r.steps, r.state, r.length)])
        for a, b in zip(arec.result, rec.result):
            assert np.array_equal(a, b), r.rid


def test_pool_admission_accounting(mods):
    binding, _ = mods
    per = 11 * 8 * 20 ** 3
    pool = binding.Pool(state_bytes=3 * per, work_bytes=32 << 20, max_boxes=4, max_n=16)
    a = pool.admit((10, 10, 10))
    b = pool.admit((10, 10, 10))
    c = pool.admit((10, 10, 10))
    assert None not in (a, b, c)
    assert pool.admit((10, 10, 10)) is None          # state region full
    pool.release(b)
    assert pool.free_bytes()[0] >= per
    d = pool.admit((10, 10, 10))
    assert d is not None
    with pytest.raises(binding.WombatError):
        pool.admit((40, 40, 40))                      # beyond max_n


def test_an_unphysical_run_fails_alone(mods):
    """Fault injection on the host: one request's loaded state carries a NaN
    density.  Its own time step fails on the device, it is released and
    recorded as failed, and the runs sharing its launches still equal their
    results served alone."""
    binding, serve = mods
    reqs = requests()
    bad = reqs[1]
    W = bad.state["W"].copy()
    W[0, 2, 3, 4] = float("nan")
    reqs[1] = serve.Request(bad.rid, bad.arrival, bad.n, bad.steps, dict(bad.state, W=W), bad.length)
    srv = serve.Server(state_bytes=1 << 26, work_bytes=64 << 20, max_boxes=8, max_n=32, tick_steps=2,
                       keep_results=True)
    recs = srv.run(reqs)
    assert recs[1].status == "failed" and recs[1].result is None
    for r, rec in zip(reqs, recs):
        if r.rid == 1:
            continue
        assert rec.status == "done"
        alone = serve.Server(state_bytes=1 << 25, work_bytes=64 << 20, max_boxes=2, max_n=32,
                             tick_steps=3, keep_results=True)
        (arec,) = alone.run([serve.Request(r.rid, 0.0, r.n, r.steps, r.state, r.length)])
        for a, b in zip(arec.result, rec.result):
            assert np.array_equal(a, b), r.rid


def test_served_results_match_the_oracle(mods, oracle_mod):
    """Each served run (admitted under the budget, sharing launches with the
    others) against the FP64 oracle advanced by the same number of steps on
    the same seeded input: within 1e-10 (4 to 9 steps)."""
    from parity import state_err
    binding, serve = mods
    reqs = requests()
    per = max(11 * 8 * (n[0] + 10) * (n[1] + 10) * (n[2] + 10) for n in [r.n for r in reqs])
    srv = serve.Server(state_bytes=2 * per + 4096, work_bytes=64 << 20, max_boxes=8, max_n=32,
                       tick_steps=2, keep_results=True, policy="srpt", tick_cells=2 * 14 ** 3)
    recs = srv.run(reqs)
    for r, rec in zip(reqs, recs):
        assert rec.status == "done"
        o = oracle_mod.Grid(r.n, r.length)
        o.load_state(r.state)
        o.advance(r.steps)
        assert state_err(rec.result, o.read()) < 1e-10, r.rid
