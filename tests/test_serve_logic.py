"""Host-side logic of the serving loop (admission by HBM budget with backfill,
completion detection, latency bookkeeping) against a fake pool on the CPU."""
import numpy as np

from paper_1701_07452_gb300 import serve


class FakePool:
    """Stands in for binding.Pool: a byte budget, slots and step counters."""

    def __init__(self, budget):
        self.budget = budget
        self.used = {}
        self.left = {}
        self.loaded = set()
        self.max_resident = 0
        self.advances = 0
        self.bad = set()       # slots whose run fails on the device
        self.released = []

    @staticmethod
    def size(n):
        return int(np.prod(n))

    def admit(self, n, length=None):
        need = self.size(n)
        if sum(self.used.values()) + need > self.budget:
            return None
        slot = 0
        while slot in self.used:
            slot += 1
        self.used[slot] = need
        self.left[slot] = 0
        self.max_resident = max(self.max_resident, len(self.used))
        return slot

    def load(self, slot, W, *a, **k):
        self.loaded.add(slot)
        if isinstance(W, str) and W == "unphysical":
            self.bad.add(slot)

    def set_steps(self, slot, n):
        self.left[slot] = n

    def advance(self, k, use_graph=True):
        self.advances += 1
        for s in self.left:
            # a failed box stops: its dt fails and its steps left drop to 0
            self.left[s] = 0 if s in self.bad else max(0, self.left[s] - k)

    def steps_left(self):
        out = [0] * 64
        for s, v in self.left.items():
            out[s] = v
        return out

    def read(self, slot):
        return ("result", slot)

    def counters(self, slot):
        return {"unphysical": 1 if slot in self.bad else 0, "steps": 0}

    def release(self, slot):
        del self.used[slot]
        del self.left[slot]
        self.bad.discard(slot)
        self.released.append(slot)


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 0.001
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 0.0)


def make_server(budget, tick, policy="fair", tick_cells=1e12):
    srv = serve.Server.__new__(serve.Server)
    srv.pool = FakePool(budget)
    srv.tick_steps = tick
    srv.use_graph = True
    srv.keep_results = True
    srv.policy = policy
    srv.tick_cells = tick_cells
    srv.ticks = 0
    return srv


def test_every_request_completes_within_budget_with_backfill():
    empty = {"W": None, "bx": None, "by": None, "bz": None}
    reqs = [serve.Request(i, 0.01 * i, (8, 8, 8) if i % 3 else (16, 16, 16), 5 + i, empty) for i in range(12)]
    srv = make_server(budget=16 ** 3 + 8 ** 3, tick=2)
    clk = FakeClock()
    recs = srv.run(reqs, clock=clk, sleep=clk.sleep)
    assert len(recs) == 12
    for r in recs:
        assert r.arrival <= r.admitted <= r.finished
        assert r.result is not None
    # never more state resident than the budget allows
    assert srv.pool.max_resident <= 2
    summ = serve.summarize(recs)
    assert summ["requests"] == 12 and summ["p99_s"] >= summ["p50_s"] > 0


def test_small_run_backfills_behind_a_big_one():
    empty = {"W": None, "bx": None, "by": None, "bz": None}
    reqs = [serve.Request(0, 0.0, (16, 16, 16), 10, empty),
            serve.Request(1, 0.0001, (16, 16, 16), 2, empty),
            serve.Request(2, 0.0002, (8, 8, 8), 2, empty)]
    srv = make_server(budget=16 ** 3 + 8 ** 3, tick=2)
    clk = FakeClock()
    recs = srv.run(reqs, clock=clk, sleep=clk.sleep)
    assert recs[2].admitted < recs[1].admitted      # later, smaller run admitted first
    assert recs[1].admitted >= recs[0].finished     # the big one waited for memory


def test_ticks_cover_the_longest_run():
    empty = {"W": None, "bx": None, "by": None, "bz": None}
    reqs = [serve.Request(0, 0.0, (8, 8, 8), 7, empty), serve.Request(1, 0.0, (8, 8, 8), 3, empty)]
    srv = make_server(budget=10 ** 6, tick=2)
    clk = FakeClock()
    recs = srv.run(reqs, clock=clk, sleep=clk.sleep)
    assert srv.ticks == 4            # ceil(7 / 2)
    assert recs[1].finished < recs[0].finished


def test_a_failed_run_is_isolated():
    """A run whose state becomes unphysical is recorded as failed and released;
    every other run completes and the loop does not stop."""
    empty = {"W": None, "bx": None, "by": None, "bz": None}
    bad = {"W": "unphysical", "bx": None, "by": None, "bz": None}
    reqs = [serve.Request(i, 0.001 * i, (8, 8, 8), 6, bad if i == 2 else empty) for i in range(5)]
    srv = make_server(budget=10 ** 6, tick=2)
    clk = FakeClock()
    recs = srv.run(reqs, clock=clk, sleep=clk.sleep)
    assert [r.status for r in recs] == ["done", "done", "failed", "done", "done"]
    assert recs[2].result is None and "unphysical" in recs[2].error
    assert all(r.result is not None for r in recs if r.status == "done")
    assert not srv.pool.used                       # every slot given back
    summ = serve.summarize(recs)
    assert summ["completed"] == 4 and summ["failed"] == 1


def test_cancellation_of_queued_and_resident_runs():
    """A resident run cancelled mid-run gives its slot back at the next tick
    and the run that waited for memory is admitted; a run cancelled before it
    arrives never enters."""
    empty = {"W": None, "bx": None, "by": None, "bz": None}
    reqs = [serve.Request(0, 0.0, (16, 16, 16), 100, empty),     # fills the budget
            serve.Request(1, 0.0005, (16, 16, 16), 4, empty),    # waits for memory
            serve.Request(2, 0.5, (8, 8, 8), 4, empty)]          # cancelled before arrival
    srv = make_server(budget=16 ** 3, tick=2)
    clk = FakeClock()
    recs = srv.run(reqs, clock=clk, sleep=clk.sleep, cancellations=[(0.01, 0), (0.02, 2)])
    assert recs[0].status == "cancelled" and recs[0].result is None
    assert recs[1].status == "done" and recs[1].admitted >= recs[0].finished
    assert recs[2].status == "cancelled" and recs[2].admitted != recs[2].admitted   # never admitted
    assert srv.ticks < 50                          # the long run did not run to its end


def test_srpt_ticks_finish_short_runs_first():
    """Under the srpt policy a tick grants steps to the runs with the least
    remaining work until its cell budget is spent: a short run that arrives
    behind long ones finishes before them, every run still gets all its
    steps, and the ticks never grant more than the budget (beyond the first
    run)."""
    empty = {"W": None, "bx": None, "by": None, "bz": None}
    reqs = [serve.Request(0, 0.0, (16, 16, 16), 40, empty),
            serve.Request(1, 0.0, (16, 16, 16), 40, empty),
            serve.Request(2, 0.0001, (8, 8, 8), 4, empty)]
    granted = []

    class CountingPool(FakePool):
        def set_steps(self, slot, n):
            super().set_steps(slot, n)
            granted.append((slot, n))

    srv = make_server(budget=10 ** 6, tick=2, policy="srpt", tick_cells=2 * 16 ** 3 * 2)
    srv.pool = CountingPool(10 ** 6)
    clk = FakeClock()
    recs = srv.run(reqs, clock=clk, sleep=clk.sleep)
    assert all(r.status == "done" for r in recs)
    assert recs[2].finished < recs[0].finished and recs[2].finished < recs[1].finished
    fair = make_server(budget=10 ** 6, tick=2)
    frecs = fair.run(reqs, clock=FakeClock(), sleep=FakeClock().sleep)
    assert all(r.status == "done" for r in frecs)


def test_srpt_grants_respect_the_cell_budget():
    from types import SimpleNamespace
    srv = make_server(budget=10 ** 6, tick=3, policy="srpt", tick_cells=10 * 8 ** 3)
    resident = {0: SimpleNamespace(n=(8, 8, 8), steps=10, rid=0), 1: SimpleNamespace(n=(8, 8, 8), steps=5, rid=1),
                2: SimpleNamespace(n=(16, 16, 16), steps=2, rid=2)}
    done = {0: 0, 1: 0, 2: 0}
    g = srv._grants(resident, done)
    # least remaining work first: run 1 (5 x 8^3), then run 0 (10 x 8^3), then 2 (2 x 16^3)
    assert g[1] == 3 and g[0] == 3 and g[2] == 0
    done = {0: 9, 1: 5, 2: 0}
    g = srv._grants(resident, done)
    assert g[0] == 1 and g[1] == 0
