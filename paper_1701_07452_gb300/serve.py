"""Continuous-batching request loop over the GPU pool (wb_pool_* C ABI).

Independent MHD runs (grid size, step count, initial data) arrive over time.
Each loop iteration admits the queued runs whose state fits the HBM budget of
the pool (first come first served, later runs may backfill when an earlier
one does not fit), loads their initial data, advances every resident run by
up to ``tick_steps`` steps in one shared persistent launch, and reads back and
releases the runs that finished.  Completion latency is measured from a run's
arrival to the end of the tick in which its last step ran.

Failures stay with their run: a run whose state becomes unphysical stops on
the device (its own time step fails, the other boxes of the launch go on), is
released and recorded as failed, and the loop keeps serving the others.  A
run can be cancelled at a given time: dropped from the queue if it has not
been admitted, released at the next tick boundary if it is resident.

Each tick runs in the pool's staged form by default (one launch per stage;
form="persistent" selects the one cooperative launch); results do not depend
on the form.  seg_len sets the pool's sweep segment length (0 keeps the
library's 32; longer segments measured no faster on the request stream of
the bench, 136 about 5 % slower).

Two tick policies.  "fair": every resident run advances up to tick_steps per
tick (processor sharing).  "srpt": each tick grants up to tick_steps steps to
the resident runs in order of least remaining work (zones x steps left)
until the granted cell-updates reach tick_cells, the rest wait.  The zones a
step carries, tick_cells / tick_steps, set the latency of short runs: a run
advances one step per step of the tick, so with many steps per tick and few
zones per step (25 and 4e6 on the bench's stream) short runs finish soon
after admission, while the pool launches only the granted runs' work (runs
without steps are left out of its workspace groups) and the GPU stays
nearly as busy.  A run's result does not depend on the policy (each box
advances on its own).
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

from . import binding


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the stream
    n: tuple                # zones per axis
    steps: int
    state: dict             # primitive W and faces (initial_conditions format)
    length: tuple = (1.0, 1.0, 1.0)


@dataclasses.dataclass
class Record:
    rid: int
    n: tuple
    steps: int
    arrival: float
    admitted: float = float("nan")
    finished: float = float("nan")
    result: tuple = None
    status: str = "pending"   # done, failed or cancelled once the loop is through
    error: str = ""


class Server:
    def __init__(self, state_bytes, work_bytes, max_boxes=512, max_n=256, tick_steps=4,
                 use_graph=True, keep_results=False, policy="fair", tick_cells=1.5e8,
                 form="staged", seg_len=0, **physics):
        self.pool = binding.Pool(state_bytes, work_bytes, max_boxes=max_boxes, max_n=max_n, **physics)
        self.pool.set_form(form)
        if seg_len:
            self.pool.config(seg_len=seg_len)
        self.tick_steps = int(tick_steps)
        self.use_graph = use_graph
        self.keep_results = keep_results
        self.policy = policy
        self.tick_cells = float(tick_cells)
        self.ticks = 0

    def _grants(self, resident, done):
        """Steps each resident run may take this tick (srpt policy)."""
        work = {s: int(np.prod(r.n)) for s, r in resident.items()}
        order = sorted(resident, key=lambda s: (work[s] * (resident[s].steps - done[s]), resident[s].rid))
        grant, acc = {}, 0.0
        for s in order:
            a = min(self.tick_steps, resident[s].steps - done[s])
            if grant and acc + a * work[s] > self.tick_cells:
                a = 0
            grant[s] = a
            acc += a * work[s]
        return grant

    def run(self, requests, clock=time.perf_counter, sleep=time.sleep, cancellations=()):
        """Serve requests until every one is done, failed or cancelled.
        cancellations: (time, rid) pairs, times after the start of the stream."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        cancels = sorted(cancellations)
        queue = []
        resident = {}   # slot -> request
        done = {}       # slot -> steps taken (srpt policy)
        records = {}
        t0 = clock()
        while pending or queue or resident:
            now = clock() - t0
            while pending and pending[0].arrival <= now:
                r = pending.popleft()
                queue.append(r)
                records[r.rid] = Record(r.rid, tuple(r.n), r.steps, r.arrival)
            # cancellations that are due: queued runs leave the queue, resident
            # runs give their slot back between launches
            while cancels and cancels[0][0] <= now:
                _, rid = cancels.pop(0)
                rec = records.get(rid)
                if rec is None:   # not arrived yet: drop it from the stream
                    for r in list(pending):
                        if r.rid == rid:
                            pending.remove(r)
                            records[rid] = rec = Record(r.rid, tuple(r.n), r.steps, r.arrival)
                    if rec is None:
                        continue
                if rec.status != "pending":
                    continue
                queue = [r for r in queue if r.rid != rid]
                for slot, r in list(resident.items()):
                    if r.rid == rid:
                        self.pool.release(slot)
                        del resident[slot]
                        done.pop(slot, None)
                rec.status = "cancelled"
                rec.finished = now
            # admission by HBM budget, FIFO with backfill
            still = []
            for r in queue:
                slot = self.pool.admit(r.n, r.length)
                if slot is None:
                    still.append(r)
                    continue
                st = r.state
                self.pool.load(slot, st["W"], st["bx"], st["by"], st["bz"], primitive=True)
                self.pool.set_steps(slot, r.steps if self.policy == "fair" else 0)
                records[r.rid].admitted = clock() - t0
                resident[slot] = r
                done[slot] = 0
            queue = still
            if not resident:
                if pending:
                    sleep(max(0.0, min(0.05, pending[0].arrival - (clock() - t0))))
                continue
            if self.policy == "srpt":
                grant = self._grants(resident, done)
                for slot, a in grant.items():
                    self.pool.set_steps(slot, a)
            self.pool.advance(self.tick_steps, use_graph=self.use_graph)
            self.ticks += 1
            left = self.pool.steps_left()
            done_at = clock() - t0
            if self.policy == "srpt":
                finished = []
                for slot in resident:
                    done[slot] += grant[slot] - left[slot]
                    if done[slot] >= resident[slot].steps or \
                            (grant[slot] > 0 and self.pool.counters(slot)["unphysical"]):
                        finished.append(slot)
            else:
                finished = [s for s in resident if left[s] == 0]
            for slot in finished:
                r = resident.pop(slot)
                done.pop(slot, None)
                rec = records[r.rid]
                rec.finished = done_at
                c = self.pool.counters(slot)
                if c["unphysical"]:
                    rec.status = "failed"
                    rec.error = f"unphysical state after {c.get('steps', '?')} steps"
                else:
                    rec.status = "done"
                    if self.keep_results:
                        rec.result = self.pool.read(slot)
                self.pool.release(slot)
        return [records[k] for k in sorted(records)]


def summarize(records):
    """Latency and throughput over the runs that completed; failed and
    cancelled runs are counted apart."""
    done = [r for r in records if r.status == "done"]
    lat = np.array([r.finished - r.arrival for r in done])
    wall = max(r.finished for r in done) - min(r.arrival for r in done)
    cells = float(sum(np.prod(r.n) * r.steps for r in done))
    return {
        "requests": len(records),
        "completed": len(done),
        "failed": sum(r.status == "failed" for r in records),
        "cancelled": sum(r.status == "cancelled" for r in records),
        "p50_s": float(np.percentile(lat, 50)),
        "p99_s": float(np.percentile(lat, 99)),
        "mean_s": float(lat.mean()),
        "wall_s": float(wall),
        "cell_updates": cells,
        "cell_updates_per_s": cells / wall,
        "solves_per_s": len(done) / wall,
    }
