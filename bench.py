#!/usr/bin/env python3
"""Benchmark of the GB300-native WOMBAT per-patch ideal-MHD step.

Workload (one GPU): the 256^3 periodic FP64 turbulence box (rho = 1, P = 1,
solenoidal velocity modes 1 <= |k| <= 8 with amplitude ~ |k|^-2 at rms Mach 1,
mean field along x at beta 100, 10 % field perturbation from a random vector
potential), advanced with the CTU+CT MHDTVD step.  One bench "step" is one
full step of that box: halo fill, CFL dt, six MHDTVD sweeps, EMFs, constrained
transport and the conservative update.

value      FP64 cell-updates/s with the state resident in HBM (CUDA events,
           max over ranks); the state (1.6 GB) is larger than L2, so no flush.
e2e        the same metric through the C ABI with host buffers: every step
           loads the state from pinned host memory, advances one step and
           reads the state back (copies inside the timed region).
roofline   the MHDTVD sweep kernel against the FP64 pipe (the step is FP64
           bound): algorithmic flops per face (the oracle's instrumented
           count, oracle/count_flops.py) x faces per launch / measured launch
           time; peak = SMs x 4 FP64 flops per clock x the SM clock sampled
           under load.  The kernel's own executed flops (ncu FP64 counters)
           are reported beside it as "executed".
cpu_baseline  the plain FP64 oracle timed on the host cores on a bounded
           sample of the same workload (all cores, and one core).
batch      the ensemble workload: a seeded subset of the 1000 boxes of edges
           {16..128}, 100 steps each, advanced in shared launches, against the
           same boxes one at a time through the single-box path.
serve      the serving workload: Poisson arrivals (50/s) of turbulence runs of
           edge log-uniform 32..192 and U{50..500} steps under a 150 GB state
           budget; p50/p99 time to completion.

--impl reference times the oracle (the slow CPU reading of the paper) as the
reference arm.  --gpus N > 1 runs N independent replicas of the box, one per
rank (the path has no data exchange between GPUs).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "FP64 cell-updates/s"
UNIT = "cell-updates/s"
N_BOX = 256
SEED = 2
# Algorithmic FP64 operations of the method: the oracle's instrumented count
# (oracle/count_flops.py 64 2 2: the turbulence data at 64^3, steps 2-3;
# add/sub/mul/div/sqrt = 1, identity operations of its dense 7x7 matrices not
# counted), per sweep face (zone state and flux, Roe state and eigen-system,
# alpha_k, g-tilde, limiter, emitted flux) and per cell-update (six sweep
# faces plus every other stage of the step); profiles/oracle_flop_count.md.
ALG_FLOPS_PER_FACE = 879.0
ALG_FLOPS_PER_CELL_UPDATE = 5871.0
# FP64 flops (DFMA = 2, DMUL = DADD = 1) the kernels execute, from the ncu
# FP64 instruction counters of one step of the 96^3 box: per interface system
# of k_sweep (the mean of the six sweeps), and per zone of the other stage
# kernels of the step together (profiles/k_sweep_96cube_ncu_full.md,
# profiles/stages_96cube_fp64_counts.md).  Counted per face of the box the
# figure leaves out the ~2 % of overlap systems a 256^3 launch adds.
EXEC_FLOPS_PER_FACE = 450.8
EXEC_STAGE_FLOPS_PER_ZONE = 431.8
# DRAM bytes (read + write) of one k_sweep launch at the 256^3 workload, the
# mean of the six sweeps of a step from one ncu capture
# (profiles/k_sweep_256cube_dram.md), valid only for the kernel sources it was
# taken on (their SHA-256 over csrc/wb_sweep.cu, wb_units.cuh, wb_device.cuh);
# the algorithmic figure is 128 B per face.
SWEEP_DRAM_CAPTURE = {"n": 256, "bytes": 3.6763e9,
                      "src_sha256": "68f8615198707e20999cb9332cdfca1bc16d4505845845c06e39a34523ecfa46"}
SWEEP_BYTES_PER_FACE = 128.0
# algorithmic state bytes per cell-update: 5 conserved fields and 3 face fields
# read and written once (the step's HBM roofline)
STEP_BYTES_PER_CELL = 128.0
# FP64 issue rate of one GB300 SM: 2 DFMA per clock (measured with the DFMA
# probe: 1196 GFLOP/s at 1995 MHz on 152 SMs), i.e. 4 flops per clock per SM.
FP64_FLOPS_PER_CLK_PER_SM = 4.0


def sweep_src_sha256():
    """SHA-256 over the sweep kernel's sources (the DRAM capture's stamp)."""
    h = hashlib.sha256()
    for name in ("wb_sweep.cu", "wb_units.cuh", "wb_device.cuh"):
        with open(os.path.join(ROOT, "paper_1701_07452_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def sweep_traffic(n):
    """Measured DRAM bytes per sweep launch, or None when no capture of the
    current kernel at this size exists."""
    cap = SWEEP_DRAM_CAPTURE
    if cap["n"] == n and cap["src_sha256"] == sweep_src_sha256():
        return cap["bytes"]
    return None


def cpu_model():
    """Host CPU model name (lscpu), for the CPU baseline's record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                name = line.split(":", 1)[1].strip()
                if name and not name.isdigit():
                    return name
    except Exception:
        pass
    return None


def step_launches(desc):
    """Kernels one wb_advance step launches: the dt kernel, 14 per pass over a
    batch of patches (6 sweeps, reference EMF, corner EMFs, half CT,
    transverse states, half-step reference EMF, corner EMFs, final CT, update)
    and the ghost fill; a grid periodic on every axis with all patches in one
    pass adds the 7 periodic-image fills of its interior-only stages."""
    npatch = desc.patches[0] * desc.patches[1] * desc.patches[2]
    per_pass = desc.batch_patches if desc.batch_patches > 0 else npatch
    passes = -(-npatch // per_pass)
    flat = desc.n[2] == 1 and desc.patches[2] == 1 and desc.bc[2] == 0
    images = passes == 1 and not flat and all(desc.bc[a] == 0 for a in range(3))
    return 2 + (21 if images else 14) * passes


def workload_name(n):
    return f"{n}^3 periodic FP64 MHD turbulence box, CTU+CT MHDTVD step"


def l2_note(n):
    """How the timed region stands to the 129 MB L2: the resident state (11
    padded FP64 fields) of an n^3 box, no flush between steps."""
    state = 11 * 8 * (n + 10) ** 3
    side = ">" if state > 129e6 else "<"
    return f"state {state / 1e9:.2f} GB {side} L2 (129 MB), no flush"


def step_roofline(value, fp64_peak_tflops):
    """The whole step against the slower of its two ceilings: FP64 flops per
    cell-update at the FP64 peak, and its state bytes at the measured HBM
    copy bandwidth.  The FP64 ceiling is taken with the algorithmic count
    (the oracle's operations) and, as "executed", with the kernels' own."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            hbm = float(json.load(f)["hbm_gbs"])
        src = "MEASURED_PEAKS.json (measured copy)"
    except (OSError, KeyError, ValueError):
        hbm, src = 6800.0, "fallback 6.8 TB/s"
    hbm_rate = hbm * 1e9 / STEP_BYTES_PER_CELL

    def ceiling(flops):
        fp64_rate = fp64_peak_tflops * 1e12 / flops
        bound = min(fp64_rate, hbm_rate)
        return {"bound": "fp64" if fp64_rate <= hbm_rate else "hbm", "fp64_rate": fp64_rate,
                "frac": value / bound, "flops_per_cell_update": flops}

    exec_flops = 6 * EXEC_FLOPS_PER_FACE + EXEC_STAGE_FLOPS_PER_ZONE
    out = ceiling(ALG_FLOPS_PER_CELL_UPDATE)
    out.update({"flops_kind": "algorithmic (oracle count)", "unit": UNIT, "hbm_rate": hbm_rate,
                "bytes_per_cell_update": STEP_BYTES_PER_CELL, "hbm_gbs": hbm, "hbm_source": src,
                "hbm_frac": value * STEP_BYTES_PER_CELL / (hbm * 1e9),
                "executed": ceiling(exec_flops)})
    return out


def sweep_faces_per_step(n):
    """Interfaces the six sweeps of one step must compute (one per zone and
    direction, predictor and corrector) -- the algorithmic count; the kernel
    also computes the patch-halo faces, which are not counted."""
    return 6 * n ** 3


class ClockSampler:
    """nvidia-smi SM clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.samples.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        sm = [float(s[0]) for s in self.samples if s and s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if len(s) > 1 and s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for name, v in zip(names, s[3:7]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.samples)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl != "reference" else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_sample(n_sample, steps, threads=0, st=None):
    """Oracle (plain FP64 CPU restatement) on an n_sample^3 box of the same
    turbulence data (st: that box's state, if already made): returns
    (cell-updates/s, wall seconds of the steps, threads used)."""
    import oracle
    from paper_1701_07452_gb300.initial_conditions import turbulence_box
    used = oracle.set_threads(threads if threads > 0 else (os.cpu_count() or 1))
    if st is None:
        st = turbulence_box(n_sample, SEED)
    g = oracle.Grid((n_sample,) * 3, st["length"])
    g.load_state(st)
    t0 = time.perf_counter()
    g.advance(steps)
    wall = time.perf_counter() - t0
    return n_sample ** 3 * steps / wall, wall, used


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    # each bench step: one oracle step of a 128^3 box (--ref-sample) of the
    # same turbulence data (about a second on 16 cores), so a default run ends
    # in under a minute
    from paper_1701_07452_gb300.initial_conditions import turbulence_box
    n_sample, steps_per = args.ref_sample, 1
    st = turbulence_box(n_sample, SEED)
    for _ in range(args.warmup):
        cpu_sample(n_sample, steps_per, st=st)
    t_total = 0.0
    used = 1
    for _ in range(args.steps):
        v, wall, used = cpu_sample(n_sample, steps_per, st=st)
        t_total += wall
    value = n_sample ** 3 * steps_per * args.steps / t_total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(N_BOX), "patches": "1 (single grid)",
                   "sample": f"{n_sample}^3 box of the same turbulence data, {steps_per} step per bench step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
                         "sample": f"{n_sample}^3 x {steps_per} step per bench step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def ensemble_boxes(nbox):
    """The first nbox boxes of the seeded 1000-box ensemble: edges drawn from
    {16, 24, 32, 48, 64, 96, 128} (seed 4), random data of seed 4000 + b."""
    import numpy as np
    from paper_1701_07452_gb300.initial_conditions import random_box
    rng = np.random.default_rng(4)
    edges = rng.choice([16, 24, 32, 48, 64, 96, 128], size=1000)[:nbox]
    states = [random_box(int(e), seed=4000 + b) for b, e in enumerate(edges)]
    boxes = [{"n": (int(e),) * 3, "length": st["length"]} for e, st in zip(edges, states)]
    return edges, boxes, states


def batch_figures(nbox, steps, form="auto", other_form=True, oracle_boxes=0):
    """Batched vs one-box-at-a-time solves/s on the ensemble subset (CUDA
    events; a solve is one box advanced `steps` steps).  oracle_boxes > 0
    also checks that many of the smallest boxes against the FP64 oracle."""
    import torch

    from paper_1701_07452_gb300 import binding as wb
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from parity import state_err
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    edges, boxes, states = ensemble_boxes(nbox)
    if form == "auto":
        tune = wb.Batch(boxes)
        for i, st in enumerate(states):
            tune.load_state(i, st)
        tune.set_steps(-1, 1000)
        tune.autotune(trial_steps=1)
        cfg = tune.get_config()
        del tune
    bt = wb.Batch(boxes)
    if form != "auto":
        bt.set_form(form)
    else:
        bt.config(seg_len=cfg["seg_len"], blocks_per_sm=cfg["blocks_per_sm"])
        bt.set_form(cfg["form"])
    cfg = bt.get_config()
    for i, st in enumerate(states):
        bt.load_state(i, st)
    bt.set_steps(-1, 1)
    bt.advance(1, use_graph=True)       # graph capture + warm-up step
    for i, st in enumerate(states):
        bt.load_state(i, st)
    bt.set_steps(-1, steps)
    torch.cuda.synchronize()
    e0, e1 = ev(), ev()
    e0.record(stream)
    bt.advance(steps, use_graph=True)
    e1.record(stream)
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) * 1e-3
    assert all(bt.counters(i)["steps"] == steps for i in range(nbox))
    out = {}
    if oracle_boxes:
        import oracle
        oracle.set_threads(os.cpu_count() or 1)
        order = sorted(range(nbox), key=lambda i: int(edges[i]))[:oracle_boxes]
        worst = 0.0
        for i in order:
            o = oracle.Grid(boxes[i]["n"], boxes[i]["length"])
            o.load_state(states[i])
            o.advance(steps)
            worst = max(worst, state_err(bt.read(i), o.read()))
        out["oracle_check"] = {"boxes": [int(edges[i]) for i in order], "steps": steps,
                               "max_rel_err": worst, "tolerance": 1e-8}
    if other_form:
        other = "staged" if cfg["form"] == "persistent" else "persistent"
        bt.set_form(other)
        for i, st in enumerate(states):
            bt.load_state(i, st)
        bt.set_steps(-1, 1)
        bt.advance(1, use_graph=True)
        for i, st in enumerate(states):
            bt.load_state(i, st)
        bt.set_steps(-1, steps)
        torch.cuda.synchronize()
        e0.record(stream)
        bt.advance(steps, use_graph=True)
        e1.record(stream)
        torch.cuda.synchronize()
        out["other_form"] = {"form": other, "solves_per_s": nbox / (e0.elapsed_time(e1) * 1e-3)}
        bt.set_form(cfg["form"])
        # per-stage breakdown of the chosen form (stage timer, no graph), one
        # more step of every box, outside the timed region
        bt.set_steps(-1, 1)
        bt.stage_timer(True)
        bt.advance(1, use_graph=False)
        out["stage_ms_one_step"] = {k: round(v, 3) for k, v in bt.stage_times().items()}
        bt.stage_timer(False)
    del bt
    # the plain path: one box at a time through the single-box API, each
    # after one untimed warm-up step
    t_plain = 0.0
    for b, st in zip(boxes, states):
        g = wb.Grid(b["n"], length=b["length"])
        g.load_state(st)
        g.advance(1)
        g.load_state(st)
        torch.cuda.synchronize()
        e0.record(stream)
        g.advance(steps, sync=False)
        e1.record(stream)
        torch.cuda.synchronize()
        t_plain += e0.elapsed_time(e1) * 1e-3
        del g
    torch.cuda.empty_cache()
    cells = float(sum(int(e) ** 3 for e in edges)) * steps
    res = {"solves_per_s": nbox / t_batch, "plain_solves_per_s": nbox / t_plain,
           "speedup": t_plain / t_batch, "batched_cell_updates_per_s": cells / t_batch,
           "plain_cell_updates_per_s": cells / t_plain, "steps": steps, "boxes": nbox,
           "form": cfg, "workload": f"the first {nbox} of the 1000 ensemble boxes (edges from "
                                    f"{{16..128}}, seed 4; random data seed 4000+b), {steps} steps "
                                    "each; a solve = one box x all its steps"}
    res.update(out)
    return res


def serve_figures(requests, steps_scale=1.0, policies=("srpt",)):
    """Serving run of the request stream: p50/p99 time from arrival to
    completion and cell-updates/s, per tick policy (the first is the line's)."""
    import numpy as np
    import torch

    from paper_1701_07452_gb300 import serve as sv
    from paper_1701_07452_gb300.initial_conditions import turbulence_box_device
    dev = torch.device("cuda", torch.cuda.current_device())
    rng = np.random.default_rng(5)
    gaps = rng.exponential(1.0 / 50.0, size=requests)
    arrivals = np.cumsum(gaps) - gaps[0]
    ns = np.rint(np.exp(rng.uniform(np.log(32), np.log(192), size=requests))).astype(int)
    nsteps = np.maximum(1, np.rint(rng.integers(50, 501, size=requests) * steps_scale)).astype(int)
    reqs = []
    for r in range(requests):
        st = turbulence_box_device(int(ns[r]), 5000 + r, dev)
        st = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in st.items()}
        reqs.append(sv.Request(r, float(arrivals[r]), (int(ns[r]),) * 3, int(nsteps[r]), st))
    runs = {}
    for policy in policies:
        # srpt: up to 25 steps per tick for the runs of least remaining work,
        # 4e6 zones per step (1e8 cell-updates per tick)
        srv = sv.Server(state_bytes=150 << 30, work_bytes=40 << 30, max_boxes=requests,
                        max_n=int(ns.max()), tick_steps=25, policy=policy, tick_cells=1e8)
        recs = srv.run(reqs)
        runs[policy] = (sv.summarize(recs), srv.ticks)
        del srv
        torch.cuda.empty_cache()
    summ, ticks = runs[policies[0]]
    res = {"cell_updates_per_s": summ["cell_updates_per_s"], "p50_s": summ["p50_s"],
           "p99_s": summ["p99_s"], "solves_per_s": summ["solves_per_s"],
           "completed": summ["completed"], "failed": summ["failed"], "wall_s": summ["wall_s"],
           "ticks": ticks, "policy": policies[0],
           "workload": f"{requests} requests, Poisson 50/s (seed 5), edge log-uniform 32..192, "
                       f"steps U{{50..500}}" + (f" x {steps_scale}" if steps_scale != 1.0 else "") +
                       ", turbulence data seed 5000+r, 150 GB state budget, 25 steps per tick "
                       "(srpt: least remaining work first, up to 4e6 zones a step, 1e8 cell-updates "
                       "per tick)"}
    for policy in policies[1:]:
        o = runs[policy][0]
        res[policy] = {"cell_updates_per_s": o["cell_updates_per_s"], "p50_s": o["p50_s"],
                       "p99_s": o["p99_s"]}
    return res


def run_mode(args):
    """Secondary workloads, one JSON line each (not the headline line)."""
    import torch

    from paper_1701_07452_gb300 import binding as wb
    from paper_1701_07452_gb300.initial_conditions import turbulence_box_device
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    if args.mode == "batch":
        r = batch_figures(args.nbox, args.batch_steps, form=args.form, other_form=True,
                          oracle_boxes=4)
        line = {"metric": "solves/s (batched vs one box at a time)", "mode": "batch",
                "value": r.pop("solves_per_s"), "unit": "solves/s", "higher_is_better": True,
                "dtype": "f64", "data": "synthetic", "config": {"workload": r.pop("workload")}}
        line.update(r)
        print(json.dumps(line), flush=True)
        return 0
    if args.mode == "serve":
        r = serve_figures(args.requests, args.steps_scale, policies=("srpt", "fair"))
        line = {"metric": "serving p50/p99 completion latency and cell-updates/s", "mode": "serve",
                "value": r.pop("cell_updates_per_s"), "unit": "cell-updates/s",
                "higher_is_better": True, "dtype": "f64", "data": "synthetic",
                "config": {"workload": r.pop("workload")}}
        line.update(r)
        print(json.dumps(line), flush=True)
        return 0
    if args.mode in ("patches", "big"):
        n, p = (512, 8) if args.mode == "patches" else (768, 12)
        st = turbulence_box_device(n, SEED, dev)
        def run(patches, batch, read=True):
            g = wb.Grid((n, n, n), patches=(patches,) * 3, length=st["length"], batch_patches=batch)
            g.load(st["W"], st["bx"], st["by"], st["bz"], on_device=True, primitive=True)
            g.advance(1)
            g.load(st["W"], st["bx"], st["by"], st["bz"], on_device=True, primitive=True)
            torch.cuda.synchronize()
            e0, e1 = ev(), ev()
            e0.record(stream)
            g.advance(args.steps, sync=False)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            out = g.read(on_device=True) if read else None
            assert g.counters()["unphysical"] == 0
            del g
            torch.cuda.empty_cache()
            return ms, out
        if args.mode == "patches":
            # every patch resident: periodic images between stages
            ms_p, out_p = run(p, 0)
            how = "all patches resident, neighbour images between stages"
        else:
            ms_p, out_p = run(p, 152, read=False)
            how = "152 patches per pipeline pass, ghost rings recomputed"
        line = {"metric": METRIC, "mode": args.mode, "value": n ** 3 * args.steps / (ms_p * 1e-3),
                "unit": UNIT, "higher_is_better": True, "steps": args.steps, "dtype": "f64",
                "ms_per_step": ms_p / args.steps, "data": "synthetic",
                "config": {"workload": f"{n}^3 periodic turbulence box in {p}^3 patches of {n // p}^3, " + how}}
        if args.mode == "big":
            # the same box as one resident grid with periodic images, when the
            # device holds it (about 250 GB at 768^3 besides the initial data)
            del out_p
            torch.cuda.empty_cache()
            need = wb.grid_bytes(wb.make_desc((n, n, n), length=st["length"])) + (4 << 30)
            free = torch.cuda.mem_get_info()[0]
            if free > need:
                ms_s, _ = run(1, 0, read=False)
                line["single_grid_value"] = n ** 3 * args.steps / (ms_s * 1e-3)
                line["single_grid_config"] = f"one {n}^3 grid, all resident, periodic images between stages"
            else:
                line["single_grid_value"] = None
                line["single_grid_config"] = f"not run: {need / 2**30:.0f} GiB needed, {free / 2**30:.0f} GiB free"
        if args.mode == "patches":
            ms_q, out_q = run(p, 152)
            ms_s, out_s = run(1, 0)
            line["pipelined_value"] = n ** 3 * args.steps / (ms_q * 1e-3)
            line["pipelined_config"] = "152 patches per pipeline pass, ghost rings recomputed"
            line["single_grid_value"] = n ** 3 * args.steps / (ms_s * 1e-3)
            line["bit_exact_vs_single_grid"] = all(bool(torch.equal(a, b)) for a, b in zip(out_p, out_s))
            line["pipelined_bit_exact_vs_single_grid"] = all(bool(torch.equal(a, b))
                                                             for a, b in zip(out_q, out_s))
        print(json.dumps(line), flush=True)
        return 0
    return 1


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=N_BOX)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--mode", default="box", choices=["box", "batch", "serve", "patches", "big"],
                    help="box: the 256^3 box (default line); batch: ensemble of boxes, batched vs "
                         "one at a time; serve: request stream; patches: 512^3 in 64^3 patches vs "
                         "the single grid; big: 768^3 in 12^3 patches")
    ap.add_argument("--nbox", type=int, default=48,
                    help="batch: boxes of the ensemble (the first nbox of the seeded 1000)")
    ap.add_argument("--batch-steps", type=int, default=100)
    ap.add_argument("--no-extras", action="store_true",
                    help="default line without the batch and serving figures")
    ap.add_argument("--form", default="auto", choices=["auto", "persistent", "staged"],
                    help="batch mode: the autotuned form, or a given one without autotuning")
    ap.add_argument("--ref-sample", type=int, default=128,
                    help="reference arm: edge of the box the oracle steps per bench step")
    ap.add_argument("--requests", type=int, default=16)
    ap.add_argument("--steps-scale", type=float, default=1.0)
    args = ap.parse_args()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.mode != "box":
        return run_mode(args)

    import numpy as np
    import torch

    from paper_1701_07452_gb300 import binding as wb
    from paper_1701_07452_gb300.initial_conditions import turbulence_box

    assert args.warmup >= 3, "at least 3 warm-up steps"
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    n = args.n
    st = turbulence_box(n, SEED + rank)
    g = wb.Grid((n, n, n), length=st["length"])
    g.load_state(st)
    fp64_peak = wb.measure_fp64_peak()

    # ---- device-resident timing --------------------------------------------
    g.advance(args.warmup, sync=True)
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        g.profile_sweeps(True)
        e0.record(stream)
        g.advance(args.steps, sync=False)
        e1.record(stream)
        torch.cuda.synchronize()
        g.profile_sweeps(False)
    barrier(world)
    ms = e0.elapsed_time(e1)
    sweep_ms, sweep_launches = g.profile_read()
    counters = g.counters()
    if counters["unphysical"]:
        raise RuntimeError(f"unphysical state during the bench: {counters}")
    ms_max = max_over_ranks(ms, world, dev)
    value = world * n ** 3 * args.steps / (ms_max * 1e-3)

    # ---- end to end through the C ABI with host buffers -------------------
    nx = ny = nz = n
    pin = dict(dtype=torch.float64, pin_memory=True)
    U_h = torch.empty((5, nz, ny, nx), **pin)
    bx_h = torch.empty((nz, ny, nx + 1), **pin)
    by_h = torch.empty((nz, ny + 1, nx), **pin)
    bz_h = torch.empty((nz + 1, ny, nx), **pin)
    # the step's result is U and the face field (the zone field is their
    # derived mean and is not read back)
    g.read(out=(U_h.numpy(), bx_h.numpy(), by_h.numpy(), bz_h.numpy(), None))
    h2d = sum(t.numel() * 8 for t in (U_h, bx_h, by_h, bz_h))
    d2h = h2d
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        g.load(U_h.numpy(), bx_h.numpy(), by_h.numpy(), bz_h.numpy())
        g.advance(1, sync=True)
        g.read(out=(U_h.numpy(), bx_h.numpy(), by_h.numpy(), bz_h.numpy(), None))
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    e2e = world * n ** 3 * args.e2e_steps / e2e_s

    # ---- CPU baseline: oracle on a bounded sample -------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the workload itself, two steps (10-20 s on the host cores), and one
        # step of a 64^3 box of the same data on one core (a few seconds)
        steps_s = 2
        v, wall, used = cpu_sample(n, steps_s, st=st)
        v1, wall1, _ = cpu_sample(64, 1, threads=1)
        cpu = {"value": v, "unit": UNIT, "cores": used, "kind": "oracle",
               "sample": f"{steps_s} steps of the {n}^3 box itself ({wall:.1f} s)",
               "one_core": {"value": v1, "unit": UNIT, "cores": 1,
                            "sample": f"1 step of a 64^3 box of the same data ({wall1:.1f} s)"},
               "cpu_model": cpu_model()}
        import oracle
        oracle.set_threads(os.cpu_count() or 1)

    # ---- batched and served workloads (rank 0 of a 1-GPU run) -------------
    extras = {}
    if rank == 0 and world == 1 and not args.no_extras:
        extras["batch"] = batch_figures(args.nbox, args.batch_steps, other_form=False,
                                        oracle_boxes=3)
        extras["serve"] = serve_figures(args.requests, args.steps_scale)

    if rank == 0:
        per_launch_ms = sweep_ms / max(sweep_launches, 1)
        faces_per_launch = sweep_faces_per_step(n) / 6.0
        achieved = ALG_FLOPS_PER_FACE * faces_per_launch / (per_launch_ms * 1e-3) / 1e12
        achieved_exec = EXEC_FLOPS_PER_FACE * faces_per_launch / (per_launch_ms * 1e-3) / 1e12
        clk_summary = clk.summary()
        sm_mhz = clk_summary["sm_mhz"] or 2070.0
        props = torch.cuda.get_device_properties(dev)
        peak = props.multi_processor_count * FP64_FLOPS_PER_CLK_PER_SM * sm_mhz * 1e6 / 1e12
        launches_per_step = step_launches(g.desc)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded turbulence IC, no dataset)",
            "config": {"workload": workload_name(n),
                       "patches": "1 (single grid)", "l2": l2_note(n),
                       "parallelism": "replicas only" if world > 1 else "1 GPU"},
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": args.e2e_steps},
            "roofline": {"bound": "alu", "kernel": "k_sweep (MHDTVD flux)", "achieved": achieved,
                         "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": sweep_traffic(n),
                         "algorithmic_bytes": SWEEP_BYTES_PER_FACE * faces_per_launch,
                         "flops_per_face": ALG_FLOPS_PER_FACE,
                         "flops_kind": "algorithmic: the oracle's FP64 operations per face "
                                       "(instrumented scalar, oracle/count_flops.py)",
                         "executed": {"flops_per_face": EXEC_FLOPS_PER_FACE, "achieved": achieved_exec,
                                      "frac": achieved_exec / peak,
                                      "source": "ncu FP64 instruction counters of k_sweep, DFMA = 2"},
                         "peak_source": "nominal: SMs x 2 DFMA/clk x 2 flops x median SM clock "
                                        "under load; DFMA probe in this process: %.3f TFLOP/s"
                                        % (fp64_peak / 1e12),
                         "sweep_ms_per_launch": per_launch_ms,
                         "sweep_share_of_step": sweep_ms / ms},
            "step_roofline": step_roofline(value, peak),
            "cpu_baseline": cpu,
            "paper_context": {
                "note": "the paper's own CPU figures for the same 3D CTU+CT MHDTVD step (context, "
                        "not a target; other hardware, unstated initial data)",
                "zone_updates_per_s_per_node": {"XC_KNL Xeon Phi 7250": 6.5e6, "XC_BDW 2x Xeon E5-2695": 4.5e6,
                                                "XE_IL Opteron 6281": 2.0e6},
                "single_broadwell_core_cce": 2.7e5,
                "source": "Sec. 'Patch Size Optimization'; Table 'Effect of vectorization on floating "
                          "point instruction count' (8 x 32^3 zones x 100 steps in 96 s)"},
            "clocks": clk_summary,
            "gpu_launches": launches_per_step * args.steps,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
