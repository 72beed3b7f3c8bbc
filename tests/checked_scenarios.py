"""Every entry point and layout run through the index-checked build of the
library (run by test_gpu_checked.py in a process with WOMBAT_CHECKED=1):
single grids periodic (interior-only stages with images), outflow and 2D,
resident and pipelined patches, protection floors, batches in both forms
with mixed boundaries, a serving pool, the no-alloc step, loads and reads
through host, pinned and device buffers, totals, div b and stage dumps.
Prints one JSON line: the selftest result and the check word after each
scenario (0 = no out-of-range index)."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main():
    assert os.environ.get("WOMBAT_CHECKED") == "1"
    import torch
    from paper_1701_07452_gb300 import binding as wb
    from paper_1701_07452_gb300 import initial_conditions as ic
    out = {"selftest": wb.check_selftest()}
    wb.check_flags()  # clear

    def note(name):
        out[name] = wb.check_flags()

    st = ic.turbulence_box((12, 10, 9), seed=3)
    g = wb.Grid((12, 10, 9), length=st["length"], keep_stages=True)
    g.load_state(st)
    g.advance(2)
    g.read()
    g.totals()
    g.divb_max()
    for which in range(12):
        g.stage(which)
    note("grid_periodic")

    g = wb.Grid((12, 10, 9), length=st["length"], bc=(1, 1, 1))
    g.load_state(st)
    g.advance(2)
    g.read()
    note("grid_outflow")

    st2 = ic.turbulence_box((16, 16, 16), seed=4)
    for patches, batch in (((2, 2, 2), 0), ((2, 2, 2), 3), ((4, 2, 1), 0)):
        g = wb.Grid((16, 16, 16), patches=patches, length=st2["length"], batch_patches=batch)
        g.load_state(st2)
        g.advance(2)
        g.read()
        g.totals()
        note(f"patches_{patches[0]}{patches[1]}{patches[2]}_batch{batch}")

    st3 = ic.turbulence_box((16, 12, 1), seed=5)
    g = wb.Grid((16, 12, 1), length=st3["length"])
    g.load_state(st3)
    g.advance(3)
    g.read()
    note("grid_2d")

    st4 = ic.expansion_box(12, 11)
    g = wb.Grid((12, 12, 12), length=(1.0, 1.0, 1.0), prot_rho=1e-3, prot_p=1e-3)
    g.load_state(st4)
    g.advance(3)
    note("grid_protection")

    # loads and reads through pinned host and device buffers
    st5 = ic.random_box((10, 9, 8), seed=6)
    g = wb.Grid((10, 9, 8), length=st5["length"])
    g.load_state(st5)
    U, bx, by, bz, B = g.read()
    pin = [torch.from_numpy(a.copy()).pin_memory() for a in (U, bx, by, bz)]
    g.load(*[t.numpy() for t in pin])
    dev = [torch.from_numpy(a.copy()).cuda() for a in (U, bx, by, bz)]
    g.load(*dev, on_device=True)
    g.advance(1)
    g.read(on_device=True)
    note("load_read")

    boxes = [{"n": (12, 10, 9), "length": (12.0, 10.0, 9.0), "bc": (0, 0, 0)},
             {"n": (10, 12, 8), "length": (10.0, 12.0, 8.0), "bc": (1, 1, 1)},
             {"n": (8, 8, 8), "length": (8.0, 8.0, 8.0), "bc": (0, 1, 0)}]
    states = [ic.random_box(b["n"], seed=10 + i) for i, b in enumerate(boxes)]
    for form in ("persistent", "staged"):
        bt = wb.Batch(boxes, work_budget=1 << 22)
        bt.set_form(form)
        for i, s in enumerate(states):
            bt.load_state(i, s)
        bt.set_steps(-1, 3)
        bt.advance(3)
        for i in range(len(boxes)):
            bt.read(i)
        note(f"batch_{form}")

    pool = wb.Pool(state_bytes=64 << 20, work_bytes=64 << 20, max_boxes=4, max_n=16)
    a = pool.admit((12, 12, 12))
    b = pool.admit((8, 10, 12))
    for slot, n in ((a, (12, 12, 12)), (b, (8, 10, 12))):
        s = ic.random_box(n, seed=20 + slot)
        pool.load(slot, s["W"], s["bx"], s["by"], s["bz"], primitive=True)
        pool.set_steps(slot, 2)
    pool.advance(2)
    pool.release(a)
    pool.read(b)
    note("pool")

    st6 = ic.random_box((8, 8, 8), seed=7)
    d = wb.make_desc((8, 8, 8), length=st6["length"])
    gg = wb.Grid((8, 8, 8), length=st6["length"])
    gg.load_state(st6)
    U, bx, by, bz, _ = gg.read(on_device=True)
    outs = [torch.empty_like(x) for x in (U, bx, by, bz)]
    dt = torch.empty(1, dtype=torch.float64, device="cuda")
    wb.step_noalloc(d, U, bx, by, bz, *outs, dt)
    torch.cuda.synchronize()
    note("noalloc")

    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
