"""TEST INFRASTRUCTURE ONLY: algorithmic FP64 operation count of one
cell-update of the CTU+CT step (Sec. "MHD in Three Dimensions", Steps 1-11,
with the App. A MHDTVD flux), taken from the oracle's instrumented scalar
(flop_count.h: add/sub/mul/div/sqrt = 1, FMA = 2; identity operations of
the dense 7x7 matrices and operations on the parameters alone not counted).

The oracle evaluates each stage on the index ranges its successors read, so
it recomputes ghost rings; the count is therefore taken per unit (zone, face
or edge) of each section and multiplied by the units one interior
cell-update needs:

  sweep face (zone state + flux, Roe state + eigen-system + alpha + g-tilde,
  limiter, emitted flux)          x 6  (3 directions, predictor + corrector)
  reference EMF (Step 2)          x 1
  corner EMF (Steps 3, 9)         x 6  (3 edges, two passes)
  constrained transport (4, 11)   x 6  (3 faces, two passes)
  transverse state (Steps 5, 7)   x 3  (one state per direction)
  half-step reference EMF (8)     x 1
  conservative update (10)        x 1
  zone field + floors (11)        x 1
  CFL rate                        x 1

Usage: python oracle/count_flops.py [n] [steps] [seed]  (defaults: the
256^3 turbulence workload's data at 64^3, 2 steps, seed 2).  Prints one
table and a JSON line with flops per sweep face and per cell-update.
"""
from __future__ import annotations

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402

PER_UPDATE = {"eref": 1, "edge": 6, "ct": 6, "trans": 3, "erefh": 1, "update": 1, "final": 1,
              "dt": 1}
SWEEP_FACES_PER_UPDATE = 6


def count(n=64, steps=2, seed=2):
    """Per-unit means of every section and the totals, on the turbulence
    workload's initial data (a cube of side n, `steps` steps)."""
    from paper_1701_07452_gb300.initial_conditions import turbulence_box
    st = turbulence_box((n, n, n), seed=seed)
    g = oracle.Grid((n, n, n), st["length"], counting=True)
    g.load_state(st)
    # the initial density is exactly 1, so the first step's divisions by it
    # are identity operations; count from the second step on
    g.advance(1)
    oracle.flop_reset()
    g.advance(steps)
    rep = oracle.flop_report()
    mean = {k: (f / u if u else 0.0) for k, (f, u) in rep.items()}
    faces = rep["face"][1]
    # per sweep face: each section's mean per its own unit (one zone, one
    # face, one limiter zone and one emitted face per face of a long pencil),
    # plus the HLL faces' share
    per_face = mean["cell"] + mean["face"] + mean["limit"] + mean["emit"]
    per_face += rep["hll"][0] / faces if faces else 0.0
    per_update = SWEEP_FACES_PER_UPDATE * per_face
    per_update += sum(PER_UPDATE[k] * mean[k] for k in PER_UPDATE)
    return {"workload": f"turbulence {n}^3, seed {seed}, {steps} steps after the first",
            "sections": {k: {"flops": f, "units": u, "per_unit": round(mean[k], 3)}
                         for k, (f, u) in rep.items()},
            "flops_per_sweep_face": round(per_face, 2),
            "flops_per_cell_update": round(per_update, 2),
            "sweep_share": round(SWEEP_FACES_PER_UPDATE * per_face / per_update, 4)}


def main():
    args = [int(a) for a in sys.argv[1:]]
    r = count(*args)
    print(f"# oracle FP64 operation count, {r['workload']}")
    print(f"{'section':8s} {'flops':>14s} {'units':>12s} {'per unit':>10s}")
    for k, v in r["sections"].items():
        print(f"{k:8s} {v['flops']:14d} {v['units']:12d} {v['per_unit']:10.2f}")
    print(f"flops per sweep face: {r['flops_per_sweep_face']:.2f}")
    print(f"flops per cell-update: {r['flops_per_cell_update']:.2f} "
          f"(sweeps {100 * r['sweep_share']:.1f} %)")
    print(json.dumps({k: r[k] for k in ("workload", "flops_per_sweep_face",
                                        "flops_per_cell_update", "sweep_share")}))


if __name__ == "__main__":
    main()
