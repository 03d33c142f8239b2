"""Run one of the synthetic workloads through the C ABI and print per-phase timings.

    python -m paper_2410_09189_gb300.run --workload icosa --steps 4 [--grid 96]
        [--precision mixed|fp64] [--host-driven] [--nrep 1]

A thin driver (argument parsing, input generation, the library's own profile counters): it
builds the library if needed, creates a context from seeded smooth random orbitals, kicks
every replica along its axis, steps, and prints one JSON line.  It is the command the
profile summaries under ``profiles/`` are taken with.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="icosa", choices=["icosa", "ring", "small"])
    ap.add_argument("--grid", type=int, default=0, help="edge points (0: the workload's own)")
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--nrep", type=int, default=0, help="replicas (0: one per kick axis)")
    ap.add_argument("--host-driven", action="store_true",
                    help="step without the CUDA graph (one launch per kernel)")
    ap.add_argument("--H-thrs", type=float, default=1e-7)
    ap.add_argument("--seed-order", type=int, default=1, choices=[1, 2],
                    help="SCF seed: 1 linear (the paper's), 2 quadratic extrapolation of H")
    ap.add_argument("--grid-basis", action="store_true",
                    help="propagate the occupied orbitals on the grid (no virtual orbitals)")
    args = ap.parse_args(argv)

    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2410_09189_gb300 import inputs, rmgtd

    torch.cuda.set_device(0)
    s = {"icosa": inputs.icosa, "ring": inputs.ring, "small": inputs.small}[args.workload]()
    if args.grid:
        s = dataclasses.replace(s, n=(args.grid,) * 3)
    axes = s.kick_axes
    nrep = args.nrep or len(axes)
    raw = inputs.smooth_random_orbitals(s).reshape(s.N, s.Ng)
    prec = rmgtd.PREC_MIXED if args.precision == "mixed" else rmgtd.PREC_FP64
    kw = {}
    if args.grid_basis:   # the occupied orbitals only, propagated on the grid
        s = dataclasses.replace(s, nvirt=0)
        raw = raw[:s.N]
        kw["grid_basis"] = True
    t0 = time.perf_counter()
    ctx = rmgtd.Context(s, raw, nrep=nrep, H_thrs=args.H_thrs, dP_thrs=1e-10, poisson_tol=1e-10,
                        precision=prec, use_graph=not args.host_driven,
                        seed_order=args.seed_order, **kw)
    torch.cuda.synchronize()
    setup = time.perf_counter() - t0
    for r in range(nrep):
        ctx.kick(r, axes[r % len(axes)], s.kappa)
    ctx.profile(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = ctx.step(args.steps)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ph, calls, launches = ctx.profile_read()
    solves, iters = ctx.profile_counters()
    ctx.close()
    print(json.dumps({"workload": s.name, "grid": list(s.n), "N": s.N, "nrep": nrep,
                      "precision": args.precision,
                      "grid_basis": bool(args.grid_basis), "seed_order": args.seed_order,
                      "setup_s": setup, "steps": args.steps,
                      "ms_per_step": wall / max(args.steps, 1) * 1e3,
                      "scf_passes_per_replica_step": float(st["passes"].mean()),
                      "series_terms_per_pass": float(st["terms_sum"].sum() / max(st["passes"].sum(), 1)),
                      "phase_ms": ph, "phase_calls": calls, "launches": launches,
                      "hartree_cg_per_solve": iters / max(solves, 1)}), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
