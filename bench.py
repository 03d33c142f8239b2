#!/usr/bin/env python
"""Benchmark of the RT-TDDFT time step (Algorithm 1) on GB300.

Workload: the benzene-like ring (12 pseudo-atoms, s-type KB on the 6 heavy atoms), 64^3 grid
at h = 0.35 bohr, N = 15 occupied + 15 virtual orbitals, three replicas kicked along x, y, z
(kappa = 1e-3) propagated together, dt = 0.05 a.u., H_thrs = 1e-7, dP_thrs = 1e-10.  One
"step" advances all three replicas by one time step, SCF passes included.  Orbitals are
seeded smooth random fields orthonormalised on the device (synthetic data).

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle on the same
workload instead (a bounded sample per step).  Under torchrun every rank propagates its own
replica set (independent problems, no data-path collective): weak scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "RT-TDDFT time-steps/sec and grid-point·orbital updates/sec, mixed vs FP64 GPU"
UNIT = "time-steps/s"
SUBSPACE_SCF = 200          # set-up SCF iterations inside the orbital block (stationary start)
SUR_STEPS = 300             # trajectory steps recorded to train the learned SCF seed
SUR_ITERS = 2000            # Adam iterations of that training
FP64_PEAK_GFLOPS = 1250.0   # GB300 float64 rate (nominal 1.25 TFLOP/s)


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-i", str(self.device), "-lms", "20"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # the timed region is short (~0.4 ms per step): let sampling start first (first line
        # written, at most 1.5 s), so the samples cover the region itself
        t0 = time.time()
        while time.time() - t0 < 1.5 and self.proc.poll() is None:
            try:
                if os.path.getsize(self.path) > 0:
                    break
            except OSError:
                break
            time.sleep(0.01)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 9:
                rows.append(p)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def _workload():
    from paper_2410_09189_gb300 import inputs
    s = inputs.ring()
    raw = inputs.smooth_random_orbitals(s).reshape(s.N, s.Ng)
    return s, raw


def _config(s, precision):
    return {"workload": "ring-12-atoms-64^3-N30-kicks-xyz", "grid": list(s.n), "h": s.h,
            "N": s.N, "nocc": s.nocc, "replicas": 3, "dt": s.dt, "kappa": s.kappa,
            "H_thrs": 1e-7, "dP_thrs": 1e-10, "precision": precision,
            "orbitals": "seeded smooth random fields, orthonormalised on the device",
            "initial_state": f"ground state inside the orbital block (<= {SUBSPACE_SCF} SCF "
                             "iterations at set-up), then kicks along x, y, z",
            "l2": "flushed (256 MiB write) between timed steps"}


# ---------------------------------------------------------------------------------------
def max_over_ranks(value: float, world: int, device: str = "cuda") -> float:
    """The largest value over all ranks (the timed region's wall on the slowest GPU);
    torch.distributed must be initialised when world > 1."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(steps: int, world: int, max_ms: float) -> float:
    """Whole-job time-steps/s: every rank advances its own replica set `steps` steps (weak
    scaling), and the job takes as long as the slowest rank."""
    return world * steps / (max_ms * 1e-3)


def run_reference(args):
    """The FP64 CPU oracle on the same workload: each step is one time step of ONE replica
    (a bounded sample), reported in the 3-replica unit."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import hamiltonian as oham, tddft
    s, raw = _workload()
    phi = oham.orthonormalize(s, raw)
    pr = tddft.Propagator(s, phi, tddft.Options(dt=s.dt))
    st = pr.initial_state()
    st["P0"] = pr.kick(st["P0"], 2, s.kappa)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        pr.step(st)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    per_rep = statistics.mean(times)
    value = 1.0 / (3.0 * per_rep)
    cores = os.cpu_count()
    try:
        from threadpoolctl import threadpool_info
        cores = max([d.get("num_threads", 1) for d in threadpool_info()] or [cores])
    except Exception:
        pass
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 3.0 * per_rep * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": _config(s, "fp64-cpu-oracle"),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": "one time step of one of the three replicas per timed "
                                      "step, scaled x3"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def cpu_baseline_sample(budget_s: float = 20.0):
    """Time the oracle as it stands on a bounded sample of the workload (host cores)."""
    from oracle import hamiltonian as oham, tddft
    s, raw = _workload()
    phi = oham.orthonormalize(s, raw)
    pr = tddft.Propagator(s, phi, tddft.Options(dt=s.dt))
    st = pr.initial_state()
    st["P0"] = pr.kick(st["P0"], 2, s.kappa)
    times = []
    t_start = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        pr.step(st)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_start > budget_s or len(times) >= 4:
            break
    per_rep = statistics.mean(times)
    cores = os.cpu_count()
    try:
        from threadpoolctl import threadpool_info
        cores = max([d.get("num_threads", 1) for d in threadpool_info()] or [cores])
    except Exception:
        pass
    return {"value": 1.0 / (3.0 * per_rep), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{len(times)} time step(s) of one replica (x3 for the 3-replica unit)"}


# ---------------------------------------------------------------------------------------
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # 152 SMs x 128 FP32 lanes x FMA x 2.07 GHz


def _mg_levels(n):
    """Level sizes of the Hartree multigrid (same coarsening rule as the library): halve while
    every dimension is even and >= 4, stopping at a level below the finest with <= 64 points;
    the first level >= 1 with <= 4096 points starts the single-block tail."""
    nx, ny, nz = n
    lv = []
    while True:
        lv.append(nx * ny * nz)
        if len(lv) >= 12 or nx % 2 or ny % 2 or nz % 2 or min(nx, ny, nz) < 4:
            break
        if len(lv) >= 2 and lv[-1] <= 64:
            break
        nx, ny, nz = nx // 2, ny // 2, nz // 2
    tail = next((l for l in range(1, len(lv)) if lv[l] <= 4096), None)
    return lv, tail


def hartree_bytes(n, solves, iters, mixed, precond="dst"):
    """Algorithmic bytes of the persistent Hartree solve: each array every phase reads or
    writes, counted once (no stencil re-reads).  Per fine point and CG iteration: A z with its
    dots 5 s_V and the vector update 10 s_V (s_V = 4 float32 / 8 float64; the first iteration
    of a solve reads no p, A p: -4 s_V), plus the preconditioner -- the sine-transform one
    (the default on this workload) 32 + 2 s_V (five line passes, each reading and writing the
    grid once: r in s_V, three float32 intermediates, z out in s_V); the multigrid V-cycle at
    level 0 45 + 2 s_V (pre-sweeps 8 + s_V, residual with the box restriction 8.5,
    prolongation 8.5, post-sweeps 12 + 8 + s_V), each coarser multi-block level 49 bytes per
    own point, the tail 8 bytes per tail point.  Per solve: moments and right-hand side
    2 s_rho + 4 s_ghost + 3 s_V."""
    sv = 4 if mixed else 8
    lv, tail = _mg_levels(n)
    if precond == "dst":
        per_it = lv[0] * (32 + 2 * sv + 15 * sv)
    else:
        nmulti = tail if tail is not None else len(lv)
        per_it = lv[0] * (45 + 2 * sv + 15 * sv)
        per_it += sum(49 * lv[l] for l in range(1, nmulti))
        if tail is not None:
            per_it += 8 * lv[tail]
    prologue = lv[0] * (2 * sv + 4 * sv + 3 * sv)
    return float(iters) * per_it + float(solves) * (prologue - 4 * sv * lv[0])


def kernel_source_sha(source, begin, end):
    """sha256 of the kernel's source text: the lines from the first one starting with
    `begin` to the first later one starting with `end` (inclusive) of csrc/`source`."""
    import hashlib
    lines = open(os.path.join(ROOT, "paper_2410_09189_gb300", "csrc", source)).read().splitlines()
    i = next(k for k, l in enumerate(lines) if l.startswith(begin))
    j = next(k for k in range(i + 1, len(lines)) if lines[k].startswith(end))
    return hashlib.sha256("\n".join(lines[i:j + 1]).encode()).hexdigest()


def _traffic(kernel, workload):
    """dram bytes per launch from the committed ncu summary, if it was taken on the current
    source of the kernel (sha256 of the kernel's source region), else None."""
    path = os.path.join(ROOT, "profiles", f"traffic_{kernel}_{workload}.txt")
    try:
        kv = dict(line.strip().split("=", 1) for line in open(path)
                  if "=" in line and not line.startswith("#"))
        if kernel_source_sha(kv["source"], kv["begin"], kv["end"]) != kv["sha256"]:
            return None
        return float(kv["dram_bytes_per_launch"])
    except Exception:
        return None


def _flops_per_phase(N, Ng, rep_passes, terms_total):
    """Algorithmic work of the float64 phases (per whole timed region)."""
    return {
        # rho = sum_ij S_ij phi_i phi_j with S symmetric: N(N+1)/2 multiply-adds per point
        "rho": float(rep_passes) * Ng * N * (N + 1),
        # H_ij = h^3 sum_g phi_i V phi_j, j >= i: N(N+1)/2 multiply-adds per point (+ V)
        "hupdate": float(rep_passes) * Ng * (N * (N + 1) + N),
        # two N x N x N products per commutator term
        "eldyn": float(terms_total) * 4.0 * N ** 3,
    }


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    __graft_entry__.build()
    from paper_2410_09189_gb300 import rmgtd

    prec = rmgtd.PREC_MIXED if args.precision == "mixed" else rmgtd.PREC_FP64
    s, raw = _workload()
    kw = dict(nrep=3, H_thrs=1e-7, dP_thrs=1e-10, poisson_tol=1e-10,
              subspace_scf=SUBSPACE_SCF)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB
    stream = torch.cuda.current_stream()

    def timed_steps(ctx, nsteps, profile, nvtx_name="rmgtd_other"):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(nsteps)]
        if profile:
            ctx.profile(True)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        st = []
        torch.cuda.nvtx.range_push(nvtx_name)
        for i in range(nsteps):
            flush.zero_()
            ev[i][0].record(stream)
            st.append(ctx.step(1))
            ev[i][1].record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        wall = time.perf_counter() - w0
        prof = ctx.profile_read() if profile else None
        return [a.elapsed_time(b) for a, b in ev], np.concatenate(st), wall, prof

    def run_path(p, nsteps, with_clocks, state=None, net=None):
        c = rmgtd.Context(s, raw, use_graph=True, precision=p, **kw)
        if state is None:
            for a in range(3):
                c.kick(a, a, s.kappa)
        else:
            c.load(state)
        if net is not None:
            c.attach_net(net)
        for _ in range(args.warmup):
            c.step(1)
        smp = ClockSampler(local)
        if with_clocks:
            smp.start()
        ms, stt, wl, prof = timed_steps(c, nsteps, profile=True,
                                        nvtx_name="rmgtd_timed" if with_clocks else "rmgtd_other")
        clk = smp.stop() if with_clocks else None
        c.close()
        tot = max_over_ranks(float(sum(ms)), world)
        return tot, stt, wl, prof[2], clk

    # timed region: every step is one CUDA graph (device-side SCF and Hartree loops)
    total_ms, st, wall, launches, clocks = run_path(prec, args.steps, True)
    rep_passes = int(st["passes"].sum())
    terms_total = int(st["terms_sum"].sum())
    value = job_throughput(args.steps, world, total_ms)
    ms_per_step = total_ms / args.steps
    other = rmgtd.PREC_FP64 if prec == rmgtd.PREC_MIXED else rmgtd.PREC_MIXED
    o_ms, o_st, _, _, _ = run_path(other, args.steps, False)
    other_path = {"precision": "fp64" if other == rmgtd.PREC_FP64 else "mixed",
                  "value": world * args.steps / (o_ms * 1e-3), "unit": UNIT,
                  "ms_per_step": o_ms / args.steps,
                  "scf_passes_per_replica_step": float(o_st["passes"].sum()) / (3.0 * args.steps)}

    # the mixed path with the learned seed: a network trained (library kernels only) on the
    # first SUR_STEPS steps of this workload's own trajectory, then the continuation timed
    # with and without it from the same state (a window the network has not seen)
    surrogate_path = None
    if prec == rmgtd.PREC_MIXED and not args.no_surrogate:
        from paper_2410_09189_gb300 import surrogate
        tctx = rmgtd.Context(s, raw, use_graph=True, precision=prec, **kw)
        for a in range(3):
            tctx.kick(a, a, s.kappa)
        t0 = time.perf_counter()
        net, rep = surrogate.train_on_trajectory(tctx, nsteps=SUR_STEPS, iters=SUR_ITERS,
                                                 batch=8, lr=5e-4)
        train_s = time.perf_counter() - t0
        state = os.path.join(tempfile.mkdtemp(), "state.bin")
        tctx.save(state)
        tctx.close()
        p_ms, p_st, _, _, _ = run_path(prec, args.steps, False, state=state)
        n_ms, n_st, _, _, _ = run_path(prec, args.steps, False, state=state, net=net)
        surrogate_path = {
            "value": world * args.steps / (n_ms * 1e-3), "unit": UNIT,
            "ms_per_step": n_ms / args.steps,
            "scf_passes_per_replica_step": float(n_st["passes"].sum()) / (3.0 * args.steps),
            "same_window_without_seed": {
                "value": world * args.steps / (p_ms * 1e-3), "ms_per_step": p_ms / args.steps,
                "scf_passes_per_replica_step": float(p_st["passes"].sum()) / (3.0 * args.steps)},
            "window": f"steps {SUR_STEPS + args.warmup + 1}..{SUR_STEPS + args.warmup + args.steps}"
                      " after the kicks",
            "training": {"trajectory_steps": SUR_STEPS, "adam_iterations": SUR_ITERS, "batch": 8,
                         "lr": 5e-4, "seconds_incl_recording": train_s,
                         "heldout_seed_rms_ratio": rep["heldout_ratio"],
                         "samples": rep["train_samples"]}}

    # second timed region, host-driven steps with CUDA events around every phase on the
    # library's stream: the per-kernel durations behind the roofline
    pctx = rmgtd.Context(s, raw, use_graph=False, precision=prec, **kw)
    for a in range(3):
        pctx.kick(a, a, s.kappa)
    for _ in range(args.warmup):
        pctx.step(1)
    p_ms, p_st, _, (phase_ms, phase_calls, _) = timed_steps(pctx, args.steps, profile=True,
                                                            nvtx_name="rmgtd_host_driven")
    h_solves, h_iters = pctx.profile_counters()
    pctx.close()
    p_rep_passes = int(p_st["passes"].sum())
    p_terms = int(p_st["terms_sum"].sum())

    peaks, peak_kind = _peaks()
    mixed = prec == rmgtd.PREC_MIXED
    flops = _flops_per_phase(s.N, s.Ng, p_rep_passes, p_terms)
    dom = max(phase_ms, key=lambda k: phase_ms[k])
    # the dominant kernel: the Hartree solve is one cooperative launch per DFT evaluation
    kname = "k_hartree_coop"
    h_calls = max(phase_calls["hartree"], 1)
    h_bytes = hartree_bytes(s.n, h_solves, h_iters, mixed) / h_calls
    h_s = phase_ms["hartree"] / h_calls * 1e-3
    achieved = h_bytes / h_s / 1e9
    roof = {"kernel": f"{kname}<{'float' if mixed else 'double'}>", "phase": "hartree",
            "dominant_phase": dom, "bound": "hbm", "achieved": achieved,
            "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
            "traffic": _traffic(kname, "ring64") if mixed else None,
            "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, mean of the "
                              "first two launches of the host-driven region (2 CG iterations "
                              "each; profiles/traffic_k_hartree_coop_ring64.txt)",
            "algorithmic_bytes_per_launch": h_bytes, "launch_ms": h_s * 1e3,
            "cg_iterations_per_solve": h_iters / max(h_solves, 1),
            "peak_source": f"{peak_kind} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
            "timing": "CUDA events on the library stream around each Hartree launch, "
                      "host-driven steps over the same workload (second timed region)"}
    # the other phases: arithmetic against the ALU peak of their precision
    alu_peak = FP32_PEAK_TFLOPS if mixed else FP64_PEAK_GFLOPS / 1e3
    phases = {}
    for ph in ("rho", "hupdate", "eldyn"):
        if phase_ms.get(ph, 0) > 0:
            tf = flops[ph] / (phase_ms[ph] * 1e-3) / 1e12
            pk = FP64_PEAK_GFLOPS / 1e3 if ph == "eldyn" else alu_peak
            phases[ph] = {"bound": "alu", "achieved": tf, "peak": pk, "unit": "TFLOP/s",
                          "frac": tf / pk, "ms_per_call": phase_ms[ph] / max(phase_calls[ph], 1)}
    roof["other_phases"] = phases
    roof["alu_peak_source"] = ("float32: 152 SMs x 128 lanes x 2 flop x 2.07 GHz = 80.5 TFLOP/s "
                               "(nominal); float64: 1.25 TFLOP/s (nominal GB300)")

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == rmgtd.PREC_FP64 else "f32+f64",
        "data": "synthetic", "config": _config(s, args.precision),
        "grid_point_orbital_updates_per_s": value * s.Ng * s.N * 3,
        "scf_passes_per_replica_step": rep_passes / (3.0 * args.steps),
        "commutator_terms_per_expansion": terms_total / max(rep_passes, 1),
        "other_path": other_path,
        "surrogate_path": surrogate_path,
        "phase_ms_per_step_host_driven": {k: v / args.steps for k, v in phase_ms.items()},
        "ms_per_step_host_driven": float(sum(p_ms)) / args.steps,
        "gpu_launches": launches, "roofline": roof, "clocks": clocks,
        "wall_s_timed_region": wall,
    }

    # end to end through the public API: host orbitals in, dipoles out every step
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    c2 = rmgtd.Context(s, raw, use_graph=True, precision=prec, **kw)
    for a in range(3):
        c2.kick(a, a, s.kappa)
    for _ in range(args.steps):
        c2.step(1)
        for a in range(3):
            c2.dipole(a)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    c2.close()
    h2d = raw.nbytes + s.pos.nbytes * 3
    result["e2e"] = {"value": world * args.steps / e2e_s, "unit": UNIT,
                     "h2d_bytes_per_step": h2d / args.steps,
                     "d2h_bytes_per_step": 3 * 3 * 8 + 3 * 24,
                     "includes": "context creation from host orbitals (upload, set-up, "
                                 "initial SCF), 3 kicks, steps, dipole read-back per step"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline_sample()
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result), flush=True)
    return 0


def run_batch8(args):
    """The batched workload: eight clusters (20-150 atoms, 48^3-96^3), three kicks each,
    stepped by one CUDA graph per time step (rmgtd_batch), against the same contexts stepped
    one after another; mixed path, launch configurations from the autotuner."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2410_09189_gb300 import inputs, rmgtd

    def make():
        out = []
        for i in range(8):
            s = inputs.cluster(i)
            raw = inputs.smooth_random_orbitals(s).reshape(s.N, s.Ng)
            c = rmgtd.Context(s, raw, nrep=3, H_thrs=1e-7, dP_thrs=1e-10, poisson_tol=1e-10,
                              precision=rmgtd.PREC_MIXED, use_graph=True)
            for a in range(3):
                c.kick(a, a, 1e-3)
            out.append(c)
        return out

    t0 = time.perf_counter()
    ctxs = make()
    setup_s = time.perf_counter() - t0
    choices = [c.autotune() for c in ctxs]
    stream = torch.cuda.current_stream()

    def timed(step_all):
        for _ in range(args.warmup):
            step_all(1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = step_all(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), st

    # both variants step the same window of the trajectory: the states after the kicks are
    # saved and restored before the second one
    tmpdir = tempfile.mkdtemp(prefix="rmgtd_batch8_")
    paths = [os.path.join(tmpdir, f"ctx{i}.bin") for i in range(len(ctxs))]
    for c, pth in zip(ctxs, paths):
        c.save(pth)
    seq_ms, seq_st = timed(lambda k: [c.step(k) for c in ctxs])
    seq_passes = float(np.mean([st["passes"].mean() for st in seq_st]))
    for c, pth in zip(ctxs, paths):
        c.load(pth)
    batch = rmgtd.Batch(ctxs)
    bat_ms, bat_st = timed(lambda k: batch.step(k))
    batch.close()
    for pth in paths:
        os.remove(pth)
    os.rmdir(tmpdir)
    passes = float(np.mean([st["passes"].mean() for st in bat_st]))
    for c in ctxs:
        c.close()
    grid_pts = sum(inputs.cluster(i).Ng * inputs.cluster(i).N for i in range(8))
    out = {"metric": "batched RT-TDDFT time-steps/sec (8 clusters x 3 kicks per step)",
           "value": args.steps / (bat_ms * 1e-3), "unit": "time-steps/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": bat_ms / args.steps,
           "higher_is_better": True, "dtype": "f32+f64", "data": "synthetic",
           "config": {"workload": "clusters-8-(20..150 atoms)-(48^3..96^3)-kicks-xyz",
                      "clusters": [{"atoms": int(len(inputs.cluster(i).Z)),
                                    "grid": list(inputs.cluster(i).n), "N": inputs.cluster(i).N}
                                   for i in range(8)],
                      "precision": "mixed", "H_thrs": 1e-7, "initial_state": "P0 = diag(f)"},
           "one_graph_per_step": {"value": args.steps / (bat_ms * 1e-3)},
           "contexts_one_after_another": {"value": args.steps / (seq_ms * 1e-3),
                                          "ms_per_step": seq_ms / args.steps,
                                          "scf_passes_per_replica_step": seq_passes},
           "window": "both variants step the same trajectory window (states restored)",
           "grid_point_orbital_updates_per_s": grid_pts * 3 * args.steps / (bat_ms * 1e-3),
           "scf_passes_per_replica_step": passes, "setup_s": setup_s,
           "autotune_choices": choices}
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true",
                    help="skip training and timing the learned SCF seed")
    ap.add_argument("--batch8", action="store_true",
                    help="time the batched workload of eight clusters instead")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.batch8:
        return run_batch8(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
