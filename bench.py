#!/usr/bin/env python
"""Benchmark of the RT-TDDFT time step (Algorithm 1) on GB300.

Headline workload (default): the 147-atom Mackay icosahedron (Z = 1 Gaussian-erf wells with an
s-type Kleinman-Bylander projector on every atom), 128^3 grid at h = 0.4 bohr, N = 74 doubly
occupied + 74 virtual orbitals, one replica kicked along z (kappa = 1e-3), dt = 0.05 a.u.,
H_thrs = 1e-7, dP_thrs = 1e-10, started from P_0 = diag(f) of seeded smooth random orbitals
orthonormalised on the device (synthetic data; no molecular inputs exist here).  One "step" is
one time step of the replica, SCF passes included.  `value` is the mixed path (tensor-core
bfloat16 split products around a float64 reference state); the float64 path is timed on the
same workload.  The accuracy of both paths is stated against the stored FP64 oracle run of the
same workload (tests/golden/icosa128_window.json).  The 12-atom ring (64^3, N = 30, three
kicks) is measured as a secondary line.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle on the same
workload.  Under torchrun every rank propagates its own replica (independent problems, no
data-path collective): weak scaling.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import platform
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
SUR_STEPS = 300             # trajectory steps recorded to train the learned SCF seed (ring)
SUR_ITERS = 2000            # Adam iterations of that training
SPECTRUM_POINTS = 2000      # frequencies of the e2e absorption spectrum (0 .. 1 Ha)
SPECTRUM_DAMPING = 0.005    # its exponential damping (Ha)
GRID_BASIS_WARMUP = 1       # steps of the grid-basis line before its timed steps
GRID_BASIS_STEPS = 3
FP64_PEAK_TFLOPS = 1.25     # GB300 float64 rate (nominal)
REF_BUDGET_S = 150.0        # wall-clock budget of the oracle's timed steps (reference arm)
CPU_BASELINE_BUDGET_S = 30.0

# the workloads: constructor, replicas and kick axes, start, stored oracle run
WORKLOADS = {
    "icosa": dict(label="icosahedron-147-atoms-128^3-N148-kick-z", nrep=1, axes=(2,),
                  subspace_scf=0, golden="icosa128_window.json", trajectory_steps=1000,
                  start="P_0 = diag(f) of the orthonormalised seeded orbitals, kick along z"),
    "ring": dict(label="ring-12-atoms-64^3-N30-kicks-xyz", nrep=3, axes=(0, 1, 2),
                 subspace_scf=200, golden="ring64_three_kicks.json", trajectory_steps=2000,
                 start="ground state inside the orbital block (<= 200 SCF iterations at set-up), "
                       "then kicks along x, y, z"),
}
BENCH_THRESHOLDS = dict(H_thrs=1e-7, dP_thrs=1e-10, poisson_tol=1e-10)


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


def _system(name):
    from paper_2410_09189_gb300 import inputs
    s = inputs.icosa() if name == "icosa" else inputs.ring()
    raw = inputs.smooth_random_orbitals(s).reshape(s.N, s.Ng)
    return s, raw


def _config(name, s, precision):
    w = WORKLOADS[name]
    return {"workload": w["label"], "grid": list(s.n), "h": s.h, "N": s.N, "nocc": s.nocc,
            "natoms": int(len(s.Z)), "kb_projectors": s.nproj, "replicas": w["nrep"],
            "dt": s.dt, "kappa": s.kappa, **BENCH_THRESHOLDS, "precision": precision,
            "orbitals": "seeded smooth random fields, orthonormalised on the device",
            "initial_state": w["start"],
            "l2": "flushed (256 MiB write) between timed steps; orbital planes exceed L2"}


def _golden(name):
    with open(os.path.join(ROOT, "tests", "golden", WORKLOADS[name]["golden"])) as f:
        return json.load(f)


def accuracy_against_oracle(d, e, t, golden, steps_done):
    """Errors of one GPU trajectory against the stored oracle run, over the stored steps the
    trajectory covers: dipole max_t |d - d_ref| / max_t |d_ref(t) - d_ref(0)| (per replica,
    worst replica reported), energy max_t |E - E_ref|, trace max_t |Tr P - Tr P_ref|.
    d[k][a], e[k][a], t[k][a]: observables after step k (k = 0: after the kicks)."""
    out = {"dipole_rel_err": 0.0, "energy_err": 0.0, "trace_err": 0.0}
    nst = 0
    for a, tr in enumerate(golden["replicas"]):
        steps = tr.get("step", list(range(len(tr["dipole"]))))
        use = [i for i, k in enumerate(steps) if k <= steps_done]
        ref = np.array(tr["dipole"])[use]
        got = np.array([d[steps[i]][a] for i in use])
        scale = np.max(np.abs(np.array(tr["dipole"]) - np.array(tr["dipole"])[0]))
        out["dipole_rel_err"] = max(out["dipole_rel_err"], float(np.max(np.abs(got - ref)) / scale))
        out["energy_err"] = max(out["energy_err"], float(np.max(np.abs(
            np.array([e[steps[i]][a] for i in use]) - np.array(tr["energy"])[use]))))
        out["trace_err"] = max(out["trace_err"], float(np.max(np.abs(
            np.array([t[steps[i]][a] for i in use]) - np.array(tr["trace"])[use]))))
        nst = steps[use[-1]]
    out["window"] = f"steps 0..{nst} after the kick(s), compared at the oracle's stored steps"
    out["oracle_thresholds"] = {k: golden["options"][k] for k in ("H_thrs", "dP_thrs")}
    return out


def trajectory_observables(ctx, nrep, nsteps, every=1):
    """dipole, energy and Tr P of every replica after each `every`-th step (k = 0: now)."""
    from paper_2410_09189_gb300 import rmgtd
    d, e, t = {}, {}, {}

    def rec(k):
        d[k] = [ctx.dipole(a) for a in range(nrep)]
        e[k] = [ctx.energy(a) for a in range(nrep)]
        t[k] = [float(np.trace(ctx.get_matrix(rmgtd.MAT_P_RE, a))) for a in range(nrep)]

    rec(0)
    k = 0
    while k < nsteps:
        n = min(every, nsteps - k)
        ctx.step(n)
        k += n
        rec(k)
    return d, e, t


# ---------------------------------------------------------------------------------------
def _host_info():
    model = platform.processor() or platform.machine()
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return {"cpu": model, "machine": platform.machine(), "logical_cores": os.cpu_count()}


_BLAS_SET = ("openblas_set_num_threads", "openblas_set_num_threads64_",
             "scipy_openblas_set_num_threads", "scipy_openblas_set_num_threads64_")
_BLAS_GET = ("openblas_get_num_threads", "openblas_get_num_threads64_",
             "scipy_openblas_get_num_threads", "scipy_openblas_get_num_threads64_")


def _blas_libs():
    """(get, set) thread-count functions of every OpenBLAS loaded in this process (numpy's and
    scipy's copies), found through /proc/self/maps -- threadpoolctl is not installed
    everywhere."""
    import ctypes
    paths = set()
    try:
        for line in open("/proc/self/maps"):
            f = line.split()[-1]
            if "blas" in os.path.basename(f).lower() and ".so" in f:
                paths.add(f)
    except OSError:
        return []
    out = []
    for p in sorted(paths):
        try:
            lib = ctypes.CDLL(p)
        except OSError:
            continue
        get = next((getattr(lib, n) for n in _BLAS_GET if hasattr(lib, n)), None)
        set_ = next((getattr(lib, n) for n in _BLAS_SET if hasattr(lib, n)), None)
        if get is not None and set_ is not None:
            get.restype = ctypes.c_int
            set_.argtypes = [ctypes.c_int]
            out.append((get, set_))
    return out


def _blas_threads():
    libs = _blas_libs()
    if libs:
        return max(int(g()) for g, _ in libs)
    return os.cpu_count()


class OracleRun:
    """The FP64 oracle on a workload, from the same start as the GPU arm: the propagator of
    Algorithm 1 (H update in the Delta-V form H_core + h^3 Phi^T diag(V) Phi -- the form the
    GPU path computes; the oracle's full grid apply gives the same H up to rounding), the
    kicked replicas, and timers for whole time steps and single SCF passes."""

    def __init__(self, name):
        from oracle import hamiltonian as oham, tddft
        self.tddft = tddft
        s, raw = _system(name)
        w = WORKLOADS[name]
        self.s = s
        t0 = time.perf_counter()
        phi = oham.orthonormalize(s, raw)
        del raw
        self.pr = tddft.Propagator(s, phi, tddft.Options(
            dt=s.dt, H_thrs=BENCH_THRESHOLDS["H_thrs"], dP_thrs=BENCH_THRESHOLDS["dP_thrs"],
            poisson_tol=BENCH_THRESHOLDS["poisson_tol"], full_apply=False))
        st0 = self.pr.initial_state(w["subspace_scf"])
        self.states = []
        for a in w["axes"]:
            st = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in st0.items()}
            st["P0"] = self.pr.kick(st["P0"], a, s.kappa)
            self.states.append(st)
        self.setup_s = time.perf_counter() - t0
        self.passes = []

    def steps(self, budget_s, max_steps):
        """Whole time steps (every replica advanced once), timed one by one until max_steps
        or the budget is used (at least one)."""
        times = []
        t_start = time.perf_counter()
        while len(times) < max_steps:
            t1 = time.perf_counter()
            for st in self.states:
                self.passes.append(self.pr.step(st)["passes"])
            times.append(time.perf_counter() - t1)
            if time.perf_counter() - t_start > budget_s:
                break
        return times

    def one_pass(self):
        """Seconds of one SCF pass of replica 0 (commutator series + DFT evaluation)."""
        st = self.states[0]
        Hbar = 0.5 * (st["H0"] + (2.0 * st["H0"] - st["Hm1"]))
        t1 = time.perf_counter()
        P1, _ = self.pr.expand(st["P0"], Hbar, self.s.dt)
        self.pr.dft(P1)
        return time.perf_counter() - t1


def run_reference(args):
    """The reference arm: the FP64 CPU oracle on the headline workload and from the same
    initial state, on the host cores.  Each timed step is one whole time step (every replica,
    SCF passes included); steps are timed until --steps or a wall-clock budget is reached, and
    the line reports the measured mean."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    name = args.workload
    orc = OracleRun(name)
    s = orc.s
    w_times = orc.steps(REF_BUDGET_S, args.warmup + args.steps)
    nw = min(args.warmup, len(w_times) - 1)
    timed = w_times[nw:]
    mean = statistics.mean(timed)
    value = 1.0 / mean
    cores = _blas_threads()
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
           "n_gpus": args.gpus, "steps": len(timed), "warmup": nw,
           "ms_per_step": mean * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": _config(name, s, "fp64-cpu-oracle"),
           "grid_point_orbital_updates_per_s": value * s.Ng * s.N * WORKLOADS[name]["nrep"],
           "same_config": True,
           "scf_passes_per_replica_step": float(np.mean(orc.passes)) if orc.passes else None,
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "host": _host_info(), "setup_s": orc.setup_s,
                            "sample": f"{len(timed)} whole time step(s) of the workload timed "
                                      f"(requested {args.steps} after {args.warmup} warm-up; "
                                      f"wall-clock budget {REF_BUDGET_S:.0f} s)"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def cpu_baseline_sample(name):
    """The oracle timed on the host cores on a bounded sample of the headline workload:
    whole time steps with all BLAS threads (about 30 s), and one SCF pass with one thread,
    scaled by the passes per step of the first measurement."""
    orc = OracleRun(name)
    times = orc.steps(CPU_BASELINE_BUDGET_S, 3)
    out = {"value": 1.0 / statistics.mean(times), "unit": UNIT, "cores": _blas_threads(),
           "kind": "oracle", "host": _host_info(), "setup_s": orc.setup_s,
           "sample": f"{len(times)} whole time step(s) of the workload from the GPU arm's start "
                     f"(budget {CPU_BASELINE_BUDGET_S:.0f} s)"}
    passes = float(np.mean(orc.passes)) * len(orc.states)
    libs = _blas_libs()
    if not libs:
        out["one_thread"] = {"unavailable": "no OpenBLAS thread control found in this process"}
        return out
    before = [int(g()) for g, _ in libs]
    try:
        for _, set_ in libs:
            set_(1)
        t1 = orc.one_pass()
    finally:
        for (_, set_), n in zip(libs, before):
            set_(n)
    out["one_thread"] = {"value": 1.0 / (t1 * passes), "cores": 1,
                         "sample": f"one SCF pass with BLAS on 1 thread, x {passes:.2f} "
                                   "passes per time step (all replicas) of the first "
                                   "measurement"}
    return out


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



def _phase_work(s, mixed, rep_passes, terms_total, h_solves, h_iters, precond):
    """Algorithmic work of each phase over the profiled region: flops, bytes and the peak
    that bounds it (the roofline's numerators)."""
    N, Ng = s.N, s.Ng
    sv = 4 if mixed else 8
    # the two contractions read the orbitals once (bfloat16 hi + lo planes, 4 B per value on
    # the mixed path; float64 on the other) and a grid array (drho written / dV read)
    orb_b = (4 if mixed else 8) * N * Ng + sv * Ng
    return {
        # rho = sum_ij S_ij phi_i phi_j with S symmetric: N(N+1)/2 multiply-adds per point
        "rho": {"flops": float(rep_passes) * Ng * N * (N + 1), "bytes": float(rep_passes) * orb_b},
        # H_ij = h^3 sum_g phi_i V phi_j, j >= i: N(N+1)/2 multiply-adds per point (+ V)
        "hupdate": {"flops": float(rep_passes) * Ng * (N * (N + 1) + N),
                    "bytes": float(rep_passes) * orb_b},
        # two N x N x N products per commutator term (float64)
        "eldyn": {"flops": float(terms_total) * 4.0 * N ** 3, "bytes": 0.0},
        "hartree": {"flops": 0.0, "bytes": hartree_bytes(s.n, h_solves, h_iters, mixed,
                                                         precond)},
    }


def _roofline_entry(phase, work, ms, calls, mixed, peaks, peak_kind):
    """Fraction of the phase's roofline: the larger of its HBM time (algorithmic bytes at the
    measured copy bandwidth) and its arithmetic time (tensor pipe for the mixed contractions,
    float64 ALU otherwise), over the measured time."""
    t = ms * 1e-3
    hbm = work["bytes"] / t / 1e9
    hbm_frac = hbm / peaks["hbm_gbs"]
    e = {"phase": phase, "ms_per_call": ms / max(calls, 1), "calls": calls,
         "hbm_gbs": hbm, "hbm_frac": hbm_frac,
         "algorithmic_bytes_per_call": work["bytes"] / max(calls, 1)}
    if phase in ("rho", "hupdate") and mixed:
        useful = work["flops"] / t / 1e12
        pipe = 3.0 * useful      # hi*hi + hi*lo + lo*hi: three bfloat16 products per product
        peak = peaks["bf16_tflops_sustained"]
        e.update({"tensor_tflops_useful": useful, "tensor_tflops_pipe": pipe,
                  "tensor_peak": peak, "tensor_frac": pipe / peak,
                  "tensor_peak_source": f"{peak_kind} bf16_tflops_sustained (the kernels run "
                                        "inside a long step); 3 split products per product"})
        if pipe / peak > hbm_frac:
            e.update({"bound": "tensor", "achieved": pipe, "peak": peak, "unit": "TFLOP/s",
                      "frac": pipe / peak})
        else:
            e.update({"bound": "hbm", "achieved": hbm, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                      "frac": hbm_frac})
    elif phase in ("rho", "hupdate", "eldyn"):
        alu = work["flops"] / t / 1e12
        e.update({"bound": "alu", "achieved": alu, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                  "frac": alu / FP64_PEAK_TFLOPS,
                  "peak_source": "GB300 float64 rate, nominal 1.25 TFLOP/s"})
    else:
        e.update({"bound": "hbm", "achieved": hbm, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                  "frac": hbm_frac})
    return e


KERNELS = {("rho", True): "k_rho_planes", ("hupdate", True): "k_gram_planes",
           ("hartree", True): "k_hartree_coop", ("eldyn", True): "k_eldyn",
           ("rho", False): "k_rho", ("hupdate", False): "k_gram_partial",
           ("hartree", False): "k_hartree_coop", ("eldyn", False): "k_eldyn"}


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

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB
    stream = torch.cuda.current_stream()
    prec = rmgtd.PREC_MIXED if args.precision == "mixed" else rmgtd.PREC_FP64
    other = rmgtd.PREC_FP64 if prec == rmgtd.PREC_MIXED else rmgtd.PREC_MIXED
    pname = {rmgtd.PREC_MIXED: "mixed", rmgtd.PREC_FP64: "fp64"}

    def measure(name, nsteps, warmup, with_clocks, want_profile=True, want_accuracy=True,
                want_other=True):
        s, raw = _system(name)
        w = WORKLOADS[name]
        nrep = w["nrep"]
        kw = dict(nrep=nrep, subspace_scf=w["subspace_scf"], **BENCH_THRESHOLDS)

        def make(p, graph=True):
            c = rmgtd.Context(s, raw, use_graph=graph, precision=p, **kw)
            for r, a in enumerate(w["axes"]):
                c.kick(r, a, s.kappa)
            return c

        def timed_steps(ctx, n, profile, tag):
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(n)]
            if profile:
                ctx.profile(True)
            if world > 1:
                dist.barrier()
            torch.cuda.synchronize()
            w0 = time.perf_counter()
            st = []
            torch.cuda.nvtx.range_push(tag)
            for i in range(n):
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

        def run_path(p, clocks, state=None, net=None):
            c = make(p) if state is None else rmgtd.Context(s, raw, use_graph=True, precision=p,
                                                             **kw)
            if state is not None:
                c.load(state)
            if net is not None:
                c.attach_net(net)
            for _ in range(warmup):
                c.step(1)
            smp = ClockSampler(local)
            if clocks:
                smp.start()
            ms, stt, wl, prof = timed_steps(c, nsteps, True,
                                            "rmgtd_timed" if clocks else "rmgtd_other")
            clk = smp.stop() if clocks else None
            c.close()
            tot = max_over_ranks(float(sum(ms)), world)
            return tot, stt, wl, prof[2], clk

        res = {"s": s, "raw": raw, "make": make, "run_path": run_path, "timed_steps": timed_steps}
        total_ms, st, wall, launches, clocks = run_path(prec, with_clocks)
        res.update(total_ms=total_ms, st=st, wall=wall, launches=launches, clocks=clocks,
                   value=job_throughput(nsteps, world, total_ms),
                   passes=float(st["passes"].sum()) / (nrep * nsteps),
                   terms=float(st["terms_sum"].sum()) / max(float(st["passes"].sum()), 1.0))
        if want_other:
            o_ms, o_st, _, _, _ = run_path(other, False)
            res["other_path"] = {"precision": pname[other],
                                 "value": job_throughput(nsteps, world, o_ms), "unit": UNIT,
                                 "ms_per_step": o_ms / nsteps,
                                 "scf_passes_per_replica_step":
                                     float(o_st["passes"].sum()) / (nrep * nsteps)}
        if want_accuracy:
            g = _golden(name)
            last = g["replicas"][0].get("step", [len(g["replicas"][0]["dipole"]) - 1])[-1]
            every = 1
            st_list = g["replicas"][0].get("step")
            if st_list and len(st_list) > 1:
                every = st_list[1] - st_list[0]
            acc, dip = {}, {}
            for p in (prec, other):
                c = make(p)
                d, e, t = trajectory_observables(c, nrep, last, every)
                c.close()
                acc[pname[p]] = accuracy_against_oracle(d, e, t, g, last)
                dip[p] = d
            # the two GPU paths at the same thresholds: the precision's own share of the error
            worst = 0.0
            for a, tr in enumerate(g["replicas"]):
                ref = np.array(tr["dipole"])
                scale = np.max(np.abs(ref - ref[0]))
                diff = max(float(np.max(np.abs(np.array(dip[prec][k][a]) - np.array(dip[other][k][a]))))
                           for k in dip[prec])
                worst = max(worst, diff / scale)
            acc["mixed_vs_fp64_gpu_dipole_rel"] = worst
            res["accuracy"] = acc
        if want_profile:
            pctx = make(prec, graph=False)
            for _ in range(warmup):
                pctx.step(1)
            p_ms, p_st, _, (phase_ms, phase_calls, _) = timed_steps(pctx, nsteps, True,
                                                                    "rmgtd_host_driven")
            h_solves, h_iters = pctx.profile_counters()
            precond = "dst" if pctx.hartree_preconditioner() == rmgtd.PRECOND_DST else "mg"
            pctx.close()
            res.update(phase_ms=phase_ms, phase_calls=phase_calls, p_ms=p_ms, p_st=p_st,
                       h_solves=h_solves, h_iters=h_iters, precond=precond)
        return res

    name = args.workload
    w = WORKLOADS[name]
    K, W = args.steps, args.warmup
    m = measure(name, K, W, True)
    s = m["s"]
    mixed = prec == rmgtd.PREC_MIXED
    peaks, peak_kind = _peaks()
    rep_passes = int(m["p_st"]["passes"].sum())
    terms = int(m["p_st"]["terms_sum"].sum())
    work = _phase_work(s, mixed, rep_passes, terms, m["h_solves"], m["h_iters"], m["precond"])
    phases = {}
    for ph in ("rho", "hupdate", "eldyn", "hartree"):
        if m["phase_ms"].get(ph, 0) > 0:
            phases[ph] = _roofline_entry(ph, work[ph], m["phase_ms"][ph], m["phase_calls"][ph],
                                         mixed, peaks, peak_kind)
            phases[ph]["kernel"] = KERNELS[(ph, mixed)]
    dom = max(phases, key=lambda k: m["phase_ms"][k])
    roof = dict(phases[dom])
    roof["dominant_phase"] = dom
    roof["traffic"] = _traffic(roof["kernel"], name) if mixed else None
    roof["traffic_source"] = (f"ncu dram__bytes_read.sum + dram__bytes_write.sum per launch "
                              f"(profiles/traffic_{roof['kernel']}_{name}.txt), null unless "
                              "taken on the kernel's current source")
    roof["timing"] = ("CUDA events on the library stream around each phase, host-driven steps "
                      "of the same workload (second timed region); a phase includes its small "
                      "helper launches")
    if dom == "hartree":
        roof["cg_iterations_per_solve"] = m["h_iters"] / max(m["h_solves"], 1)
        roof["preconditioner"] = m["precond"]
    roof["peak_source"] = f"{peak_kind} MEASURED_PEAKS.json"
    roof["other_phases"] = {k: v for k, v in phases.items() if k != dom}

    result = {
        "metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": m["total_ms"] / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16x3+f32+f64" if mixed else "f64", "data": "synthetic",
        "config": _config(name, s, args.precision),
        "grid_point_orbital_updates_per_s": m["value"] * s.Ng * s.N * w["nrep"],
        "scf_passes_per_replica_step": m["passes"],
        "commutator_terms_per_expansion": m["terms"],
        "accuracy": m["accuracy"],
        "other_path": m["other_path"],
        "phase_ms_per_step_host_driven": {k: v / K for k, v in m["phase_ms"].items()},
        "ms_per_step_host_driven": float(sum(m["p_ms"])) / K,
        "gpu_launches": m["launches"], "roofline": roof, "clocks": m["clocks"],
        "wall_s_timed_region": m["wall"],
    }

    # end to end through the public API: context from host orbitals, kicks, the workload's
    # trajectory length with every replica's dipole read back after every step
    torch.cuda.synchronize()
    nsteps_e2e = w["trajectory_steps"]
    t0 = time.perf_counter()
    c2 = m["make"](prec)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    dip = np.empty((nsteps_e2e + 1, w["nrep"], 3))
    for r in range(w["nrep"]):
        dip[0, r] = c2.dipole(r)
    for k in range(nsteps_e2e):
        c2.step(1, stats=False)
        for r in range(w["nrep"]):
            dip[k + 1, r] = c2.dipole(r)
    # the absorption spectrum of the kicked runs (each run's dipole along its kick)
    t_sp = time.perf_counter()
    d_kick = np.array([dip[:, r, w["axes"][r]] for r in range(w["nrep"])])
    omega = np.linspace(0.0, 1.0, SPECTRUM_POINTS)
    spec = rmgtd.spectrum(d_kick, s.dt, s.kappa, SPECTRUM_DAMPING, omega)
    spectrum_s = time.perf_counter() - t_sp
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    c2.close()
    h2d = m["raw"].nbytes + s.pos.nbytes * 3
    result["e2e"] = {"value": world * nsteps_e2e / e2e_s, "unit": UNIT,
                     "h2d_bytes_per_step": h2d / nsteps_e2e,
                     "d2h_bytes_per_step": 24 * w["nrep"],
                     "steps": nsteps_e2e, "setup_s": t_setup,
                     "steady_state_steps_per_s": nsteps_e2e / max(e2e_s - t_setup, 1e-9),
                     "includes": "context creation from host orbitals (upload, set-up), the "
                                 "kick(s), the workload's trajectory with the dipole of every "
                                 "replica read back after every step, and the absorption "
                                 "spectrum of the kicked dipoles (rmgtd_spectrum)",
                     "spectrum": {"frequencies": SPECTRUM_POINTS, "omega_max_ha": 1.0,
                                  "damping_ha": SPECTRUM_DAMPING, "seconds": spectrum_s,
                                  "finite": bool(np.all(np.isfinite(spec))),
                                  "note": "the icosahedron starts far from its ground state "
                                          "(P_0 = diag(f) of seeded orbitals), so this is the "
                                          "pipeline's cost, not a physical spectrum"}}
    if not args.no_grid_basis:
        result["grid_basis_path"] = _grid_basis_path(rmgtd, peaks)

    # secondary line: the ring workload, with the learned seed's comparison
    if name == "icosa" and not args.no_ring:
        r = measure("ring", max(K, 40), W, False, want_profile=False)
        ring = {"workload": WORKLOADS["ring"]["label"], "value": r["value"], "unit": UNIT,
                "ms_per_step": r["total_ms"] / max(K, 40), "steps": max(K, 40),
                "scf_passes_per_replica_step": r["passes"], "other_path": r["other_path"],
                "accuracy": r["accuracy"],
                "grid_point_orbital_updates_per_s": r["value"] * r["s"].Ng * r["s"].N * 3}
        if mixed and not args.no_surrogate:
            ring["surrogate_path"] = _surrogate_path(rmgtd, r, max(K, 40), world)
        result["ring_workload"] = ring
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline_sample(name)
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result), flush=True)
    return 0


def _grid_basis_path(rmgtd, peaks):
    """Secondary line: the occupied orbitals propagated on the grid (the complete-grid-basis
    limit) on the ring, kicked along x, y, z, both precisions; the series phase rated as the
    term kernel's algorithmic bytes (term read and write, and the running sum read and written
    per point and orbital) over its time."""
    import torch
    s, raw = _system("ring")
    s = dataclasses.replace(s, nvirt=0)
    raw = raw[:s.N]
    out = {"workload": "ring-12-atoms-64^3-15-occupied-orbitals-on-the-grid-kicks-xyz"}
    for name, prec in (("mixed", rmgtd.PREC_MIXED), ("fp64", rmgtd.PREC_FP64)):
        ctx = rmgtd.Context(s, raw, nrep=3, H_thrs=1e-7 if name == "fp64" else 1e-6,
                            dP_thrs=1e-10, poisson_tol=1e-10, precision=prec, grid_basis=True)
        for a in range(3):
            ctx.kick(a, a, s.kappa)
        ctx.step(GRID_BASIS_WARMUP, stats=False)
        ctx.profile(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = ctx.step(GRID_BASIS_STEPS)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        ph, calls, _ = ctx.profile_read()
        ctx.close()
        terms = float(st["terms_sum"].sum())
        # per point and orbital: the term read and written (2 planes of T) and the running sum
        # read and written (float64: psi_1, 2 planes; mixed: the float32 hi/lo pair, 4 planes)
        per_term = (8 * 8 if name == "fp64" else 8 * 6) * s.Ng * s.N
        series_ms = ph["eldyn"]
        achieved = per_term * terms / (series_ms * 1e-3) / 1e9 if series_ms > 0 else None
        out[name] = {"value": GRID_BASIS_STEPS / wall, "unit": UNIT,
                     "ms_per_step": wall / GRID_BASIS_STEPS * 1e3,
                     "scf_passes_per_replica_step": float(st["passes"].mean()),
                     "series_terms_per_replica_pass": terms / max(float(st["passes"].sum()), 1.0),
                     "series_ms_per_step": series_ms / GRID_BASIS_STEPS,
                     "series_hbm_gbs": achieved,
                     "series_hbm_frac": achieved / peaks["hbm_gbs"] if achieved else None,
                     "bytes_per_term_and_replica": per_term}
    out["note"] = ("series phase = KB projections + fused TMA term kernel + the device-side "
                   "stopping test (terms queued in batches between read-backs) + the fold of "
                   "the float32 sum; H_thrs above each path's floor (1e-7 float64, 1e-6 "
                   "mixed: the float32 terms leave ~1e-8 of noise in V)")
    return out


def _surrogate_path(rmgtd, r, nsteps, world):
    """The mixed path with the learned SCF seed on the ring: a network trained (library
    kernels only) on the first SUR_STEPS steps of the workload's own trajectory, then the
    continuation timed with and without it from the same state (a window the network has
    not seen)."""
    from paper_2410_09189_gb300 import surrogate
    tctx = r["make"](rmgtd.PREC_MIXED)
    t0 = time.perf_counter()
    net, rep = surrogate.train_on_trajectory(tctx, nsteps=SUR_STEPS, iters=SUR_ITERS, batch=8,
                                             lr=5e-4)
    train_s = time.perf_counter() - t0
    state = os.path.join(tempfile.mkdtemp(), "state.bin")
    tctx.save(state)
    tctx.close()
    p_ms, p_st, _, _, _ = r["run_path"](rmgtd.PREC_MIXED, False, state=state)
    n_ms, n_st, _, _, _ = r["run_path"](rmgtd.PREC_MIXED, False, state=state, net=net)
    return {
        "value": world * nsteps / (n_ms * 1e-3), "unit": UNIT, "ms_per_step": n_ms / nsteps,
        "scf_passes_per_replica_step": float(n_st["passes"].sum()) / (3.0 * nsteps),
        "same_window_without_seed": {
            "value": world * nsteps / (p_ms * 1e-3), "ms_per_step": p_ms / nsteps,
            "scf_passes_per_replica_step": float(p_st["passes"].sum()) / (3.0 * nsteps)},
        "window": f"{nsteps} steps after step {SUR_STEPS} (+ warm-up) of the kicked trajectory",
        "training": {"trajectory_steps": SUR_STEPS, "adam_iterations": SUR_ITERS, "batch": 8,
                     "lr": 5e-4, "seconds_incl_recording": train_s,
                     "heldout_seed_rms_ratio": rep["heldout_ratio"],
                     "samples": rep["train_samples"]}}


def run_batch8(args):
    """The batched workload: eight clusters (20-150 atoms, 48^3-96^3), three kicks each,
    stepped by one CUDA graph per time step (rmgtd_batch, the clusters back to back: the
    line's value), against the contexts stepped one after another and against the graph with
    every cluster on its own share of the SMs on a parallel branch (shares in proportion to
    the clusters' solo step times); mixed path, launch configurations from the autotuner; all
    variants step the same window of the trajectory."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2410_09189_gb300 import inputs, rmgtd

    systems = [inputs.cluster(i) for i in range(8)]
    n_sms = torch.cuda.get_device_properties(0).multi_processor_count

    def make(budget=None):
        out = []
        for i, s in enumerate(systems):
            raw = inputs.smooth_random_orbitals(s).reshape(s.N, s.Ng)
            c = rmgtd.Context(s, raw, nrep=3, H_thrs=1e-7, dP_thrs=1e-10, poisson_tol=1e-10,
                              precision=rmgtd.PREC_MIXED, use_graph=True,
                              sm_budget=0 if budget is None else int(budget[i]))
            for a in range(3):
                c.kick(a, a, 1e-3)
            out.append(c)
        return out

    t0 = time.perf_counter()
    ctxs = make()
    setup_s = time.perf_counter() - t0
    choices = [c.autotune() for c in ctxs]
    stream = torch.cuda.current_stream()
    # SM budgets of the concurrent variant: shares of the SMs in proportion to each cluster's
    # own step time on the whole GPU (at least 4 SMs), summing to at most the SM count --
    # latency-bound small systems lose little on few SMs, bandwidth-bound large ones need many
    solo_ms = []
    for c in ctxs:
        c.step(2)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c.step(5)
        e1.record(stream)
        torch.cuda.synchronize()
        solo_ms.append(e0.elapsed_time(e1) / 5)
    work = np.array(solo_ms)
    budgets = np.maximum(4, np.floor(n_sms * work / work.sum())).astype(int)
    while budgets.sum() > n_sms:
        budgets[int(np.argmax(budgets))] -= 1

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
    passes = float(np.mean([st["passes"].mean() for st in bat_st]))
    for c in ctxs:
        c.close()
    # the concurrent variant: the same states in contexts sized to their SM budgets, one graph
    # per step with a parallel branch per cluster
    t0 = time.perf_counter()
    cctx = make(budgets)
    setup_c = time.perf_counter() - t0
    cchoices = [c.autotune() for c in cctx]
    for c, pth in zip(cctx, paths):
        c.load(pth)
    cbatch = rmgtd.Batch(cctx)
    con_ms, con_st = timed(lambda k: cbatch.step(k))
    cbatch.close()
    con_passes = float(np.mean([st["passes"].mean() for st in con_st]))
    for c in cctx:
        c.close()
    for pth in paths:
        os.remove(pth)
    os.rmdir(tmpdir)
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
           "concurrent_sm_budgets": {"value": args.steps / (con_ms * 1e-3),
                                     "ms_per_step": con_ms / args.steps,
                                     "sm_budgets": [int(b) for b in budgets],
                                     "solo_ms_per_step_whole_gpu": solo_ms,
                                     "scf_passes_per_replica_step": con_passes,
                                     "setup_s": setup_c, "autotune_choices": cchoices},
           "one_graph_per_step_back_to_back": {"value": args.steps / (bat_ms * 1e-3),
                                               "ms_per_step": bat_ms / args.steps},
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
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="icosa", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ring", action="store_true", help="skip the secondary ring line")
    ap.add_argument("--no-grid-basis", action="store_true",
                    help="skip the grid-basis propagation line")
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
