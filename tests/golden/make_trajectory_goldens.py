"""Write the stored oracle trajectories the full-size GPU parity tests compare against.

Calls only ``oracle/`` (and the seeded input generators of ``inputs``); no value here comes
from the CUDA path.  Each golden is one JSON file beside this script:

* ``ring64_three_kicks.json`` -- the 12-atom ring on its 64^3 grid (N = 30), started from
  the ground state inside the orbital block (``Propagator.subspace_ground_state``), then
  three replicas kicked along x, y and z (kappa = 1e-3, Eq. 34 with a delta envelope) and
  propagated by Algorithm 1 for 2,000 steps of dt = 0.05; every fifth step is stored.
* ``icosa128_window.json`` -- the 147-atom icosahedron on its 128^3 grid (N = 148), started
  from P_0 = diag(f) of the orthonormalised seeded orbitals, kicked along z and propagated
  for a 64-step window.
* ``ring64_grid_basis.json`` -- the ring's 15 occupied orbitals propagated on its 64^3 grid
  (the complete-grid-basis limit, ``oracle/gridprop.py``), from the orthonormalised first 15
  seeded orbitals, kicked along z, 20 steps, every step stored.

Both use the Delta-V form of the Hamiltonian update, H = H_core + h^3 Phi^T diag(V_H + V_xc)
Phi, which equals the full grid apply of Algorithm 1's H update up to rounding (pinned in
``tests/test_oracle_propagation.py``); it saves the oracle the 37-point stencil on every
orbital in every pass.  Thresholds are tighter than the benchmark's so that the stored series
sits well inside the tolerance of the tests that read it.

Usage: ``python tests/golden/make_trajectory_goldens.py ring|icosa|grid`` (minutes to an
hour of CPU time each).
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import gridprop, hamiltonian as oham, tddft  # noqa: E402
from paper_2410_09189_gb300 import inputs  # noqa: E402

RING = dict(name="ring64_three_kicks", nsteps=2000, record_every=5, H_thrs=1e-10, dP_thrs=1e-12,
            poisson_tol=1e-12, subspace_scf=600, subspace_mix=0.3, subspace_tol=1e-12)
ICOSA = dict(name="icosa128_window", nsteps=64, record_every=1, H_thrs=1e-10, dP_thrs=1e-13,
             poisson_tol=1e-12)
GRID = dict(name="ring64_grid_basis", nsteps=20, axis=2, H_thrs=1e-10, dP_thrs=1e-12,
            poisson_tol=1e-12)


def make_grid():
    """The ring's occupied orbitals propagated on the grid (oracle/gridprop.py)."""
    import dataclasses
    cfg = GRID
    s0 = inputs.ring()
    s = dataclasses.replace(s0, nvirt=0)
    raw = inputs.smooth_random_orbitals(s0).reshape(s0.N, s0.Ng)[:s.N]
    psi0 = oham.orthonormalize(s, raw)
    opts = tddft.Options(dt=s.dt, H_thrs=cfg["H_thrs"], dP_thrs=cfg["dP_thrs"],
                         poisson_tol=cfg["poisson_tol"])
    t0 = time.time()
    out = gridprop.run(s, psi0, s.occupations, opts, nsteps=cfg["nsteps"], axis=cfg["axis"],
                       kappa=s.kappa)
    doc = {
        "what": f"oracle grid propagation of the {s.name} workload's occupied orbitals (float64 CPU)",
        "written_by": "tests/golden/make_trajectory_goldens.py (oracle/ only)",
        "workload": {"name": s.name, "grid": list(s.n), "h": s.h, "nocc": s.nocc,
                     "natoms": int(len(s.Z)), "nproj": s.nproj, "dt": s.dt, "kappa": s.kappa,
                     "axis": cfg["axis"]},
        "options": {k: v for k, v in cfg.items() if k != "name"},
        "initial_state": "the orthonormalised first nocc seeded orbitals",
        "step": list(range(cfg["nsteps"] + 1)),
        "dipole": out["dipole"].tolist(), "energy": out["energy"].tolist(),
        "electrons": out["electrons"].tolist(), "passes": out["passes"],
        "cpu_seconds": time.time() - t0,
    }
    path = os.path.join(HERE, cfg["name"] + ".json")
    with open(path + ".tmp", "w") as f:
        json.dump(doc, f, indent=None, separators=(",", ":"))
    os.replace(path + ".tmp", path)
    print(f"wrote {path}", flush=True)


def _trajectory(pr, st0, axis, kappa, nsteps, every, log):
    st = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in st0.items()}
    st["P0"] = pr.kick(st["P0"], axis, kappa)
    _, aux0 = pr.dft(st["P0"])
    out = {"step": [0], "dipole": [pr.dipole(st["P0"]).tolist()],
           "energy": [pr.energy(st["P0"], aux0)], "trace": [float(np.real(np.trace(st["P0"])))],
           "passes": []}
    t0 = time.time()
    for j in range(nsteps):
        s = pr.step(st)
        out["passes"].append(int(s["passes"]))
        if (j + 1) % every == 0 or j + 1 == nsteps:
            out["step"].append(j + 1)
            out["dipole"].append(pr.dipole(st["P0"]).tolist())
            out["energy"].append(pr.energy(st["P0"], st["aux"]))
            out["trace"].append(float(np.real(np.trace(st["P0"]))))
            log(f"axis {axis} step {j + 1}/{nsteps} passes {s['passes']} "
                f"d={out['dipole'][-1]} {time.time() - t0:.0f}s")
    return out


def make(which: str):
    log = lambda m: print(m, flush=True)  # noqa: E731
    if which == "ring":
        cfg = RING
        s = inputs.ring()
        axes = (0, 1, 2)
    else:
        cfg = ICOSA
        s = inputs.icosa()
        axes = (2,)
    raw = inputs.smooth_random_orbitals(s).reshape(s.N, s.Ng)
    phi = oham.orthonormalize(s, raw)
    del raw
    opts = tddft.Options(dt=s.dt, H_thrs=cfg["H_thrs"], dP_thrs=cfg["dP_thrs"],
                         poisson_tol=cfg["poisson_tol"], full_apply=False)
    pr = tddft.Propagator(s, phi, opts)
    t0 = time.time()
    if cfg.get("subspace_scf"):
        P, H, aux, iters, err = pr.subspace_ground_state(cfg["subspace_scf"], cfg["subspace_mix"],
                                                         cfg["subspace_tol"])
        log(f"subspace ground state: {iters} iterations, last change {err:.3e}, "
            f"{time.time() - t0:.0f}s")
        st0 = {"P0": P.astype(np.complex128), "H0": H, "Hm1": H.copy(), "aux": aux,
               "t": 0.0, "j": 0}
        gs = {"iterations": int(iters), "last_change": float(err)}
    else:
        st0 = pr.initial_state()
        gs = None
    doc = {
        "what": f"oracle trajectory of the {s.name} workload (Algorithm 1, float64 CPU)",
        "written_by": "tests/golden/make_trajectory_goldens.py (oracle/ only)",
        "workload": {"name": s.name, "grid": list(s.n), "h": s.h, "N": s.N, "nocc": s.nocc,
                     "natoms": int(len(s.Z)), "nproj": s.nproj, "dt": s.dt,
                     "kappa": s.kappa, "kick_axes": list(axes)},
        "options": {k: v for k, v in cfg.items() if k != "name"},
        "hamiltonian_update": "Delta-V form H_core + h^3 Phi^T diag(V_H+V_xc) Phi",
        "initial_state": ("ground state inside the orbital block" if gs else
                          "P_0 = diag(f) of the orthonormalised seeded orbitals"),
        "subspace_ground_state": gs,
        "dipole_gs": pr.dipole(st0["P0"]).tolist(),
        "energy_gs": pr.energy(st0["P0"], st0["aux"]),
        "replicas": [],
    }
    for a in axes:
        tr = _trajectory(pr, st0, a, s.kappa, cfg["nsteps"], cfg["record_every"], log)
        tr["axis"] = a
        doc["replicas"].append(tr)
    doc["cpu_seconds"] = time.time() - t0
    path = os.path.join(HERE, cfg["name"] + ".json")
    with open(path + ".tmp", "w") as f:
        json.dump(doc, f, indent=None, separators=(",", ":"))
    os.replace(path + ".tmp", path)
    log(f"wrote {path}")


if __name__ == "__main__":
    which = sys.argv[1] if len(sys.argv) > 1 else "ring"
    make_grid() if which == "grid" else make(which)
