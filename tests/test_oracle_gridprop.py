"""Pins of the oracle's propagation on the grid (the complete-grid-basis limit, Section 2.2).

* On a 9 x 8 x 8 grid, Algorithm 1 with the complete basis -- all 576 eigenvectors of the core
  Hamiltonian as the active space, P_0 = diag(f) -- and the grid propagation of the occupied
  orbital give the same dipoles and energies (the same SCF thresholds; 1e-12 of the dipole's
  variation), with a kick, a KB projector and a field pulse.  A sign or factor error in the
  orbital series, the kick's phase, the field term or the mean potential fails it.
* Orthonormality and the electron count after every step.
"""
import dataclasses
import math

import numpy as np
import pytest

from oracle import gridprop, hamiltonian as ham, tddft
from paper_2410_09189_gb300 import inputs


def _tiny_complete():
    s0 = inputs.small()
    n = (9, 8, 8)
    Ng = n[0] * n[1] * n[2]
    s = dataclasses.replace(s0, n=n, h=0.5, nvirt=Ng - s0.nocc,
                            proj_atom=np.array([1]), proj_l=np.array([0]),
                            proj_m=np.array([0]), proj_rc=np.array([0.7]),
                            E_kb=np.array([0.8]))
    v_ion = (ham.v_local(s) + ham.v_external(s)).ravel()
    Hd = ham.apply_h(s, v_ion, np.eye(Ng), ham.projectors(s))
    w, W = np.linalg.eigh(0.5 * (Hd + Hd.T))
    return s, W.T / s.h ** 1.5


@pytest.fixture(scope="module")
def tiny():
    return _tiny_complete()


def _pulse(t):
    return np.array([0.02 * math.sin(1.3 * t), 0.0, 0.03 * math.exp(-((t - 0.04) / 0.03) ** 2)])


@pytest.mark.parametrize("driving", ["kick", "field"])
def test_grid_propagation_equals_algorithm_1_in_the_complete_basis(tiny, driving):
    s, phi = tiny
    o = tddft.Options(dt=0.02, H_thrs=1e-11, dP_thrs=1e-13, poisson_tol=1e-13)
    kw = dict(axis=2, kappa=0.1) if driving == "kick" else dict(kappa=0.0, field=_pulse)
    ref = tddft.run(s, phi, o, nsteps=4, **kw)
    got = gridprop.run(s, phi[:s.nocc], s.occupations[:s.nocc], o, nsteps=4, **kw)
    scale = np.max(np.abs(ref["dipole"] - ref["dipole"][0]))
    assert scale > 1e-4
    assert np.max(np.abs(got["dipole"] - ref["dipole"])) < 1e-12 * max(scale, 1.0)
    assert np.max(np.abs(got["energy"] - ref["energy"])) < 1e-11
    # (pass counts may differ by one: the element-wise max of H_new - H_1 in the eigenvector
    # basis is not max|V_new - V_1| on the grid)


def test_grid_propagation_keeps_orthonormal_orbitals():
    s = inputs.small()
    raw = inputs.smooth_random_orbitals(s).reshape(s.N, s.Ng)[:3]
    L = np.linalg.cholesky(s.h ** 3 * raw @ raw.T)
    psi0 = np.linalg.solve(L, raw)
    f = np.array([2.0, 2.0, 1.0])
    o = tddft.Options(dt=0.05, H_thrs=1e-10, dP_thrs=1e-12, poisson_tol=1e-12)
    r = gridprop.run(s, psi0, f, o, nsteps=5, axis=0, kappa=0.05, energies=False)
    psi = r["propagator"].psi
    S = s.h ** 3 * psi.conj() @ psi.T
    assert np.max(np.abs(S - np.eye(3))) < 1e-12
    assert np.max(np.abs(r["electrons"] - 5.0)) < 1e-10


def test_stored_grid_trajectory_starts_from_its_recipe():
    """The stored full-size grid-basis run (tests/golden/ring64_grid_basis.json) starts where
    its recipe says: the ring's orthonormalised first 15 seeded orbitals kicked along z; its
    step-0 dipole and energy are the oracle's."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "ring64_grid_basis.json")
    with open(path) as f:
        g = json.load(f)
    s0 = inputs.ring()
    s = dataclasses.replace(s0, nvirt=0)
    raw = inputs.smooth_random_orbitals(s0).reshape(s0.N, s0.Ng)[:s.N]
    psi0 = ham.orthonormalize(s, raw)
    o = g["options"]
    opts = tddft.Options(dt=s.dt, H_thrs=o["H_thrs"], dP_thrs=o["dP_thrs"],
                         poisson_tol=o["poisson_tol"])
    gp = gridprop.GridPropagator(s, psi0, s.occupations, opts)
    gp.kick(g["workload"]["axis"], s.kappa)
    assert np.max(np.abs(gp.dipole() - np.array(g["dipole"][0]))) < 1e-12
    assert abs(gp.energy() - g["energy"][0]) < 1e-9
    assert len(g["dipole"]) == o["nsteps"] + 1
