"""Pins of the oracle's ground-state SCF (the orbitals that define the active space).

The oracle finds the lowest eigenpairs with ARPACK's Lanczos iteration inside a Pulay-mixed
density loop.  On a 9 x 8 x 8 grid (576 points, a KB projector) the whole grid Hamiltonian
fits in a dense matrix, so each claim is checked against a dense LAPACK diagonalisation:

* independent electrons: the eigenvalues and the occupied projector sum_i f_i |phi_i><phi_i|
  equal those of the dense matrix, the orbitals are grid-normalised (h^3 phi.phi = 1) with
  the stated sign convention;
* with Hartree and LDA exchange-correlation: the returned density is a fixed point of the
  Kohn-Sham map -- the N lowest dense eigenvectors of H[rho] rebuild rho -- and the returned
  orbitals are eigenvectors of H[rho];
* the Kohn-Sham energy is stationary and minimal at the returned orbitals: rotating an
  occupied orbital into a virtual one by +-theta raises it by (eps_v - eps_o) f theta^2 to
  leading order, with no first-order change.

A wrong normalisation, occupation, density formula, mixing that stops away from the fixed
point, or a missed eigenpair fails one of them.
"""
import dataclasses

import numpy as np
import pytest

from oracle import gridprop, groundstate, hamiltonian as ham, tddft
from oracle.lda import lda
from oracle.poisson import hartree
from paper_2410_09189_gb300 import inputs


def _tiny(hartree_xc: bool, nvirt: int = 3):
    s0 = inputs.small()
    return dataclasses.replace(s0, n=(9, 8, 8), h=0.5, nvirt=nvirt, hartree_xc=hartree_xc,
                               proj_atom=np.array([1]), proj_l=np.array([0]),
                               proj_m=np.array([0]), proj_rc=np.array([0.7]),
                               E_kb=np.array([0.8]))


def _dense_h(s, v_total):
    Hd = ham.apply_h(s, v_total, np.eye(s.Ng), ham.projectors(s))
    assert np.max(np.abs(Hd - Hd.T)) < 1e-10 * np.max(np.abs(Hd))
    return 0.5 * (Hd + Hd.T)


def _v_ion(s):
    return (ham.v_local(s) + ham.v_external(s)).ravel()


def test_independent_electrons_match_dense_diagonalisation():
    s = _tiny(hartree_xc=False)
    gs = groundstate.ground_state(s)
    w, W = np.linalg.eigh(_dense_h(s, _v_ion(s)))
    assert np.max(np.abs(gs["eps"] - w[:s.N])) < 1e-9
    phi = gs["phi"]
    h3 = s.h ** 3
    assert np.max(np.abs(h3 * phi @ phi.T - np.eye(s.N))) < 1e-10
    # the occupied projector (independent of the eigenvectors' phases)
    f = s.occupations
    P = (f[:, None] * phi).T @ phi * h3
    Wo = W[:, :s.N]
    Pd = (f[None, :] * Wo) @ Wo.T
    assert np.max(np.abs(P - Pd)) < 1e-8
    # each orbital of a simple eigenvalue is the dense eigenvector up to its sign, and the
    # sign puts a largest-magnitude value positive (ties between mirror points of an odd
    # orbital make the choice of point, not the convention, arbitrary)
    for i in range(s.N):
        gap = min(abs(w[i] - w[j]) for j in range(s.N + 1) if j != i)
        if gap > 1e-6:
            assert abs(abs(s.h ** 1.5 * phi[i] @ W[:, i]) - 1.0) < 1e-10
        assert phi[i][np.argmax(np.abs(phi[i]))] > 0
    assert np.allclose(gs["rho"], (f[:, None] * phi * phi).sum(0), atol=1e-14)


def test_scf_density_is_a_fixed_point_of_the_kohn_sham_map():
    s = _tiny(hartree_xc=True)
    gs = groundstate.ground_state(s, tol=1e-11)
    rho = gs["rho"]
    assert abs(s.h ** 3 * rho.sum() - 2.0 * s.nocc) < 1e-9
    shape = (s.n[2], s.n[1], s.n[0])
    vh = hartree(s, rho.reshape(shape), tol=1e-14).ravel()
    vxc, _ = lda(rho)
    v = _v_ion(s) + vh + vxc
    w, W = np.linalg.eigh(_dense_h(s, v))
    f = s.occupations
    rho_d = (f[None, :] * W[:, :s.N] ** 2).sum(1) / s.h ** 3
    assert np.max(np.abs(rho_d - rho)) < 1e-8 * np.max(rho)
    assert np.max(np.abs(gs["eps"] - w[:s.N])) < 1e-8
    # the returned orbitals are eigenvectors of H[rho] with the returned eigenvalues
    hphi = ham.apply_h(s, v, gs["phi"], ham.projectors(s))
    res = hphi - gs["eps"][:, None] * gs["phi"]
    assert np.max(np.abs(res)) < 1e-6 * np.max(np.abs(hphi))
    # a density that is not the fixed point fails the same test
    rho_bad = rho * (1.0 + 1e-3 * np.cos(np.arange(s.Ng)))
    vh_b = hartree(s, rho_bad.reshape(shape), tol=1e-14).ravel()
    w_b, W_b = np.linalg.eigh(_dense_h(s, _v_ion(s) + vh_b + lda(rho_bad)[0]))
    rho_bd = (f[None, :] * W_b[:, :s.N] ** 2).sum(1) / s.h ** 3
    assert np.max(np.abs(rho_bd - rho_bad)) > 1e-6 * np.max(rho)


def test_kohn_sham_energy_is_stationary_and_minimal():
    s = _tiny(hartree_xc=True)
    gs = groundstate.ground_state(s, tol=1e-11)
    phi, eps = gs["phi"], gs["eps"]
    o = tddft.Options(poisson_tol=1e-14)
    occ = s.occupations[:s.nocc]

    def energy(psi):
        return gridprop.GridPropagator(s, psi, occ, o).energy()

    e0 = energy(phi[:s.nocc])
    v = s.nocc   # the lowest virtual orbital
    theta = 2e-3
    ep, em = [], []
    for sgn, out in ((1.0, ep), (-1.0, em)):
        psi = phi[:s.nocc].copy()
        psi[0] = np.cos(theta) * phi[0] + sgn * np.sin(theta) * phi[v]
        out.append(energy(psi))
    curv = ep[0] + em[0] - 2.0 * e0
    assert curv > 0.0
    # second order: f (eps_v - eps_o) theta^2 per side, less the (small) response of the fields
    expect = 2.0 * s.occupations[0] * (eps[v] - eps[0]) * theta ** 2
    assert 0.5 * expect < curv < 1.5 * expect
    # no first-order change: the orbitals make the energy stationary
    assert abs(ep[0] - em[0]) < 1e-3 * curv
