"""Pins of the oracle's propagation (Algorithm 1) against results fixed by the mathematics.

* Commutator expansion (Eq. 19 / 33) = spectral propagator W exp(omega) W^dagger
  (Section 2.2) = scipy expm, within dP_thrs.
* Harmonic oscillator: eigenvalues (n + 3/2) omega, and the kicked dipole of the
  two-level active space, d_z(t) = -N_e a sin(2 kappa a) sin(omega t), a = (2 omega)^-1/2.
* Tr P conserved, P Hermitian, (P/2)^2 = P/2 for a closed shell.
* Zero-field energy conservation after the kick (Section 4.2: no drift).
* Time-domain TRK sum rule: d'(0+) = -kappa Tr(P_0 [[M,H],M]) -> -kappa N_e (complete basis).
* The two Hamiltonian-update forms (full apply vs H_core + Phi^T V_Hxc Phi) agree, and
  2 H_0 - H_-1 = H[2 V_0 - V_-1] (Algorithm 1 line 11 is linear in V).
"""
import math

import numpy as np
import pytest
from scipy.linalg import expm

from oracle import groundstate, hamiltonian as ham, tddft
from paper_2410_09189_gb300 import inputs


def _rand_herm(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return 0.5 * (A + A.conj().T)


@pytest.mark.parametrize("n,tau", [(5, 0.05), (30, 0.05), (30, 0.4)])
def test_commutator_series_equals_spectral_and_expm(n, tau):
    rng = np.random.default_rng(n)
    H = rng.standard_normal((n, n))
    H = 0.5 * (H + H.T)
    P0 = _rand_herm(n, n + 1)
    P, k = tddft.commutator_series(P0, H, tau, 1e-14)
    Pspec = tddft.spectral_propagate(P0, H, tau)
    U = expm(-1j * tau * H)
    Pexp = U @ P0 @ U.conj().T
    assert np.max(np.abs(P - Pspec)) < 1e-12
    assert np.max(np.abs(P - Pexp)) < 1e-12
    assert k > 3
    # Tr of every correction vanishes: trace is conserved
    assert abs(np.trace(P) - np.trace(P0)) < 1e-12


@pytest.fixture(scope="module")
def ho():
    s = inputs.harmonic(n=32, h=0.4, omega=0.5, nvirt=3)
    gs = groundstate.ground_state(s)
    return s, gs


def test_harmonic_eigenvalues(ho):
    s, gs = ho
    w = s.v_ext_omega
    assert abs(gs["eps"][0] - 1.5 * w) < 1e-6
    assert np.all(np.abs(gs["eps"][1:4] - 2.5 * w) < 1e-6)


def test_harmonic_two_level_kick_closed_form(ho):
    s, gs = ho
    w = s.v_ext_omega
    kappa = 0.05
    o = tddft.Options(dt=0.1, H_thrs=1e-10, dP_thrs=1e-14)
    r = tddft.run(s, gs["phi"], o, nsteps=100, axis=2, kappa=kappa)
    a = 1.0 / math.sqrt(2 * w)
    t = r["t"]
    expect = -2.0 * a * math.sin(2 * kappa * a) * np.sin(w * t)
    amp = 2.0 * a * math.sin(2 * kappa * a)
    assert np.max(np.abs(r["dipole"][:, 2] - expect)) < 2e-6 * amp
    assert np.max(np.abs(r["dipole"][:, :2])) < 1e-10
    # constant H: the extrapolated H_1 is already self-consistent
    assert max(r["passes"]) == 1


def test_trace_hermiticity_idempotency(small_ground_state):
    s, gs = small_ground_state
    o = tddft.Options(H_thrs=1e-9, dP_thrs=1e-12)
    r = tddft.run(s, gs["phi"], o, nsteps=40)
    P = r["state"]["P0"]
    assert np.max(np.abs(r["trace"] - s.n_electrons)) < 1e-12
    assert np.max(np.abs(P - P.conj().T)) < 1e-14
    Q = P / 2
    assert np.max(np.abs(Q @ Q - Q)) < 1e-9


def test_ground_state_is_stationary(small_ground_state):
    s, gs = small_ground_state
    pr = tddft.Propagator(s, gs["phi"], tddft.Options())
    st = pr.initial_state()
    H0 = st["H0"]
    off = H0 - np.diag(np.diag(H0))
    assert np.max(np.abs(off[: s.nocc, s.nocc:])) < 1e-7
    assert np.allclose(np.diag(H0), gs["eps"], atol=1e-7)


def test_energy_conservation(small_ground_state):
    s, gs = small_ground_state
    o = tddft.Options(H_thrs=1e-9, dP_thrs=1e-12)
    r = tddft.run(s, gs["phi"], o, nsteps=200)
    e = r["energy"][1:]
    assert np.max(np.abs(e - e[0])) < 1e-7
    # no drift: the second half does not wander further than the first
    half = len(e) // 2
    assert np.max(np.abs(e[half:] - e[0])) < 2 * np.max(np.abs(e[:half] - e[0])) + 1e-9


def test_hamiltonian_update_forms_and_extrapolation(small_ground_state):
    s, gs = small_ground_state
    full = tddft.Propagator(s, gs["phi"], tddft.Options(full_apply=True))
    dv = tddft.Propagator(s, gs["phi"], tddft.Options(full_apply=False))
    P = np.diag(s.occupations).astype(complex)
    P = full.kick(P, 2, 0.2)
    Ha, aux_a = full.dft(P)
    Hb, aux_b = dv.dft(P)
    assert np.max(np.abs(Ha - Hb)) < 1e-10
    P2 = full.kick(P, 0, 0.3)
    Hc, aux_c = full.dft(P2)
    # linear extrapolation of H equals H of the extrapolated potential
    v_ex = 2 * aux_c["v_hxc"] - aux_a["v_hxc"]
    H_ex = dv.Hcore + dv._sym(dv.h3 * (dv.phi @ (v_ex * dv.phi).T))
    assert np.max(np.abs((2 * Hc - Ha) - H_ex)) < 1e-10


def test_trk_slope_complete_basis():
    s = inputs.harmonic(n=10, h=0.45, omega=1.0, nvirt=999)
    assert s.N == s.Ng
    v = (ham.v_external(s)).ravel()
    Hgrid = ham.apply_h(s, v, np.eye(s.Ng) / math.sqrt(s.h ** 3))
    Hgrid = 0.5 * (Hgrid + Hgrid.T)
    w, W = np.linalg.eigh(Hgrid)
    phi = W.T / math.sqrt(s.h ** 3)
    kappa, dt = 1e-4, 0.002
    o = tddft.Options(dt=dt, H_thrs=1e-12, dP_thrs=1e-15)
    r = tddft.run(s, phi, o, nsteps=2, axis=2, kappa=kappa)
    pr = r["propagator"]
    d = r["dipole"][:, 2]
    slope = (-3 * d[0] + 4 * d[1] - d[2]) / (2 * dt)
    P0 = np.diag(s.occupations)
    Mz, H = pr.M[2], pr.Hcore
    dc = (Mz @ H - H @ Mz) @ Mz - Mz @ (Mz @ H - H @ Mz)
    trk = np.trace(P0 @ dc)
    assert abs(slope + kappa * trk) < 1e-5 * kappa * abs(trk)
    assert abs(trk / s.n_electrons - 1.0) < 2e-2


def test_subspace_ground_state_is_stationary_projector():
    """Subspace SCF: the result is idempotent, commutes with its own H, and with independent
    electrons one undamped iteration is exactly the eigh projector."""
    s = inputs.scaled(inputs.ring(), n=24, h=0.7, nvirt=10)
    raw = inputs.smooth_random_orbitals(s).reshape(s.N, s.Ng)
    phi = ham.orthonormalize(s, raw)
    pr = tddft.Propagator(s, phi, tddft.Options(poisson_tol=1e-13))
    P, H, _, it, err = pr.subspace_ground_state(200, 0.3, 1e-10)
    assert err <= 1e-10 and it < 200
    Q = P / 2
    assert np.max(np.abs(Q @ Q - Q)) < 1e-9
    assert np.max(np.abs(H @ P - P @ H)) < 1e-8
    assert abs(np.trace(P) - s.n_electrons) < 1e-10
    h = inputs.harmonic(n=16, h=0.6, omega=0.8, nvirt=4)
    rawh = inputs.smooth_random_orbitals(h).reshape(h.N, h.Ng)
    prh = tddft.Propagator(h, ham.orthonormalize(h, rawh), tddft.Options())
    P1, H1, _, _, _ = prh.subspace_ground_state(1, 1.0, 0.0)
    w, W = np.linalg.eigh(prh.Hcore)
    assert np.max(np.abs(P1 - 2.0 * np.outer(W[:, 0], W[:, 0]))) < 1e-12
