"""Pins of the oracle's propagation (Algorithm 1) against results fixed by the mathematics.

* Commutator expansion (Eq. 19 / 33) = spectral propagator W exp(omega) W^dagger
  (Section 2.2) = scipy expm, within dP_thrs.
* Harmonic oscillator: eigenvalues (n + 3/2) omega, and the kicked dipole of the
  two-level active space, d_z(t) = -N_e a sin(2 kappa a) sin(omega t), a = (2 omega)^-1/2.
* Tr P conserved, P Hermitian, (P/2)^2 = P/2 for a closed shell.
* Zero-field energy conservation after the kick (Section 4.2: no drift).
* Time-domain TRK sum rule: d'(0+) = -kappa Tr(P_0 [[M,H],M]) -> -kappa N_e (complete basis).
* The two Hamiltonian-update forms (full apply vs H_core + Phi^T V_Hxc Phi) agree, and
  2 H_0 - H_-1 = H[2 V_0 - V_-1] (Algorithm 1's extrapolation is linear in V).
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


def test_harmonic_two_level_field_linear_response(ho):
    """A weak field E_z(t) = E0 sin(W t) on the harmonic oscillator's two-level active space
    (ground orbital and the z-excited one, coupled by M_z with element a = (2 w)^(-1/2)): the
    dipole is the convolution of the kick response, d(t) = -4 a^2 E0 integral_0^t
    sin(w (t - s)) sin(W s) ds = -4 a^2 E0 (W sin(w t) - w sin(W t)) / (W^2 - w^2), to the
    O(E0^2) nonlinearity and the O(dt^2) time stepping (Algorithm 1's V_{j-1} + V_j in Omega).
    A wrong sign or factor of the field term, or a field sampled at one end of the step only,
    moves d(t) by far more than the bound."""
    s, gs = ho
    w = s.v_ext_omega
    E0, W = 1e-4, 0.3
    o = tddft.Options(dt=0.05, H_thrs=1e-12, dP_thrs=1e-15)
    r = tddft.run(s, gs["phi"], o, nsteps=300, axis=2, kappa=0.0,
                  field=lambda t: np.array([0.0, 0.0, E0 * math.sin(W * t)]))
    a = 1.0 / math.sqrt(2 * w)
    t = r["t"]
    expect = -4.0 * a * a * E0 * (W * np.sin(w * t) - w * np.sin(W * t)) / (W * W - w * w)
    d = r["dipole"][:, 2] - r["dipole"][0, 2]
    amp = np.max(np.abs(expect))
    assert np.max(np.abs(d - expect)) < 2e-3 * amp, np.max(np.abs(d - expect)) / amp
    assert np.max(np.abs(r["dipole"][:, :2] - r["dipole"][0, :2])) < 1e-10


def test_xc_energy_gradient_is_the_xc_hamiltonian_with_a_frozen_core(small_ground_state):
    """The Kohn-Sham exchange-correlation matrix is the gradient of the xc energy with respect
    to the density matrix, with a frozen core density added to rho inside the xc (Section 3.1's
    frozen semicore): [E_xc(P + e D) - E_xc(P - e D)] / 2e = Tr(H_xc D) for a symmetric D, with
    E_xc = E - Tr(P H_core) - 1/2 h^3 sum rho V_H - E_ion from the oracle's energy and
    H_xc = h^3 Phi^T diag(V_xc) Phi from its H.  An energy that weights eps_xc by rho instead
    of rho + rho_core, or a V_xc without the core, fails by orders of magnitude."""
    import dataclasses
    s, gs = small_ground_state
    s = dataclasses.replace(s, rho_core=inputs.gaussian_core_density(s, charge=0.6, width=0.7))
    pr = tddft.Propagator(s, gs["phi"], tddft.Options(poisson_tol=1e-13))
    f = s.occupations
    rng = np.random.default_rng(11)
    D = rng.standard_normal((s.N, s.N))
    D = 0.5 * (D + D.T) / np.linalg.norm(D, 2)
    # P >= 0.1 I and |e D| << 0.1: rho >= 0 everywhere for P, P + e D and P - e D (a negative
    # density would meet the LDA's floor and break the finite difference)
    P = np.diag(f + 0.1).astype(complex)

    def exc_energy(PP):
        H, aux = pr.dft(PP)
        e_nonxc = (float(np.trace(np.real(PP) @ pr.Hcore)) + 0.5 * pr.h3 * float(aux["rho"] @ aux["vh"])
                   + pr.E_ion)
        return pr.energy(PP, aux) - e_nonxc, aux

    _, aux = exc_energy(P)
    Hxc = pr.h3 * (pr.phi @ (aux["vxc"] * pr.phi).T)
    eps = 1e-4
    g = (exc_energy(P + eps * D)[0] - exc_energy(P - eps * D)[0]) / (2 * eps)
    expect = float(np.trace(Hxc @ D))
    assert abs(g - expect) < 1e-6 * abs(expect), (g, expect)
    # the core changes the xc energy and matrix (it is not silently ignored)
    pr0 = tddft.Propagator(dataclasses.replace(s, rho_core=None), gs["phi"],
                           tddft.Options(poisson_tol=1e-13))
    _, aux0 = pr0.dft(P)
    assert np.max(np.abs(aux0["vxc"] - aux["vxc"])) > 1e-3
