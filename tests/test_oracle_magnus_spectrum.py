"""Pins of the oracle's second-order Magnus term, non-orthogonal series and spectrum.

* Omega_1 + Omega_2 (Section 2.2, H linear over the step): on the harmonic oscillator's
  four-level active space driven by a field ramp E_z(t) = E_1 t (so H(t) is exactly linear in
  t), the error of P at t = 4 against an independent high-order ODE integration of
  dP/dt = -i[H(t), P] falls as dt^2 with Omega_1 alone and as dt^4 with Omega_2 added.  A
  wrong sign or factor of Omega_2, or Omega_2 without the field's end values, leaves the
  order at 2.
* Non-orthogonal basis (Section 2.2, Appendix A.2): the series with S^-1 Hbar on raw
  (non-orthonormal) orbitals reproduces the orthogonal propagation of the
  Cholesky-orthonormalised orbitals L^-1 Phi: same dipoles and energies, P_o = L^T P_n L,
  Tr(P S) = N_e and P S P = 2 P.
* Strength function: the trapezoid time sum equals its geometric-series closed form for
  damped sinusoids; the kicked oscillator's line sits at omega_0 and carries N_e (sum rule).
"""
import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp

from oracle import groundstate, spectrum, tddft
from paper_2410_09189_gb300 import inputs


@pytest.fixture(scope="module")
def ho():
    s = inputs.harmonic(n=32, h=0.4, omega=0.5, nvirt=3)
    gs = groundstate.ground_state(s)
    return s, gs


def _ramp_error(s, phi, dt, magnus2, E1=0.05, T=4.0):
    ramp = lambda t: np.array([0.0, 0.0, E1 * t])
    o = tddft.Options(dt=dt, H_thrs=1e-12, dP_thrs=1e-16, magnus2=magnus2)
    r = tddft.run(s, phi, o, nsteps=int(round(T / dt)), kappa=0.0, field=ramp)
    pr, P = r["propagator"], r["state"]["P0"]
    N = P.shape[0]
    Hc, Mz = pr.Hcore, pr.M[2]

    def rhs(t, y):
        Q = y.reshape(N, N)
        H = Hc + E1 * t * Mz
        return (-1j * (H @ Q - Q @ H)).ravel()

    P0 = np.diag(s.occupations).astype(complex)
    ref = solve_ivp(rhs, (0.0, T), P0.ravel(), method="DOP853", rtol=1e-13, atol=1e-15)
    Pref = ref.y[:, -1].reshape(N, N)
    return float(np.max(np.abs(P - Pref)))


def test_magnus_truncation_orders_on_a_linear_ramp(ho):
    s, gs = ho
    e1 = [_ramp_error(s, gs["phi"], dt, False) for dt in (0.2, 0.1)]
    e2 = [_ramp_error(s, gs["phi"], dt, True) for dt in (0.2, 0.1)]
    r1, r2 = e1[0] / e1[1], e2[0] / e2[1]
    assert 3.3 < r1 < 4.7, (e1, r1)
    assert 12.0 < r2 < 20.0, (e2, r2)
    assert e2[1] < 0.05 * e1[1], (e1, e2)


def test_omega2_vanishes_for_a_constant_hamiltonian(ho):
    """Without a field H_0 = H_1 = H_core: Omega_2 = 0, the kicked trajectories coincide."""
    s, gs = ho
    a = tddft.run(s, gs["phi"], tddft.Options(dt=0.1, dP_thrs=1e-15), nsteps=20, kappa=0.05)
    b = tddft.run(s, gs["phi"], tddft.Options(dt=0.1, dP_thrs=1e-15, magnus2=True), nsteps=20,
                  kappa=0.05)
    assert np.max(np.abs(a["dipole"] - b["dipole"])) < 1e-14


def test_nonorthogonal_series_equals_the_orthonormalised_basis():
    s = inputs.small()
    raw = inputs.smooth_random_orbitals(s).reshape(s.N, s.Ng)
    h3 = s.h ** 3
    L = np.linalg.cholesky(h3 * raw @ raw.T)
    phi_o = np.linalg.solve(L, raw)
    kw = dict(dt=0.05, H_thrs=1e-11, dP_thrs=1e-14, poisson_tol=1e-13)
    ro = tddft.run(s, phi_o, tddft.Options(**kw), nsteps=8, axis=2, kappa=1e-2)
    rn = tddft.run(s, raw, tddft.Options(nonorthogonal=True, **kw), nsteps=8, axis=2, kappa=1e-2)
    # the raw orbitals are far from orthonormal, so the test is not trivial
    S = rn["propagator"].S
    assert np.max(np.abs(S - np.eye(s.N))) > 0.1
    scale = np.max(np.abs(ro["dipole"] - ro["dipole"][0]))
    assert np.max(np.abs(rn["dipole"] - ro["dipole"])) < 1e-8 * scale
    assert np.max(np.abs(rn["energy"] - ro["energy"])) < 1e-9
    Pn, Po = rn["state"]["P0"], ro["state"]["P0"]
    assert np.max(np.abs(L.T @ Pn @ L - Po)) < 1e-9
    ne = float(np.sum(s.occupations))
    assert np.max(np.abs(rn["trace"] - ne)) < 1e-10
    assert np.max(np.abs(Pn @ S @ Pn - 2.0 * Pn)) < 1e-9


def _damped_sine_sum(A, w0, gamma, w, dt, nt):
    """sum_n wt_n A sin(w0 t_n) e^{-gamma t_n} sin(w t_n) dt (trapezoid weights) in closed form:
    sin a sin b = (cos(a - b) - cos(a + b))/2 and sum_{n=0}^{M} r^n = (1 - r^{M+1})/(1 - r)."""
    M = nt - 1

    def csum(beta):
        r = np.exp((1j * beta - gamma) * dt)
        geo = (1.0 - r ** (M + 1)) / (1.0 - r)
        return np.real(geo - 0.5 * (1.0 + r ** M))

    return A * dt * 0.5 * (csum(w0 - w) - csum(w0 + w))


def test_strength_function_equals_the_geometric_closed_form():
    dt, nt, kappa, gamma = 0.07, 3001, 2e-3, 0.013
    omega = np.linspace(0.01, 3.0, 211)
    amps = [(-1.3e-3, 0.41, 0.2), (2.2e-4, 1.7, -0.05), (-7e-4, 0.93, 1.5)]
    t = dt * np.arange(nt)
    d = np.array([off + A * np.sin(w0 * t) for A, w0, off in amps])
    S = spectrum.strength_function(d, dt, kappa, gamma, omega)
    expect = sum(_damped_sine_sum(A, w0, gamma, omega, dt, nt) for A, w0, _ in amps)
    expect *= -2.0 * omega / (np.pi * kappa * 3)
    assert np.max(np.abs(S - expect)) < 1e-11 * np.max(np.abs(expect))


def test_kicked_oscillator_line_position_and_sum_rule():
    """d_z(t) = -N_e a sin(2 kappa a) sin(w0 t), a = (2 w0)^-1/2 (the kicked two-level closed
    form): one line at w0 whose strength is N_e (f = 2 w0 a^2 per electron = 1)."""
    w0, ne, kappa = 0.5, 2.0, 1e-4
    a = 1.0 / math.sqrt(2 * w0)
    dt, nt, gamma = 0.1, 10001, 0.01
    t = dt * np.arange(nt)
    d = -ne * a * math.sin(2 * kappa * a) * np.sin(w0 * t)
    omega = np.arange(1, 5001) * 1e-3
    S = spectrum.strength_function(d[None, :], dt, kappa, gamma, omega)
    assert abs(omega[np.argmax(S)] - w0) <= 1e-3
    assert np.min(S) > -1e-3 * np.max(S)
    total = float(np.sum(S) * 1e-3)
    assert abs(total - ne) < 0.01 * ne, total
