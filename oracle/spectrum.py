"""Absorption spectrum from the kicked dipole series (Section 4: a sum of Fourier transforms of
mu_x(t), mu_y(t), mu_z(t) from three runs kicked along x, y and z).

TEST INFRASTRUCTURE ONLY (see the package header).

Reading (the paper gives no formula): with the electronic dipole d_q(t) = Tr(Re P M_q) of the
run kicked along q by kappa, the dynamic polarisability is
    alpha_q(omega) = -(1/kappa) int_0^T (d_q(t) - d_q(0)) e^{i omega t - gamma t} dt,
the exponential damping gamma giving each line a Lorentzian width, and the dipole strength
function is the orientation mean
    S(omega) = (2 omega / pi) (1/n_q) sum_q Im alpha_q(omega)
             = -(2 omega / (pi kappa n_q)) sum_q int (d_q(t) - d_q(0)) e^{-gamma t} sin(omega t) dt,
normalised so that int_0^inf S d omega = N_e in a complete basis (the Thomas-Reiche-Kuhn sum
rule).  The time integral is the trapezoid rule over the samples t_n = n dt, n = 0..nt-1.

Pinned by: the geometric-series closed form of the trapezoid sum for a damped sinusoid, the
sum rule and line position of the kicked harmonic oscillator.
"""
from __future__ import annotations

import numpy as np


def strength_function(d: np.ndarray, dt: float, kappa: float, gamma: float,
                      omega: np.ndarray) -> np.ndarray:
    """S(omega) from d of shape (n_q, nt): row q is the q component of the run kicked along q."""
    d = np.atleast_2d(np.asarray(d, dtype=np.float64))
    nq, nt = d.shape
    t = dt * np.arange(nt)
    w = np.ones(nt)
    w[0] = w[-1] = 0.5
    if nt == 1:
        w[0] = 0.0
    total = np.zeros(len(omega))
    for q in range(nq):
        g = (d[q] - d[q, 0]) * np.exp(-gamma * t) * w * dt
        total += np.sin(np.outer(omega, t)) @ g
    return -2.0 * np.asarray(omega) / (np.pi * kappa * nq) * total
