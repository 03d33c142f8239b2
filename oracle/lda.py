"""LDA exchange-correlation, spin-unpolarised: Slater exchange + Perdew-Zunger 1981 correlation.

The paper's runs use PBE (Section 4); the hot path uses LDA (Slater + PZ81), the functional
the paper cites for the first real-space RT-TDDFT (Section 1).

  exchange:    eps_x = -(3/4)(3 rho/pi)^(1/3),  V_x = -(3 rho/pi)^(1/3)
  correlation: r_s = (3/(4 pi rho))^(1/3)
    r_s >= 1:  eps_c = gamma / (1 + beta1 sqrt(r_s) + beta2 r_s)
    r_s <  1:  eps_c = A ln r_s + B + C r_s ln r_s + D r_s
    V_c = eps_c - (r_s/3) d eps_c / d r_s
  gamma=-0.1423, beta1=1.0529, beta2=0.3334, A=0.0311, B=-0.048, C=0.0020, D=-0.0116.
  rho < 1e-14 gives eps = V = 0.

Pinned by: V = d(rho eps)/d rho by finite differences, the Fermi-wavevector form of Slater
exchange eps_x = -3 k_F/(4 pi) with k_F = (3 pi^2 rho)^(1/3), the Gell-Mann-Brueckner
high-density slope d eps_c / d ln r_s -> (1 - ln 2)/pi^2, and the continuity of eps_c and
V_c across r_s = 1 (the conditions PZ81 imposed on B, C, D).
"""
from __future__ import annotations

import numpy as np

RHO_FLOOR = 1e-14
PZ_GAMMA, PZ_BETA1, PZ_BETA2 = -0.1423, 1.0529, 0.3334
PZ_A, PZ_B, PZ_C, PZ_D = 0.0311, -0.048, 0.0020, -0.0116


def exchange(rho: np.ndarray):
    """Slater exchange (V_x, eps_x) for rho >= RHO_FLOOR (no floor applied here)."""
    t = np.cbrt(3.0 * rho / np.pi)
    return -t, -0.75 * t


def correlation(rho: np.ndarray):
    """PZ81 correlation (V_c, eps_c) for rho >= RHO_FLOOR (no floor applied here)."""
    rs = np.cbrt(3.0 / (4.0 * np.pi * rho))
    lo = rs >= 1.0
    sq = np.sqrt(rs)
    den = 1.0 + PZ_BETA1 * sq + PZ_BETA2 * rs
    ec_lo = PZ_GAMMA / den
    dec_lo = -PZ_GAMMA * (0.5 * PZ_BETA1 / sq + PZ_BETA2) / (den * den)
    lnr = np.log(rs)
    ec_hi = PZ_A * lnr + PZ_B + PZ_C * rs * lnr + PZ_D * rs
    dec_hi = PZ_A / rs + PZ_C * (lnr + 1.0) + PZ_D
    ec = np.where(lo, ec_lo, ec_hi)
    dec = np.where(lo, dec_lo, dec_hi)
    return ec - rs / 3.0 * dec, ec


def lda(rho: np.ndarray):
    """Return (V_xc, eps_xc) for a density array (any shape)."""
    rho = np.asarray(rho, dtype=np.float64)
    ok = rho >= RHO_FLOOR
    r = np.where(ok, rho, 1.0)
    vx, ex = exchange(r)
    vc, ec = correlation(r)
    vxc = np.where(ok, vx + vc, 0.0)
    exc = np.where(ok, ex + ec, 0.0)
    return vxc, exc
