"""Kohn-Sham Hamiltonian on the uniform grid (Section 2.1, Eqs. 1, 2 and 4).

H psi = -1/2 Lap_12 psi + (V_loc + V_ext + V_H + V_xc) psi + sum_p beta_p E_p <beta_p|psi>

* Grid: point i of an axis with n points sits at (i - (n-1)/2) h, so the box centre is
  the origin; arrays are (nz, ny, nx) with x fastest.  Eq. 1 prints +1/2 Lap: the sign is
  a typo, the kinetic term is -1/2 Lap.
* Inner products use the grid quadrature of Eq. 4 in 3-D: <a|b> = h^3 sum a b.
* Local well of atom a: -Z_a erf(|r-R_a|/rc_a)/|r-R_a|, value -2 Z_a/(rc_a sqrt(pi)) at
  r = 0 (the potential of a Gaussian ion charge).
* Kleinman-Bylander projectors (separable nonlocal part, Section 2.1): s-type
  exp(-r^2/rc^2), p-type (q-R_q) exp(-r^2/rc^2), zero beyond r > 5 rc, normalised on the
  grid to h^3 sum beta^2 = 1.
* Ion-ion energy of Gaussian ions: sum_{a<b} Z_a Z_b erf(R_ab/sqrt(rc_a^2+rc_b^2))/R_ab.

Pinned by: brute-force KB matrix elements, the plane-wave / polynomial pins of ``fd``,
and the harmonic-oscillator eigenvalues (n + 3/2) omega.
"""
from __future__ import annotations

import math
from typing import List, Tuple

import numpy as np
from scipy.special import erf

from . import fd


def axis_coords(npts: int, h: float) -> np.ndarray:
    return (np.arange(npts) - 0.5 * (npts - 1)) * h


def coords(sys) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Broadcastable x, y, z coordinate arrays of shape (1,1,nx), (1,ny,1), (nz,1,1)."""
    nx, ny, nz = sys.n
    x = axis_coords(nx, sys.h)[None, None, :]
    y = axis_coords(ny, sys.h)[None, :, None]
    z = axis_coords(nz, sys.h)[:, None, None]
    return x, y, z


def full_coords(sys) -> List[np.ndarray]:
    x, y, z = coords(sys)
    shape = (sys.n[2], sys.n[1], sys.n[0])
    return [np.broadcast_to(c, shape).copy() for c in (x, y, z)]


def v_local(sys) -> np.ndarray:
    """Sum of Gaussian-erf wells, shape (nz, ny, nx)."""
    x, y, z = coords(sys)
    v = np.zeros((sys.n[2], sys.n[1], sys.n[0]))
    for a in range(len(sys.Z)):
        r = np.sqrt((x - sys.pos[a, 0]) ** 2 + (y - sys.pos[a, 1]) ** 2
                    + (z - sys.pos[a, 2]) ** 2)
        rc = sys.rc_loc[a]
        with np.errstate(divide="ignore", invalid="ignore"):
            w = np.where(r > 0.0, -sys.Z[a] * erf(r / rc) / r,
                         -2.0 * sys.Z[a] / (rc * math.sqrt(math.pi)))
        v += w
    return v


def v_external(sys) -> np.ndarray:
    """Static external well (harmonic test mode only): 0.5 omega^2 r^2, else zero."""
    x, y, z = coords(sys)
    shape = (sys.n[2], sys.n[1], sys.n[0])
    if sys.v_ext_omega > 0.0:
        return np.broadcast_to(0.5 * sys.v_ext_omega ** 2 * (x * x + y * y + z * z),
                               shape).copy()
    return np.zeros(shape)


def projectors(sys) -> List[Tuple[np.ndarray, np.ndarray]]:
    """KB projectors as (flat grid indices, normalised values) pairs."""
    x, y, z = full_coords(sys)
    x, y, z = x.ravel(), y.ravel(), z.ravel()
    out = []
    h3 = sys.h ** 3
    for p in range(sys.nproj):
        a = sys.proj_atom[p]
        rc = sys.proj_rc[p]
        dx, dy, dz = x - sys.pos[a, 0], y - sys.pos[a, 1], z - sys.pos[a, 2]
        r2 = dx * dx + dy * dy + dz * dz
        idx = np.nonzero(r2 <= 25.0 * rc * rc)[0]
        val = np.exp(-r2[idx] / (rc * rc))
        if sys.proj_l[p] == 1:
            val = val * (dx, dy, dz)[sys.proj_m[p]][idx]
        val = val / math.sqrt(h3 * np.sum(val * val))
        out.append((idx, val))
    return out


def apply_nonlocal(sys, projs, psi: np.ndarray) -> np.ndarray:
    """sum_p beta_p E_p h^3 <beta_p, psi> for a batch psi of shape (k, Ng)."""
    out = np.zeros_like(psi)
    h3 = sys.h ** 3
    for p, (idx, val) in enumerate(projs):
        c = h3 * (psi[:, idx] @ val)                 # (k,)
        out[:, idx] += sys.E_kb[p] * np.outer(c, val)
    return out


def apply_h(sys, v_total: np.ndarray, psi: np.ndarray, projs=None) -> np.ndarray:
    """H psi for psi of shape (k, Ng): kinetic + local potential `v_total` + KB part."""
    if projs is None:
        projs = projectors(sys)
    shape = (sys.n[2], sys.n[1], sys.n[0])
    vt = v_total.ravel()
    out = np.empty_like(psi)
    for i in range(psi.shape[0]):
        f = psi[i].reshape(shape)
        out[i] = (-0.5 * fd.laplacian(f, sys.h)).ravel() + vt * psi[i]
    if projs:
        out += apply_nonlocal(sys, projs, psi)
    return out


def ion_energy(sys) -> float:
    e = 0.0
    for a in range(len(sys.Z)):
        for b in range(a):
            R = float(np.linalg.norm(sys.pos[a] - sys.pos[b]))
            s = math.sqrt(sys.rc_loc[a] ** 2 + sys.rc_loc[b] ** 2)
            e += sys.Z[a] * sys.Z[b] * math.erf(R / s) / R
    return e


def orthonormalize(sys, phi: np.ndarray) -> np.ndarray:
    """Cholesky-QR in float64 so that h^3 Phi Phi^T = I (rows of `phi` are orbitals)."""
    h3 = sys.h ** 3
    S = h3 * (phi @ phi.T)
    L = np.linalg.cholesky(S)
    return np.linalg.solve(L, phi)
