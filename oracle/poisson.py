"""Hartree potential on the grid: Lap_12 V_H = -4 pi rho (Section 2.1; Algorithm 1's density-functional update).

The paper solves Poisson's equation by multigrid; the oracle solves the *same discrete
equation* by preconditioned conjugate gradients, which reaches the identical solution
without any multigrid machinery:

* operator: the 12th-order Laplacian of ``fd`` (the kinetic-energy stencil);
* boundary: the ghost layers hold the monopole + dipole field of rho about the box centre,
      V_b(r) = Q/|r| + p.r/|r|^3,  Q = h^3 sum rho,  p = h^3 sum rho r,
  (exact outside a spherical charge, so the Gaussian closed form is reachable);
  ``bc="zero"`` gives Dirichlet-zero ghosts instead;
* system: (-Lap_0) V = 4 pi rho + B g, where Lap_0 has zero ghosts and B g is the ghost
  contribution; solved to a relative residual of `tol` (default 1e-13);
* preconditioner: exact inverse of the 12th-order symbol in the sine basis (DST-I); it
  changes only the iteration count, never the converged discrete solution.

Pinned by: the potential of a Gaussian charge, Q erf(r/(sqrt2 sigma))/r, and the
residual of the returned V measured with ``fd.laplacian_padded``.
"""
from __future__ import annotations

import numpy as np
from scipy.fft import dstn, idstn

from . import fd
from .hamiltonian import coords


def multipole_ghosts(sys, rho: np.ndarray, bc: str = "multipole") -> np.ndarray:
    """Array padded by 6 per face whose interior is zero and whose faces hold V_b."""
    r = fd.ORDER_N
    nx, ny, nz = sys.n
    h = sys.h
    gp = np.zeros((nz + 2 * r, ny + 2 * r, nx + 2 * r))
    if bc == "zero":
        return gp
    h3 = h ** 3
    x, y, z = coords(sys)
    Q = h3 * rho.sum()
    p = np.array([h3 * (rho * x).sum(), h3 * (rho * y).sum(), h3 * (rho * z).sum()])
    xe = (np.arange(nx + 2 * r) - r - 0.5 * (nx - 1)) * h
    ye = (np.arange(ny + 2 * r) - r - 0.5 * (ny - 1)) * h
    ze = (np.arange(nz + 2 * r) - r - 0.5 * (nz - 1)) * h
    X = np.broadcast_to(xe[None, None, :], gp.shape)
    Y = np.broadcast_to(ye[None, :, None], gp.shape)
    Zc = np.broadcast_to(ze[:, None, None], gp.shape)
    R = np.sqrt(X * X + Y * Y + Zc * Zc)
    with np.errstate(divide="ignore", invalid="ignore"):
        V = Q / R + (p[0] * X + p[1] * Y + p[2] * Zc) / R ** 3
    inside = np.zeros_like(gp, dtype=bool)
    inside[r:r + nz, r:r + ny, r:r + nx] = True
    gp[~inside] = V[~inside]
    return gp


def _dst_symbol(sys) -> np.ndarray:
    nx, ny, nz = sys.n
    lam = np.zeros((nz, ny, nx))
    for ax, npts in ((2, nx), (1, ny), (0, nz)):
        th = np.pi * np.arange(1, npts + 1) / (npts + 1)
        s = -fd.symbol(th, sys.h)                     # positive
        shape = [1, 1, 1]
        shape[ax] = npts
        lam = lam + s.reshape(shape)
    return lam


def hartree(sys, rho: np.ndarray, tol: float = 1e-13, x0=None, bc: str = "multipole",
            maxiter: int = 5000, return_info: bool = False):
    """Solve Lap_12 V = -4 pi rho with multipole (or zero) ghosts; returns V (nz,ny,nx)."""
    rho = rho.reshape(sys.n[2], sys.n[1], sys.n[0])
    gp = multipole_ghosts(sys, rho, bc)
    b = 4.0 * np.pi * rho + fd.laplacian_padded(gp, sys.h)
    lam = _dst_symbol(sys)

    def A(v):
        return -fd.laplacian(v, sys.h)

    def Minv(r):
        return idstn(dstn(r, type=1) / lam, type=1)

    x = np.zeros_like(rho) if x0 is None else x0.reshape(rho.shape).copy()
    r = b - A(x)
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return (x, 0) if return_info else x
    z = Minv(r)
    p = z.copy()
    rz = np.vdot(r, z)
    it = 0
    while np.linalg.norm(r) > tol * bn and it < maxiter:
        Ap = A(p)
        alpha = rz / np.vdot(p, Ap)
        x += alpha * p
        r -= alpha * Ap
        z = Minv(r)
        rz_new = np.vdot(r, z)
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
    return (x, it) if return_info else x
