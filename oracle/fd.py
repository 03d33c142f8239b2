"""Central finite-difference second derivative and the 3-D Laplacian (Section 2.1, Eq. 2).

The 2n+1-point central formula psi''(x0) ~ a0 psi(x0) + sum_i a_i (psi(x0+ih) + psi(x0-ih))
is made exact for polynomials of degree <= 2n.  The closed form used here (Fornberg) is
    a_m = 2 (-1)^(m+1) (n!)^2 / (m^2 (n-m)! (n+m)!),   a_0 = -2 sum_m a_m.
The hot path uses n = 6 (12th order, radius-6, 37-point 3-D stencil).  The paper's adaptive
mixed-order form (Eq. 3) is not used: its mixing parameter is fitted to atomic orbitals.

Pinned by: exactness on all monomials of degree <= 12 (the property Eq. 2 states), the
plane-wave symbol at interior points, sum a = 0 and sum m^2 a_m = 1.
"""
from __future__ import annotations

from fractions import Fraction
from math import factorial

import numpy as np

ORDER_N = 6       # half-width of the stencil; 2n = 12th order


def fd_coefficients_exact(n: int = ORDER_N):
    """Exact rational coefficients [a_0, a_1, ..., a_n] of the 2n+1-point second derivative."""
    a = [Fraction(0)] * (n + 1)
    for m in range(1, n + 1):
        a[m] = Fraction(2 * (-1) ** (m + 1) * factorial(n) ** 2,
                        m * m * factorial(n - m) * factorial(n + m))
    a[0] = -2 * sum(a[1:])
    return a


def fd_coefficients(n: int = ORDER_N) -> np.ndarray:
    return np.array([float(c) for c in fd_coefficients_exact(n)])


def pad_zero(f: np.ndarray, r: int = ORDER_N) -> np.ndarray:
    """Embed a (nz, ny, nx) array in zeros: Dirichlet-zero ghost layers of width r."""
    return np.pad(f, r, mode="constant")


def laplacian_padded(fp: np.ndarray, h: float, n: int = ORDER_N) -> np.ndarray:
    """Laplacian at the interior points of a ghost-padded array (ghost width n per face).

    Only the face slabs of the padding are read (the stencil is a 3-axis star), so edge
    and corner ghosts are irrelevant.
    """
    a = fd_coefficients(n)
    nz, ny, nx = (s - 2 * n for s in fp.shape)
    c = fp[n:n + nz, n:n + ny, n:n + nx]
    out = 3.0 * a[0] * c
    for m in range(1, n + 1):
        out = out + a[m] * (fp[n:n + nz, n:n + ny, n + m:n + m + nx]
                            + fp[n:n + nz, n:n + ny, n - m:n - m + nx])
        out = out + a[m] * (fp[n:n + nz, n + m:n + m + ny, n:n + nx]
                            + fp[n:n + nz, n - m:n - m + ny, n:n + nx])
        out = out + a[m] * (fp[n + m:n + m + nz, n:n + ny, n:n + nx]
                            + fp[n - m:n - m + nz, n:n + ny, n:n + nx])
    return out / (h * h)


def laplacian(f: np.ndarray, h: float, n: int = ORDER_N) -> np.ndarray:
    """12th-order Laplacian of a grid function with Dirichlet-zero ghosts."""
    return laplacian_padded(pad_zero(f, n), h, n)


def laplacian_1d(f: np.ndarray, h: float, n: int = ORDER_N) -> np.ndarray:
    """1-D second derivative with zero ghosts (used by the polynomial pins)."""
    a = fd_coefficients(n)
    fp = np.pad(f, n)
    L = len(f)
    out = a[0] * f
    for m in range(1, n + 1):
        out = out + a[m] * (fp[n + m:n + m + L] + fp[n - m:n - m + L])
    return out / (h * h)


def symbol(theta: np.ndarray, h: float, n: int = ORDER_N) -> np.ndarray:
    """Fourier symbol of the 1-D operator on exp(i theta x/h): (a0 + 2 sum a_m cos m theta)/h^2."""
    a = fd_coefficients(n)
    s = a[0] * np.ones_like(theta)
    for m in range(1, n + 1):
        s = s + 2.0 * a[m] * np.cos(m * theta)
    return s / (h * h)
