"""Ground-state Kohn-Sham orbitals that define the active space (Algorithm 1's ground state).

Self-consistent field at the Gamma point: for the current density, the N lowest
eigenpairs of the sparse grid Hamiltonian are found with ARPACK (scipy ``eigsh``, smallest
algebraic), the density sum_i f_i |phi_i|^2 is rebuilt and Pulay-mixed until it stops
changing.  Orbitals are returned grid-normalised (h^3 sum phi_i phi_j = delta_ij) with the
sign fixed so that each orbital's largest-magnitude value is positive.

Pinned by (tests/test_oracle_groundstate.py): on a 576-point grid with a KB projector, a
dense LAPACK diagonalisation of the whole grid Hamiltonian -- the independent-electron
eigenpairs and occupied projector, the Kohn-Sham fixed point rho = rho(eig(H[rho])) with
Hartree and LDA, and the stationarity and minimality of the Kohn-Sham energy under an
occupied-virtual rotation; also the harmonic-oscillator eigenvalues.
"""
from __future__ import annotations

import numpy as np
from scipy.sparse.linalg import LinearOperator, eigsh

from . import hamiltonian as ham
from .lda import lda
from .poisson import hartree


def _lowest(sys, v_total, projs, k, v0, tol):
    Ng = sys.Ng

    def mv(x):
        return ham.apply_h(sys, v_total, x.reshape(1, Ng), projs).ravel()

    op = LinearOperator((Ng, Ng), matvec=mv, dtype=np.float64)
    # Single-vector Lanczos can miss copies of a degenerate eigenvalue: ask for a margin
    # of extra pairs and keep the k lowest.
    kk = min(Ng - 2, k + max(6, k // 2))
    w, v = eigsh(op, k=kk, which="SA", v0=v0, tol=tol, ncv=min(Ng - 1, max(2 * kk + 1, 40)))
    order = np.argsort(w)[:k]
    return w[order], v[:, order].T


def ground_state(sys, tol: float = 1e-9, maxit: int = 200, mix: float = 0.4,
                 eig_tol: float = 1e-12, verbose: bool = False):
    """Return dict(phi=(N,Ng), eps=(N,), rho, v_hxc, iterations)."""
    projs = ham.projectors(sys)
    v_ion = (ham.v_local(sys) + ham.v_external(sys)).ravel()
    f = sys.occupations
    h3 = sys.h ** 3
    rng = np.random.default_rng(sys.seed + 999)
    v0 = rng.standard_normal(sys.Ng)
    rho = None
    v_hxc = np.zeros(sys.Ng)
    vh = None
    hist_in, hist_res = [], []
    it = 0
    for it in range(1, maxit + 1):
        eps, vecs = _lowest(sys, v_ion + v_hxc, projs, sys.N, v0, eig_tol)
        phi = vecs / np.sqrt(h3)
        rho_out = (f[:, None] * phi * phi).sum(0)
        if not sys.hartree_xc:
            rho = rho_out
            break
        if rho is None:
            err = np.inf
            rho = rho_out
        else:
            # Pulay (DIIS) mixing of the density residual rho_out - rho_in.
            res = rho_out - rho
            err = np.max(np.abs(res))
            hist_in.append(rho.copy())
            hist_res.append(res)
            if len(hist_in) > 6:
                hist_in.pop(0)
                hist_res.pop(0)
            m = len(hist_in)
            B = np.empty((m + 1, m + 1))
            B[:m, :m] = [[np.dot(a, b) for b in hist_res] for a in hist_res]
            B[m, :m] = B[:m, m] = 1.0
            B[m, m] = 0.0
            rhs = np.zeros(m + 1)
            rhs[m] = 1.0
            c = np.linalg.lstsq(B, rhs, rcond=None)[0][:m]
            rho = sum(ci * (ri + mix * fi) for ci, ri, fi in zip(c, hist_in, hist_res))
            rho = np.maximum(rho, 0.0)
        if verbose:
            print(f"gs it {it} err {err:.3e} eps0 {eps[0]:.8f}")
        if err < tol:
            rho = rho_out
            break
        shape = (sys.n[2], sys.n[1], sys.n[0])
        vh = hartree(sys, rho.reshape(shape), x0=vh).ravel()
        vxc, _ = lda(rho)
        v_hxc = vh + vxc
        v0 = vecs[0]
    for i in range(sys.N):
        j = np.argmax(np.abs(phi[i]))
        if phi[i, j] < 0:
            phi[i] = -phi[i]
    return {"phi": phi, "eps": eps, "rho": rho, "v_hxc": v_hxc, "iterations": it}
