"""Propagation of the occupied orbitals on the grid: the complete-grid-basis limit of
Algorithm 1, in float64.

TEST INFRASTRUCTURE ONLY (see the package header).

Section 2.2's propagation holds in any basis; the grid itself (N = N_g) is the complete
limit of the active space.  With P = sum_n f_n |psi_n><psi_n|, the propagated
e^{Omega} P e^{Omega^dagger} equals sum_n f_n (e^{Omega} psi_n)(e^{Omega} psi_n)^dagger, so
applying the exponential to the occupied orbitals propagates P without truncation:

* Step (Algorithm 1's time loop in the grid basis, where H depends on time only through the
  potential V = V_H + V_xc):
    V_1 <- 2 V_0 - V_-1                                  (the extrapolation)
    repeat:
      psi_1 = sum_k psi^(k), psi^(0) = psi_0, psi^(k) = (-i dt / k) Hbar psi^(k-1),
        Hbar = T + V_ion + V_NL + (V_0 + V_1)/2 + sum_q Ebar_q q   (the series of Eq. 33
        acting on the orbitals), stopped when max|psi^(k)| <= dP_thrs
      V_new = V_H + V_xc of rho = sum_n f_n |psi_1,n|^2; err = max|V_new - V_1|; V_1 <- V_new
    until err <= H_thrs      (in the grid basis H_new - H_1 is diagonal: max|V_new - V_1|)
    psi_1 re-orthonormalised by Cholesky (S = h^3 psi psi^dagger = L L^dagger,
    psi <- L^-1 psi), then V_-1 <- V_0, V_0 <- V_1, psi_0 <- psi_1.
* Kick: psi <- e^{-i kappa q} psi (the kick's exponential is diagonal on the grid).
* Observables: d_q = h^3 sum q rho; E = sum_n f_n h^3 <psi_n|T + V_ion + V_NL|psi_n>
  + 1/2 h^3 sum rho V_H + h^3 sum (rho + rho_core) eps_xc + E_ion.

Pinned by: the density-matrix propagation of Algorithm 1 (``tddft``) with the complete basis
of a 10^3 grid (all 1000 eigenvectors of the core Hamiltonian as the active space), which must
give the same dipoles and energies; orthonormality and electron count.
"""
from __future__ import annotations

from typing import Optional

import numpy as np

from . import hamiltonian as ham
from .lda import lda
from .poisson import hartree


class GridPropagator:
    """Occupied orbitals psi (n_occ, Ng) complex, propagated on the grid."""

    def __init__(self, sys, psi0: np.ndarray, f: np.ndarray, opts, field=None):
        self.sys = sys
        self.opts = opts
        self.field = field
        self.h3 = sys.h ** 3
        self.shape = (sys.n[2], sys.n[1], sys.n[0])
        self.f = np.asarray(f, dtype=np.float64)
        self.psi = np.asarray(psi0, dtype=np.complex128).copy()
        self.projs = ham.projectors(sys)
        self.v_ion = (ham.v_local(sys) + ham.v_external(sys)).ravel()
        self.q = [c.ravel() for c in ham.full_coords(sys)]
        self.E_ion = ham.ion_energy(sys)
        core = getattr(sys, "rho_core", None)
        self.rho_core = np.zeros(sys.Ng) if core is None else np.asarray(core, float).ravel()
        self.vh = None
        self.t = 0.0
        v, self.aux = self.potential(self.psi)
        self.V0 = v
        self.Vm1 = v.copy()

    # --- building blocks -------------------------------------------------------------
    def density(self, psi) -> np.ndarray:
        return np.real(np.einsum("n,ng->g", self.f, np.abs(psi) ** 2))

    def potential(self, psi):
        rho = self.density(psi)
        if self.sys.hartree_xc:
            vh = hartree(self.sys, rho.reshape(self.shape), tol=self.opts.poisson_tol,
                         x0=self.vh).ravel()
            self.vh = vh
            vxc, exc = lda(rho + self.rho_core)
        else:
            vh = np.zeros_like(rho)
            vxc = np.zeros_like(rho)
            exc = np.zeros_like(rho)
        return vh + vxc, {"rho": rho, "vh": vh, "vxc": vxc, "exc": exc}

    def field_at(self, t: float) -> np.ndarray:
        if self.field is None:
            return np.zeros(self.sys.Ng)
        e = np.asarray(self.field(t), dtype=float)
        return e[0] * self.q[0] + e[1] * self.q[1] + e[2] * self.q[2]

    def taylor(self, psi0, vbar):
        """exp(-i dt Hbar) psi0 by the series; returns (psi, terms)."""
        o = self.opts
        psi = psi0.copy()
        term = psi0.copy()
        k = 0
        while True:
            k += 1
            if k > o.max_terms:
                raise RuntimeError(f"orbital series exceeded {o.max_terms} terms")
            term = (-1j * o.dt / k) * ham.apply_h(self.sys, self.v_ion + vbar, term, self.projs)
            psi += term
            err = float(np.max(np.abs(term)))
            if not np.isfinite(err):
                raise RuntimeError("orbital series diverged")
            if err <= o.dP_thrs:
                return psi, k

    def orthonormalize(self, psi):
        S = self.h3 * (psi.conj() @ psi.T)     # S_nm = h^3 <psi_n|psi_m>
        L = np.linalg.cholesky(S.T)            # S^T = S^* = L L^dagger
        return np.linalg.solve(L, psi)

    def kick(self, axis: int, kappa: float):
        self.psi = np.exp(-1j * kappa * self.q[axis])[None, :] * self.psi

    def step(self):
        o = self.opts
        dt = o.dt
        V1 = 2.0 * self.V0 - self.Vm1
        ebar = 0.5 * (self.field_at(self.t) + self.field_at(self.t + dt))
        terms = []
        for npass in range(1, o.max_scf + 1):
            psi1, k = self.taylor(self.psi, 0.5 * (self.V0 + V1) + ebar)
            terms.append(k)
            Vnew, aux = self.potential(psi1)
            err = float(np.max(np.abs(Vnew - V1)))
            V1 = Vnew
            if err <= o.H_thrs:
                break
        else:
            raise RuntimeError(f"SCF loop exceeded {o.max_scf} passes")
        self.psi = self.orthonormalize(psi1)
        self.Vm1, self.V0 = self.V0, V1
        self.aux = aux
        self.t += dt
        return {"passes": npass, "terms": terms, "V_err": err}

    # --- observables -----------------------------------------------------------------
    def dipole(self) -> np.ndarray:
        rho = self.density(self.psi)
        return np.array([self.h3 * float(np.dot(q, rho)) for q in self.q])

    def energy(self) -> float:
        """Energy of the current orbitals (the fields re-evaluated from their density)."""
        _, aux = self.potential(self.psi)
        hpsi = ham.apply_h(self.sys, self.v_ion, self.psi, self.projs)
        e = float(np.real(np.sum(self.f * np.sum(self.psi.conj() * hpsi, axis=1)))) * self.h3
        e += 0.5 * self.h3 * float(np.dot(aux["rho"], aux["vh"]))
        e += self.h3 * float(np.dot(aux["rho"] + self.rho_core, aux["exc"]))
        return e + self.E_ion

    def electrons(self) -> float:
        return self.h3 * float(np.sum(self.density(self.psi)))


def run(sys, psi0, f, opts, nsteps: int, axis: int = 2, kappa: float = 0.0, field=None,
        energies: bool = True):
    """Kick along `axis` and propagate on the grid; per-step dipole (and energy)."""
    gp = GridPropagator(sys, psi0, f, opts, field=field)
    if kappa != 0.0:
        gp.kick(axis, kappa)
    out = {"t": [0.0], "dipole": [gp.dipole()], "energy": [gp.energy()] if energies else [],
           "electrons": [gp.electrons()], "passes": [], "terms": []}
    for _ in range(nsteps):
        st = gp.step()
        out["t"].append(gp.t)
        out["dipole"].append(gp.dipole())
        if energies:
            out["energy"].append(gp.energy())
        out["electrons"].append(gp.electrons())
        out["passes"].append(st["passes"])
        out["terms"].append(st["terms"])
    for key in ("t", "dipole", "energy", "electrons"):
        out[key] = np.array(out[key])
    out["propagator"] = gp
    return out
