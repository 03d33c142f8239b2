"""Algorithm 1 of the paper (RT-TDDFT density-matrix propagation), step by step in float64.

Active space: the N = N_occ + N_virt orbitals Phi (rows of ``phi``, grid-normalised), so
the overlap is the identity and the orthogonal commutator expansion applies (Section 3.1).

* Matrices (Algorithm 1's set-up): H_ij = h^3 <phi_i|H|phi_j>, M_q,ij = h^3 <phi_i|q|phi_j>,
  q measured from the box centre.  H is real symmetric at Gamma (Eq. 35 discussion); the
  oracle symmetrises it, (H + H^T)/2, so both sides see the same real symmetric matrix.
* P_0 = diag(f), f = 2 occupied / 0 virtual.  H_0 = H[rho(P_0)], H_-1 = H_0 (the set-up).
* Kick (Eq. 34 with a delta envelope): applied at t = 0+ as P <- e^{-i kappa M_q} P e^{i kappa M_q},
  evaluated with the same commutator expansion (Omega = -i kappa M_q); no field afterwards.
* Step j (the time loop), with Omega = -i dt (H_0 + H_1)/2 (Eq. 15, first-order Magnus):
    H_1 <- 2 H_0 - H_-1                                   (linear extrapolation)
    repeat:                                               (Hamiltonian SCF loop)
        P_1 <- P_0 + sum_k dP_k,  dP_0 = P_0,
        dP_k = (Omega dP_{k-1} + dP_{k-1} Omega^dagger)/k  (Eq. 33, the commutator series)
        stop the series when max_ij |dP_k| <= dP_thrs
        H_new <- DFT(rho(P_1)); H_err = max_ij |H_new - H_1|; H_1 <- H_new
    until H_err <= H_thrs
    H_-1 <- H_0, H_0 <- H_1, P_0 <- P_1                   (the shift)
  Reading of the loop order: the paper computes H_err before the update and never defines
  H_1^old on the first pass; here H_err compares the Hamiltonian the propagation used with
  the one its density produces, and a pass is one DFT evaluation.
* Time-dependent external field E(t) (optional): the external potential enters Omega through
  V_{j-1} + V_j, its values at both ends of the step (Algorithm 1's Omega assignment), i.e.
  Omega = -i dt ((H_0 + H_1)/2 + sum_q (E_q(t_j) + E_q(t_j + dt))/2 M_q); a field
  kappa delta(t) along q is the kick along q.
* Second-order Magnus term (option ``magnus2``, Section 2.2): with H linear in time over the
  step, Omega_2 = (dt^2/12)[H_0, H_1] (hbar = 1), each H with the field's value at its end,
  is added to Omega; Omega stays anti-Hermitian and the same series applies.
* Non-orthogonal basis (option ``nonorthogonal``, Section 2.2 and Appendix A.2): Phi is used
  as given, S = h^3 Phi Phi^T, Omega = -i dt S^-1 (Hbar + V), so that the series is
  dP_k = (1/k)(-i dt)(S^-1 Hbar dP_{k-1} - dP_{k-1} Hbar S^-1); the kick uses S^-1 M_q; the
  start is P = L^-T diag(f) L^-1 (S = L L^T: the occupations on the Cholesky-orthonormalised
  orbitals); the electron count is Tr(Re P S).
* rho(P)(r) = sum_ij Re(P)_ij phi_i(r) phi_j(r) (the density of P = sum f |psi><psi|; the
  imaginary part of a Hermitian P cancels).
* DFT(rho): Hartree by ``poisson.hartree``, LDA by ``lda.lda``, then
  H = h^3 Phi (H[rho] Phi^T) with the *full* grid Hamiltonian applied to every orbital.
* Observables: electronic dipole d_q = Tr(Re(P) M_q) (Algorithm 1's dipole without mu_0), and
  E = Tr(Re(P) H_core) + 1/2 h^3 sum rho V_H + h^3 sum rho eps_xc + E_ion.
* Frozen core density rho_core (optional, ``sys.rho_core``; Section 3.1's frozen semicore
  electrons): a fixed density added to rho in the exchange-correlation only, V_xc and eps_xc
  of rho + rho_core and E_xc = h^3 sum (rho + rho_core) eps_xc; the Hartree potential, the
  dipole and Tr P see rho alone.

Pinned by: the two-level closed form of the kicked harmonic oscillator, the spectral
propagator W exp(omega) W^dagger (Section 2.2), Tr(P) conservation, energy conservation,
the time-domain Thomas-Reiche-Kuhn slope, the linear response to a weak field, the global
order (2 and 4) of the Magnus truncations against an independent ODE integration, and the
non-orthogonal series against the orthonormalised basis (Appendix A.2).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np
from scipy.linalg import eigh as _eigh

from . import hamiltonian as ham
from .lda import lda
from .poisson import hartree


class NotConverged(RuntimeError):
    pass


@dataclasses.dataclass
class Options:
    dt: float = 0.05
    H_thrs: float = 1e-7
    dP_thrs: float = 1e-10
    max_scf: int = 50
    max_terms: int = 200
    poisson_tol: float = 1e-13
    full_apply: bool = True
    magnus2: bool = False        # add Omega_2 = (dt^2/12)[H_0, H_1] (Section 2.2)
    nonorthogonal: bool = False  # propagate in the given basis with S^-1 H (Section 2.2)


def commutator_series(P0: np.ndarray, Hbar: np.ndarray, tau: float, thrs: float,
                      max_terms: int = 200):
    """P = e^{-i tau Hbar} P0 e^{+i tau Hbar} by the series of Eq. 33; returns (P, terms)."""
    return omega_series(P0, -1j * tau * Hbar, thrs, max_terms)


def omega_series(P0: np.ndarray, Omega: np.ndarray, thrs: float, max_terms: int = 200):
    """P = e^{Omega} P0 e^{Omega^dagger} as P0 + sum_k dP_k, dP_k = (Omega dP_{k-1} +
    dP_{k-1} Omega^dagger)/k, dP_0 = P0 (Eq. 33; with Omega = -i dt S^-1 Hbar the series of the
    non-orthogonal basis, Section 2.2); stops at max|dP_k| <= thrs.  Returns (P, terms)."""
    OmegaH = Omega.conj().T
    P = P0.astype(np.complex128).copy()
    dP = P.copy()
    k = 0
    err = 2.0 * thrs
    while err > thrs:
        k += 1
        if k > max_terms:
            raise NotConverged(f"commutator series exceeded {max_terms} terms")
        dP = (Omega @ dP + dP @ OmegaH) / k
        P += dP
        err = float(np.max(np.abs(dP)))
        if not np.isfinite(err):
            raise NotConverged("commutator series diverged")
    return P, k


def spectral_propagate(P0: np.ndarray, Hbar: np.ndarray, tau: float) -> np.ndarray:
    """Exact U P0 U^dagger with U = W exp(-i tau w) W^T from the eigenpairs of Hbar."""
    w, W = _eigh(Hbar)
    U = (W * np.exp(-1j * tau * w)) @ W.T
    return U @ P0 @ U.conj().T


class Propagator:
    """Algorithm 1 in a fixed orthonormal basis ``phi`` of shape (N, Ng)."""

    def __init__(self, sys, phi: np.ndarray, opts: Optional[Options] = None, field=None):
        self.sys = sys
        self.field = field      # None or t -> (E_x, E_y, E_z)
        self.opts = opts or Options()
        self.phi = np.ascontiguousarray(phi, dtype=np.float64)
        self.h3 = sys.h ** 3
        self.shape = (sys.n[2], sys.n[1], sys.n[0])
        self.projs = ham.projectors(sys)
        self.v_ion = (ham.v_local(sys) + ham.v_external(sys)).ravel()
        hphi = ham.apply_h(sys, self.v_ion, self.phi, self.projs)
        self.Hcore = self._sym(self.h3 * (self.phi @ hphi.T))
        self.M = [self._sym(self.h3 * (self.phi @ (q.ravel() * self.phi).T))
                  for q in ham.full_coords(sys)]
        self.E_ion = ham.ion_energy(sys)
        self.vh = None
        # overlap S = h^3 Phi Phi^T; the identity in an orthonormal basis
        self.S = self._sym(self.h3 * (self.phi @ self.phi.T))
        self.Sinv = np.linalg.inv(self.S) if self.opts.nonorthogonal else None
        core = getattr(sys, "rho_core", None)
        self.rho_core = np.zeros(sys.Ng) if core is None else np.asarray(core, float).ravel()

    @staticmethod
    def _sym(A):
        return 0.5 * (A + A.T)

    # --- Algorithm 1 building blocks -------------------------------------------------
    def density(self, P: np.ndarray) -> np.ndarray:
        X = np.real(P) @ self.phi
        return np.sum(self.phi * X, axis=0)

    def dft(self, P: np.ndarray):
        """H_1 <- DFT(rho(P)) (the density-functional update); also returns the grid fields for observables."""
        rho = self.density(P)
        if self.sys.hartree_xc:
            vh = hartree(self.sys, rho.reshape(self.shape), tol=self.opts.poisson_tol,
                         x0=self.vh).ravel()
            self.vh = vh
            vxc, exc = lda(rho + self.rho_core)   # the frozen core enters the xc only
        else:
            vh = np.zeros_like(rho)
            vxc = np.zeros_like(rho)
            exc = np.zeros_like(rho)
        v_hxc = vh + vxc
        if self.opts.full_apply:
            hphi = ham.apply_h(self.sys, self.v_ion + v_hxc, self.phi, self.projs)
            H = self._sym(self.h3 * (self.phi @ hphi.T))
        else:
            H = self.Hcore + self._sym(self.h3 * (self.phi @ (v_hxc * self.phi).T))
        return H, {"rho": rho, "vh": vh, "vxc": vxc, "exc": exc, "v_hxc": v_hxc}

    def expand(self, P0, Hbar, tau):
        return commutator_series(P0, Hbar, tau, self.opts.dP_thrs, self.opts.max_terms)

    def kick(self, P, axis: int, kappa: float):
        Omega = -1j * kappa * self._metric(self.M[axis])
        P1, _ = omega_series(P, Omega, self.opts.dP_thrs, self.opts.max_terms)
        return P1

    def _metric(self, A):
        """S^-1 A in the non-orthogonal basis, A otherwise."""
        return self.Sinv @ A if self.opts.nonorthogonal else A

    def trace(self, P) -> float:
        """Number of electrons Tr(Re P S) (Tr P in an orthonormal basis)."""
        return float(np.trace(np.real(P) @ self.S)) if self.opts.nonorthogonal else \
            float(np.real(np.trace(P)))

    def dipole(self, P) -> np.ndarray:
        return np.array([np.trace(np.real(P) @ M) for M in self.M])

    def energy(self, P, aux) -> float:
        e = float(np.trace(np.real(P) @ self.Hcore))
        e += 0.5 * self.h3 * float(np.dot(aux["rho"], aux["vh"]))
        e += self.h3 * float(np.dot(aux["rho"] + self.rho_core, aux["exc"]))
        return e + self.E_ion

    # --- driver ----------------------------------------------------------------------
    def subspace_ground_state(self, iters: int, mix: float = 0.3, tol: float = 1e-10):
        """SCF inside the orbital block: P <- (1-mix) P + mix P_aufbau(H[rho(P)]).

        P_aufbau = sum_n f_n w_n w_n^T over the eigenvectors of H in ascending order
        (scipy eigh), i.e. the ground-state density matrix of Algorithm 1's set-up restricted
        to the active space.  Returns (P, H, aux, iterations, last max|P_new - P|).
        """
        f = self.sys.occupations
        P = np.diag(f).astype(np.float64)
        H, aux = self.dft(P)
        err, it = np.inf, 0
        for it in range(1, iters + 1):
            w, W = _eigh(H)
            Pn = (W * f) @ W.T
            err = float(np.max(np.abs(Pn - P)))
            P = (1.0 - mix) * P + mix * Pn
            H, aux = self.dft(P)
            if err <= tol:
                break
        return P, H, aux, it, err

    def initial_state(self, subspace_scf: int = 0, mix: float = 0.3, tol: float = 1e-10):
        if subspace_scf > 0:
            if self.opts.nonorthogonal:
                raise ValueError("the subspace ground state needs an orthonormal basis")
            P, H0, aux, _, _ = self.subspace_ground_state(subspace_scf, mix, tol)
            P0 = P.astype(np.complex128)
        elif self.opts.nonorthogonal:
            # occupations on the Cholesky-orthonormalised orbitals L^-1 Phi (S = L L^T):
            # P = L^-T diag(f) L^-1, the back transformation R^-1 P_o L^-1 of Appendix A.2
            X = np.linalg.inv(np.linalg.cholesky(self.S))
            P0 = (X.T @ np.diag(self.sys.occupations) @ X).astype(np.complex128)
            H0, aux = self.dft(P0)
        else:
            f = self.sys.occupations
            P0 = np.diag(f).astype(np.complex128)
            H0, aux = self.dft(P0)
        return {"P0": P0, "H0": H0, "Hm1": H0.copy(), "aux": aux, "t": 0.0, "j": 0}

    def field_term(self, t: float) -> np.ndarray:
        """sum_q (E_q(t) + E_q(t + dt))/2 M_q for the step starting at t (zero without a field)."""
        if self.field is None:
            return np.zeros_like(self.Hcore)
        return 0.5 * (self.field_at(t) + self.field_at(t + self.opts.dt))

    def field_at(self, t: float) -> np.ndarray:
        """sum_q E_q(t) M_q (zero without a field)."""
        if self.field is None:
            return np.zeros_like(self.Hcore)
        e = np.asarray(self.field(t), dtype=float)
        return sum(e[q] * self.M[q] for q in range(3))

    def omega(self, H0, H1, t: float) -> np.ndarray:
        """Omega of the step from t to t + dt with H changing linearly from H_0 to H_1 (the
        field's values at both ends added): Omega_1 = -i dt (H_0 + H_1)/2 (S^-1 in front in
        the non-orthogonal basis), plus Omega_2 = (dt^2/12)[H_0, H_1] with the magnus2
        option (Section 2.2)."""
        dt = self.opts.dt
        Om = -1j * dt * self._metric(0.5 * (H0 + H1) + self.field_term(t))
        if self.opts.magnus2:
            if self.opts.nonorthogonal:
                raise ValueError("Omega_2 is implemented for an orthonormal basis only")
            A = H0 + self.field_at(t)
            B = H1 + self.field_at(t + dt)
            Om = Om + (dt * dt / 12.0) * (A @ B - B @ A)
        return Om

    def step(self, st):
        o = self.opts
        P0, H0, Hm1 = st["P0"], st["H0"], st["Hm1"]
        H1 = 2.0 * H0 - Hm1
        terms = []
        for npass in range(1, o.max_scf + 1):
            P1, k = omega_series(P0, self.omega(H0, H1, st["t"]), o.dP_thrs, o.max_terms)
            terms.append(k)
            Hnew, aux = self.dft(P1)
            err = float(np.max(np.abs(Hnew - H1)))
            H1 = Hnew
            if err <= o.H_thrs:
                break
        else:
            raise NotConverged(f"SCF loop exceeded {o.max_scf} passes")
        st["Hm1"], st["H0"], st["P0"], st["aux"] = H0, H1, P1, aux
        st["t"] += o.dt
        st["j"] += 1
        return {"passes": npass, "terms": terms, "H_err": err}


def run(sys, phi, opts: Optional[Options] = None, nsteps: int = 10, axis: int = 2,
        kappa: Optional[float] = None, subspace_scf: int = 0, subspace_mix: float = 0.3,
        field=None):
    """Kick along `axis` and propagate (in the external field `field(t)` if given); returns
    per-step dipole, energy, trace, stats."""
    pr = Propagator(sys, phi, opts, field=field)
    st = pr.initial_state(subspace_scf, subspace_mix)
    kap = sys.kappa if kappa is None else kappa
    out = {"dipole_gs": pr.dipole(st["P0"]), "energy_gs": pr.energy(st["P0"], st["aux"])}
    if kap != 0.0:
        st["P0"] = pr.kick(st["P0"], axis, kap)
    _, aux0 = pr.dft(st["P0"])          # observables at t = 0+ (state H_0 is unchanged)
    out.update({"t": [0.0], "dipole": [pr.dipole(st["P0"])],
                "energy": [pr.energy(st["P0"], aux0)],
                "trace": [pr.trace(st["P0"])], "passes": [], "terms": []})
    for _ in range(nsteps):
        s = pr.step(st)
        out["t"].append(st["t"])
        out["dipole"].append(pr.dipole(st["P0"]))
        out["energy"].append(pr.energy(st["P0"], st["aux"]))
        out["trace"].append(pr.trace(st["P0"]))
        out["passes"].append(s["passes"])
        out["terms"].append(s["terms"])
    for key in ("t", "dipole", "energy", "trace"):
        out[key] = np.array(out[key])
    out["propagator"] = pr
    out["state"] = st
    return out
