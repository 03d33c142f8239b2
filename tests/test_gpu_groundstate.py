"""Ground state on the GPU (Algorithm 1's ground state; option ground_state_scf) against the
oracle's SCF ground state (ARPACK eigenpairs, Pulay mixing), and the N_virt study (Section
4.1: the spectrum's convergence with the number of virtual orbitals) against the
complete-grid-basis propagation.

* Two-well system (N = 16): the 16 orbital energies within 1e-6 Ha and the density within 1e-6
  of its maximum; H_0 in the new basis is diag(eps) (P_0 = diag(f) is stationary).
* Harmonic oscillator (independent electrons): eps_0 = 3w/2 and the triply degenerate 5w/2.
* Ring on a ragged grid with s-type KB projectors (N = 25).
* N_virt study: kicked two-well trajectories with 3, 15 and 47 virtual orbitals of the GPU
  ground state approach the grid-basis propagation of its occupied orbital.
"""
import dataclasses

import numpy as np
import pytest

from oracle import groundstate
from paper_2410_09189_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    from paper_2410_09189_gb300 import rmgtd
    return rmgtd


def _raw(s):
    return inputs.smooth_random_orbitals(s).reshape(s.N, s.Ng)


def test_two_well_ground_state_matches_oracle(lib, small_ground_state):
    rmgtd = lib
    s, gs = small_ground_state
    with rmgtd.Context(s, _raw(s), ground_state_scf=300, ground_state_tol=1e-9) as ctx:
        it, drho, res, eps = ctx.ground_state_info()
        rho = ctx.density(0)
        H0 = ctx.get_matrix(rmgtd.MAT_H0, 0)
    assert drho <= 1e-9 and res <= 1e-9, (it, drho, res)
    assert np.max(np.abs(eps - gs["eps"])) < 1e-6, np.max(np.abs(eps - gs["eps"]))
    assert np.max(np.abs(rho - gs["rho"])) < 1e-6 * np.max(gs["rho"])
    assert np.max(np.abs(H0 - np.diag(np.diag(H0)))) < 1e-6
    assert np.max(np.abs(np.diag(H0) - eps)) < 1e-6


def test_harmonic_ground_state_levels(lib):
    rmgtd = lib
    s = inputs.harmonic(n=32, h=0.4, omega=0.5, nvirt=3)
    w = s.v_ext_omega
    with rmgtd.Context(s, _raw(s), ground_state_scf=200, ground_state_tol=1e-9) as ctx:
        _, _, _, eps = ctx.ground_state_info()
    assert abs(eps[0] - 1.5 * w) < 1e-6
    assert np.all(np.abs(eps[1:4] - 2.5 * w) < 1e-6)


def test_ring_ground_state_with_projectors_matches_oracle(lib):
    rmgtd = lib
    s = dataclasses.replace(inputs.ring(n=32, h=0.6, nvirt=10), n=(20, 22, 24))
    assert s.nproj > 0
    ref = groundstate.ground_state(s, tol=1e-10)
    with rmgtd.Context(s, _raw(s), ground_state_scf=300, ground_state_tol=1e-9) as ctx:
        it, drho, res, eps = ctx.ground_state_info()
        rho = ctx.density(0)
    assert np.max(np.abs(eps - ref["eps"])) < 1e-6, np.max(np.abs(eps - ref["eps"]))
    assert np.max(np.abs(rho - ref["rho"])) < 1e-6 * np.max(ref["rho"])


def test_virtual_orbital_count_converges_to_the_grid_basis(lib):
    """The dipole after a z kick, over 20 steps, with N_virt = 3, 15, 47 virtual orbitals of
    the GPU ground state, against the grid-basis propagation of the same occupied orbital:
    the error falls as N_virt grows (the active space approaches the complete basis)."""
    rmgtd = lib
    base = inputs.small()
    nsteps, dt, kap = 20, 0.05, 5e-2
    kw = dict(dt=dt, H_thrs=1e-10, dP_thrs=1e-12, poisson_tol=1e-13, ground_state_scf=300,
              ground_state_tol=1e-9)

    def run(s, **extra):
        with rmgtd.Context(s, _raw(s), **kw, **extra) as ctx:
            ctx.kick(0, 2, kap)
            d = [ctx.dipole(0)[2]]
            for _ in range(nsteps):
                ctx.step(1)
                d.append(ctx.dipole(0)[2])
        return np.array(d)

    ref = run(dataclasses.replace(base, nvirt=0), grid_basis=True)
    scale = np.max(np.abs(ref - ref[0]))
    errs = [np.max(np.abs(run(dataclasses.replace(base, nvirt=nv)) - ref)) / scale
            for nv in (3, 15, 47)]
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 0.3 * errs[0], errs
