"""Propagation of the occupied orbitals on the grid (the complete-grid-basis limit, Section
2.2) on the GPU against the oracle's grid propagation.

* Two-well system (one occupied orbital, 24^3): replica 0 kicked along z, replica 1 driven
  by a field pulse along x; dipole within 1e-6 of its variation and energy 1e-9 on the float64
  path, 1e-4 and 1e-6 of |E| with float32 series terms (mixed).
* Ring on a ragged 20 x 22 x 24 grid (15 occupied orbitals, s-type KB projectors), kicked
  along x.
* The quadratic potential seed (seed_order 2) against the oracle's linear one.
* A series cap that cannot be met reports RMGTD_ENOTCONVERGED and keeps the state; the
  matrix calls are refused on a grid-basis context.
"""
import dataclasses
import math

import numpy as np
import pytest

from oracle import gridprop as ogrid, hamiltonian as oham, tddft
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


def _pulse(t):
    return np.array([0.04 * math.sin(0.8 * t) * math.exp(-((t - 0.3) / 0.25) ** 2), 0.0, 0.0])


def _rel(d, ref):
    return float(np.max(np.abs(d - ref)) / np.max(np.abs(ref - ref[0])))


def _gpu_run(rmgtd, s, psi0, nsteps, dt, kicks, fields, nrep, precision="fp64", **kw):
    prec = rmgtd.PREC_FP64 if precision == "fp64" else rmgtd.PREC_MIXED
    # the float32 terms leave ~1e-8 of noise in V: the mixed SCF stops above it
    H_thrs = 1e-10 if precision == "fp64" else 1e-8
    with rmgtd.Context(s, psi0, dt=dt, H_thrs=H_thrs, dP_thrs=1e-12, poisson_tol=1e-13,
                       nrep=nrep, grid_basis=True, orthonormalize=False, precision=prec,
                       **kw) as ctx:
        for r, (axis, kap) in kicks.items():
            ctx.kick(r, axis, kap)
        for r, f in fields.items():
            ctx.set_field(r, np.array([f(j * dt) for j in range(nsteps + 1)]))
        d = [[ctx.dipole(r) for r in range(nrep)]]
        e = [[ctx.energy(r) for r in range(nrep)]]
        for _ in range(nsteps):
            ctx.step(1)
            d.append([ctx.dipole(r) for r in range(nrep)])
            e.append([ctx.energy(r) for r in range(nrep)])
    return np.array(d), np.array(e)


# float64 path: dipole 1e-6 of its variation, energy 1e-9; mixed path (float32 series terms):
# dipole 1e-4, energy 1e-6 of |E|
_TOL = {"fp64": (1e-6, None), "mixed": (1e-4, 1e-6)}


def _etol(precision, ref):
    rel = _TOL[precision][1]
    return 1e-9 if rel is None else rel * np.max(np.abs(ref["energy"]))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_two_well_grid_propagation_matches_oracle(lib, small_ground_state, precision):
    rmgtd = lib
    s, gs = small_ground_state
    s1 = dataclasses.replace(s, nvirt=0)
    psi0 = gs["phi"][:s.nocc]
    f = s1.occupations
    nsteps, dt = 10, 0.05
    o = tddft.Options(dt=dt, H_thrs=1e-10, dP_thrs=1e-12, poisson_tol=1e-13)
    ref_k = ogrid.run(s1, psi0, f, o, nsteps=nsteps, axis=2, kappa=1e-2)
    ref_f = ogrid.run(s1, psi0, f, o, nsteps=nsteps, kappa=0.0, field=_pulse)
    d, e = _gpu_run(rmgtd, s1, psi0, nsteps, dt, {0: (2, 1e-2)}, {1: _pulse}, 2, precision)
    for r, ref in ((0, ref_k), (1, ref_f)):
        assert _rel(d[:, r], ref["dipole"]) < _TOL[precision][0], (r, _rel(d[:, r], ref["dipole"]))
        assert np.max(np.abs(e[:, r] - ref["energy"])) < _etol(precision, ref)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_ring_grid_propagation_with_projectors_matches_oracle(lib, precision):
    rmgtd = lib
    s = dataclasses.replace(inputs.ring(n=32, h=0.6, nvirt=0), n=(20, 22, 24))
    raw = inputs.smooth_random_orbitals(s).reshape(s.N, s.Ng)
    psi0 = oham.orthonormalize(s, raw)
    assert s.nproj > 0
    nsteps, dt = 5, 0.05
    o = tddft.Options(dt=dt, H_thrs=1e-10, dP_thrs=1e-12, poisson_tol=1e-13)
    ref = ogrid.run(s, psi0, s.occupations, o, nsteps=nsteps, axis=0, kappa=1e-2)
    d, e = _gpu_run(rmgtd, s, psi0, nsteps, dt, {0: (0, 1e-2)}, {}, 1, precision)
    assert _rel(d[:, 0], ref["dipole"]) < _TOL[precision][0], _rel(d[:, 0], ref["dipole"])
    assert np.max(np.abs(e[:, 0] - ref["energy"])) < _etol(precision, ref)


def test_grid_basis_failure_and_refusals(lib, small_ground_state):
    rmgtd = lib
    s, gs = small_ground_state
    s1 = dataclasses.replace(s, nvirt=0)
    psi0 = gs["phi"][:s.nocc]
    with rmgtd.Context(s1, psi0, grid_basis=True, orthonormalize=False, max_terms=3) as ctx:
        ctx.kick(0, 2, 1e-2)
        d0 = ctx.dipole(0)
        with pytest.raises(rmgtd.RmgtdError) as ei:
            ctx.step(1)
        assert ei.value.code == rmgtd.ENOTCONVERGED
        assert np.array_equal(ctx.dipole(0), d0)
        with pytest.raises(rmgtd.RmgtdError) as ei:
            ctx.get_matrix(rmgtd.MAT_P_RE, 0)
        assert ei.value.code == rmgtd.ESTATE
    with pytest.raises(rmgtd.RmgtdError) as ei:
        rmgtd.Context(s, gs["phi"], grid_basis=True, orthonormalize=False)   # nvirt > 0
    assert ei.value.code == rmgtd.EINVAL


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_quadratic_potential_seed_matches_oracle(lib, precision):
    """seed_order 2 (V_1 = 3 V_0 - 3 V_-1 + V_-2) moves only the SCF loop's starting point:
    the trajectory matches the oracle's (linear seed) within the same bounds."""
    rmgtd = lib
    s = dataclasses.replace(inputs.ring(n=32, h=0.6, nvirt=0), n=(20, 22, 24))
    raw = inputs.smooth_random_orbitals(s).reshape(s.N, s.Ng)
    psi0 = oham.orthonormalize(s, raw)
    nsteps, dt = 8, 0.05
    o = tddft.Options(dt=dt, H_thrs=1e-10, dP_thrs=1e-12, poisson_tol=1e-13)
    ref = ogrid.run(s, psi0, s.occupations, o, nsteps=nsteps, axis=2, kappa=2e-2)
    d, e = _gpu_run(rmgtd, s, psi0, nsteps, dt, {0: (2, 2e-2)}, {}, 1, precision, seed_order=2)
    assert _rel(d[:, 0], ref["dipole"]) < _TOL[precision][0], _rel(d[:, 0], ref["dipole"])
    assert np.max(np.abs(e[:, 0] - ref["energy"])) < _etol(precision, ref)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_ragged_grid_uses_the_plain_term_kernel(lib, precision):
    """x = 21 points: a row is not a whole number of 16-byte units, so the term kernel stages
    its tiles with plain loads instead of TMA; same bounds against the oracle."""
    rmgtd = lib
    s = dataclasses.replace(inputs.small(), n=(21, 22, 23), nvirt=0)
    raw = inputs.smooth_random_orbitals(s).reshape(s.N, s.Ng)
    psi0 = oham.orthonormalize(s, raw)
    nsteps, dt = 5, 0.05
    o = tddft.Options(dt=dt, H_thrs=1e-10, dP_thrs=1e-12, poisson_tol=1e-13)
    ref = ogrid.run(s, psi0, s.occupations, o, nsteps=nsteps, axis=1, kappa=2e-2)
    d, e = _gpu_run(rmgtd, s, psi0, nsteps, dt, {0: (1, 2e-2)}, {}, 1, precision)
    assert _rel(d[:, 0], ref["dipole"]) < _TOL[precision][0], _rel(d[:, 0], ref["dipole"])
    assert np.max(np.abs(e[:, 0] - ref["energy"])) < _etol(precision, ref)
