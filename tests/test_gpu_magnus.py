"""The second-order Magnus term, the non-orthogonal basis and the strength function on the GPU
against the oracle.

* Omega_2 = (dt^2/12)[H_0 + V_0, H_1 + V_1] (Section 2.2): replica 0 driven by a field pulse
  (its end values enter Omega_2), replica 1 kicked; the two-well system (N = 16, cluster
  commutator kernel) and a ragged ring grid (N = 70, cooperative kernel).  At dt = 0.1 the
  pulse's dipole moves by ~2e-3 of its variation when Omega_2 is dropped, well above both
  tolerances (1e-6 float64, 1e-4 mixed).
* Non-orthogonal basis (Section 2.2, Appendix A.2): raw smooth orbitals (S far from I),
  replica 0 kicked, replica 1 in a pulse; dipole, energy and Tr(P S) against the oracle's
  S^-1 series.
* rmgtd_spectrum against the oracle's strength function (float64, 1e-11 of the peak).
"""
import dataclasses
import math

import numpy as np
import pytest

from oracle import hamiltonian as oham, spectrum as ospectrum, tddft
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


def _pulse(E0, W, t0, tau, axis):
    def f(t):
        e = np.zeros(3)
        e[axis] = E0 * math.sin(W * t) * math.exp(-((t - t0) / tau) ** 2)
        return e
    return f


def _rel(d, ref):
    return float(np.max(np.abs(d - ref)) / np.max(np.abs(ref - ref[0])))


def _case(name, small_ground_state):
    if name == "two-well-N16":
        s, gs = small_ground_state
        return s, gs["phi"], gs["phi"], False
    s = dataclasses.replace(inputs.ring(n=32, h=0.6, nvirt=55), n=(20, 22, 24))
    raw = inputs.smooth_random_orbitals(s).reshape(s.N, s.Ng)
    return s, raw, oham.orthonormalize(s, raw), True


def _run_gpu(rmgtd, s, raw, prec, ortho, nsteps, dt, fields, kicks, **kw):
    H_thrs, dP_thrs = (1e-10, 1e-13) if prec == rmgtd.PREC_FP64 else (1e-8, 1e-11)
    with rmgtd.Context(s, raw, dt=dt, H_thrs=H_thrs, dP_thrs=dP_thrs, poisson_tol=1e-13,
                       nrep=2, precision=prec, orthonormalize=ortho, **kw) as ctx:
        for r, f in fields.items():
            ctx.set_field(r, np.array([f(j * dt) for j in range(nsteps + 1)]))
        for r, (axis, kap) in kicks.items():
            ctx.kick(r, axis, kap)
        S = ctx.get_matrix(rmgtd.MAT_S, 0)
        d = [[ctx.dipole(r) for r in range(2)]]
        e = [[ctx.energy(r) for r in range(2)]]
        tr = [[float(np.sum(ctx.get_matrix(rmgtd.MAT_P_RE, r) * S)) for r in range(2)]]
        for _ in range(nsteps):
            ctx.step(1)
            d.append([ctx.dipole(r) for r in range(2)])
            e.append([ctx.energy(r) for r in range(2)])
            tr.append([float(np.sum(ctx.get_matrix(rmgtd.MAT_P_RE, r) * S)) for r in range(2)])
    return np.array(d), np.array(e), np.array(tr)


@pytest.mark.parametrize("case", ["two-well-N16", "ring-N70"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_omega2_trajectory_matches_oracle(lib, small_ground_state, case, precision):
    rmgtd = lib
    s, raw, phi, ortho = _case(case, small_ground_state)
    nsteps, dt = 15, 0.1
    field = _pulse(0.1, 0.9, 0.6, 0.4, 2)
    o2 = tddft.Options(dt=dt, H_thrs=1e-10, dP_thrs=1e-13, poisson_tol=1e-13, magnus2=True)
    o1 = dataclasses.replace(o2, magnus2=False)
    ref_f = tddft.run(s, phi, o2, nsteps=nsteps, kappa=0.0, field=field)["dipole"]
    ref_k = tddft.run(s, phi, o2, nsteps=nsteps, axis=1, kappa=2e-2)["dipole"]
    # the test can see Omega_2: dropping it moves the driven dipole by far more than the
    # float64 bound (and by 4e-4 to 2e-3 of the variation, beyond the mixed bound too)
    no2 = tddft.run(s, phi, o1, nsteps=nsteps, kappa=0.0, field=field)["dipole"]
    tol = 1e-6 if precision == "fp64" else 1e-4
    assert _rel(no2, ref_f) > 100 * 1e-6
    prec = rmgtd.PREC_FP64 if precision == "fp64" else rmgtd.PREC_MIXED
    d, _, _ = _run_gpu(rmgtd, s, raw, prec, ortho, nsteps, dt, {0: field}, {1: (1, 2e-2)},
                       magnus_order=2)
    assert _rel(d[:, 0], ref_f) < tol, _rel(d[:, 0], ref_f)
    assert _rel(d[:, 1], ref_k) < tol, _rel(d[:, 1], ref_k)


@pytest.mark.parametrize("case", ["two-well-N16", "ring-N70"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nonorthogonal_trajectory_matches_oracle(lib, small_ground_state, case, precision):
    rmgtd = lib
    s, _, phi_o, _ = _case(case, small_ground_state)
    if case == "two-well-N16":
        raw = inputs.smooth_random_orbitals(s).reshape(s.N, s.Ng)   # cond(S) = 37
    else:
        # the ring's raw smooth orbitals have cond(S) = 5.4e3, which the mixed path's float32 /
        # bfloat16-split rounding does not survive; a mixed orthonormal basis, B Phi_o with
        # B = I + 0.25 G / sqrt(N), is non-orthogonal with cond(S) = 3.7
        rng = np.random.default_rng(7)
        B = np.eye(s.N) + 0.25 * rng.standard_normal((s.N, s.N)) / math.sqrt(s.N)
        raw = B @ phi_o
    nsteps, dt = 12, 0.05
    field = _pulse(0.05, 0.6, 0.3, 0.3, 0)
    o = tddft.Options(dt=dt, H_thrs=1e-10, dP_thrs=1e-13, poisson_tol=1e-13, nonorthogonal=True)
    ref_k = tddft.run(s, raw, o, nsteps=nsteps, axis=2, kappa=1e-2)
    ref_f = tddft.run(s, raw, o, nsteps=nsteps, kappa=0.0, field=field)
    assert np.max(np.abs(ref_k["propagator"].S - np.eye(s.N))) > 0.1
    prec = rmgtd.PREC_FP64 if precision == "fp64" else rmgtd.PREC_MIXED
    d, e, tr = _run_gpu(rmgtd, s, raw, prec, False, nsteps, dt, {1: field}, {0: (2, 1e-2)},
                        nonorthogonal=True)
    tol = 1e-6 if precision == "fp64" else 1e-4
    vh0 = ref_k["propagator"].initial_state()["aux"]["vh"]
    for r, ref in ((0, ref_k), (1, ref_f)):
        assert _rel(d[:, r], ref["dipole"]) < tol, (r, _rel(d[:, r], ref["dipole"]))
        # mixed: the float32 Hartree correction is solved to 3e-6 of dV_H = V_H - V_H(0), which
        # this strongly non-stationary start makes O(0.1-1); the energy error is bounded by
        # 10 x 3e-6 x h^3 sum rho |dV_H| (the last step's fields)
        aux = ref["state"]["aux"]
        dvh = ref["propagator"].h3 * float(np.sum(aux["rho"] * np.abs(aux["vh"] - vh0)))
        etol = 1e-9 if precision == "fp64" else 10 * 3e-6 * dvh
        assert np.max(np.abs(e[:, r] - ref["energy"])) < etol
        assert np.max(np.abs(tr[:, r] - ref["trace"])) < 1e-9


def test_nonorthogonal_requires_a_plain_propagation(lib, small_ground_state):
    rmgtd = lib
    s, gs = small_ground_state
    with pytest.raises(rmgtd.RmgtdError) as ei:
        rmgtd.Context(s, gs["phi"], nonorthogonal=True, magnus_order=2)
    assert ei.value.code == rmgtd.EINVAL


@pytest.mark.parametrize("nq,nt,nw", [(3, 4097, 777), (1, 2, 5), (2, 40001, 1201)])
def test_spectrum_matches_oracle(lib, nq, nt, nw):
    rmgtd = lib
    rng = np.random.default_rng(nt + nw)
    dt, kappa, gamma = 0.05, 1e-3, 0.02
    t = dt * np.arange(nt)
    d = np.array([rng.standard_normal() * 1e-3
                  + sum(rng.standard_normal() * 1e-4 * np.sin(w * t) for w in (0.3, 0.71, 1.9))
                  for _ in range(nq)])
    omega = np.sort(rng.uniform(0.0, 4.0, nw))
    S = rmgtd.spectrum(d, dt, kappa, gamma, omega)
    ref = ospectrum.strength_function(d, dt, kappa, gamma, omega)
    scale = max(np.max(np.abs(ref)), 1e-300)
    assert np.max(np.abs(S - ref)) <= 1e-11 * scale + 1e-300
    with pytest.raises(rmgtd.RmgtdError):
        rmgtd.spectrum(d, 0.0, kappa, gamma, omega)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_quadratic_seed_converges_to_the_same_trajectory(lib, small_ground_state, precision):
    """seed_order 2 (H_1 = 3 H_0 - 3 H_-1 + H_-2) changes only the SCF loop's starting point:
    the kicked trajectory matches the oracle's (linear seed, Algorithm 1's extrapolation) within the
    same bounds."""
    rmgtd = lib
    s, gs = small_ground_state
    nsteps, dt = 16, 0.05
    o = tddft.Options(dt=dt, H_thrs=1e-10, dP_thrs=1e-13, poisson_tol=1e-13)
    ref = tddft.run(s, gs["phi"], o, nsteps=nsteps, axis=2, kappa=1e-2)["dipole"]
    prec = rmgtd.PREC_FP64 if precision == "fp64" else rmgtd.PREC_MIXED
    H_thrs, dP_thrs = (1e-10, 1e-13) if precision == "fp64" else (1e-8, 1e-11)
    with rmgtd.Context(s, gs["phi"], dt=dt, H_thrs=H_thrs, dP_thrs=dP_thrs, poisson_tol=1e-13,
                       precision=prec, orthonormalize=False, seed_order=2) as ctx:
        ctx.kick(0, 2, 1e-2)
        d = [ctx.dipole(0)]
        for _ in range(nsteps):
            ctx.step(1)
            d.append(ctx.dipole(0))
    tol = 1e-6 if precision == "fp64" else 1e-4
    assert _rel(np.array(d), ref) < tol, _rel(np.array(d), ref)
