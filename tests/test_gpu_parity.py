"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element.

Tolerances (float64 path): grid operators and set-up matrices to 1e-10 relative (rounding
order of 37-term stencils and grid sums of up to 10^6 terms), Hartree to the CG tolerance,
dipole time series to 1e-6 of the dipole variation -- the target the method states for the
float64 path -- with the SCF and series thresholds tightened so that the iteration history
does not dominate.
"""
import dataclasses
import os
import tempfile

import numpy as np
import pytest

from oracle import groundstate, hamiltonian as oham, lda as olda, poisson as opoisson, tddft
from paper_2410_09189_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    return torch


def _rmgtd():
    from paper_2410_09189_gb300 import rmgtd
    return rmgtd


def _ring_small(n=(30, 34, 38), h=0.5, nvirt=15):
    s = inputs.ring(n=32, h=h, nvirt=nvirt)
    return dataclasses.replace(s, n=tuple(n))


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


# ----------------------------------------------------------------------------------------
def test_apply_h_all_dtypes(torch_dev):
    torch = torch_dev
    rmgtd = _rmgtd()
    s = _ring_small(n=(37, 41, 43), h=0.45)
    s.proj_l = s.proj_l.copy()
    s.proj_m = s.proj_m.copy()
    s.proj_l[1], s.proj_m[1] = 1, 2      # one p-type projector
    s.proj_l[4], s.proj_m[4] = 1, 0
    raw = inputs.smooth_random_orbitals(s).reshape(s.N, s.Ng)
    x = np.random.default_rng(5).standard_normal((3, s.Ng))
    v_ion = (oham.v_local(s) + oham.v_external(s)).ravel()
    ref = oham.apply_h(s, v_ion, x)
    with rmgtd.Context(s, raw) as ctx:
        xd = torch.from_numpy(x).cuda()
        hx = torch.empty_like(xd)
        ctx.apply_h(xd, hx, rep=-1)
        assert _rel(hx.cpu().numpy(), ref) < 1e-12
        x32 = xd.float()
        h32 = torch.empty_like(x32)
        ctx.apply_h(x32, h32, rep=-1)
        assert _rel(h32.double().cpu().numpy(), ref) < 2e-5
        y = np.random.default_rng(6).standard_normal((3, s.Ng))
        refy = oham.apply_h(s, v_ion, y)
        z = torch.complex(xd, torch.from_numpy(y).cuda()).contiguous()
        hz = torch.empty_like(z)
        ctx.apply_h(z, hz, rep=-1)
        got = hz.cpu().numpy()
        assert _rel(got.real, ref) < 1e-12 and _rel(got.imag, refy) < 1e-12
        z64 = z.to(torch.complex64)
        hz64 = torch.empty_like(z64)
        ctx.apply_h(z64, hz64, rep=-1)
        got = hz64.cpu().numpy()
        assert _rel(got.real, ref) < 2e-5 and _rel(got.imag, refy) < 2e-5


def test_setup_matrices(torch_dev):
    rmgtd = _rmgtd()
    s = _ring_small(n=(30, 34, 38), h=0.5, nvirt=22)     # N = 37: ragged against every tile
    raw = inputs.smooth_random_orbitals(s).reshape(s.N, s.Ng)
    phi = oham.orthonormalize(s, raw)
    pr = tddft.Propagator(s, phi, tddft.Options(poisson_tol=1e-13))
    st = pr.initial_state()
    with rmgtd.Context(s, raw, poisson_tol=1e-13) as ctx:
        S = ctx.get_matrix(rmgtd.MAT_S)
        assert np.max(np.abs(S - np.eye(s.N))) < 1e-12
        assert np.max(np.abs(ctx.get_matrix(rmgtd.MAT_HCORE) - pr.Hcore)) < 1e-10
        for q, which in enumerate((rmgtd.MAT_MX, rmgtd.MAT_MY, rmgtd.MAT_MZ)):
            assert np.max(np.abs(ctx.get_matrix(which) - pr.M[q])) < 1e-10
        H0 = ctx.get_matrix(rmgtd.MAT_H0)
        assert np.max(np.abs(H0 - st["H0"])) < 1e-9
        assert np.max(np.abs(H0 - H0.T)) == 0.0
        rho = ctx.density(0)
        assert _rel(rho, pr.density(st["P0"])) < 1e-12
        assert abs(ctx.energy(0) - pr.energy(st["P0"], st["aux"])) < 1e-9


@pytest.mark.parametrize("precond", ["dst", "mg"])
def test_hartree_and_xc(torch_dev, precond):
    """Hartree solve with either preconditioner (the operator and stopping test are the same)
    against the oracle's; the sine-transform preconditioner needs fewer CG iterations."""
    torch = torch_dev
    rmgtd = _rmgtd()
    s = _ring_small(n=(40, 36, 44), h=0.4)
    raw = inputs.smooth_random_orbitals(s).reshape(s.N, s.Ng)
    x, y, z = oham.full_coords(s)
    rho = (np.exp(-((x - 1.1) ** 2 + (y + 0.4) ** 2 + z ** 2) / 2.0)
           + 0.5 * np.exp(-((x + 2.0) ** 2 + (y - 1.0) ** 2 + (z - 0.7) ** 2) / 1.5))
    ref = opoisson.hartree(s, rho, tol=1e-13)
    vref, eref = olda.lda(rho.ravel())
    with rmgtd.Context(s, raw, poisson_tol=1e-13) as ctx:
        iters = {}
        rd = torch.from_numpy(rho.ravel()).cuda()
        for kind in (["mg", "dst"] if precond == "dst" else ["mg"]):
            ctx.set_hartree_preconditioner(rmgtd.PRECOND_DST if kind == "dst" else rmgtd.PRECOND_MG)
            vh = torch.zeros_like(rd)
            n0, i0 = ctx.profile_counters()
            ctx.hartree(rd, vh)
            n1, i1 = ctx.profile_counters()
            assert n1 - n0 == 1
            iters[kind] = i1 - i0
            assert _rel(vh.cpu().numpy(), ref.ravel()) < 1e-10
        if precond == "dst":
            assert iters["dst"] < iters["mg"], iters
        vxc = torch.empty_like(rd)
        exc = torch.empty_like(rd)
        ctx.xc(rd, vxc, exc)
        # one float64 Newton step from float32 seeds: <= 2^-43 relative per root (see k_lda)
        assert _rel(vxc.cpu().numpy(), vref) < 1e-12
        assert _rel(exc.cpu().numpy(), eref) < 1e-12
        # a second solve warm-started from the answer converges at once to the same V
        ctx.hartree(rd, vh)
        assert _rel(vh.cpu().numpy(), ref.ravel()) < 1e-10


def test_hartree_long_lines(torch_dev):
    """A 72-point axis: lines longer than 64 points take more than two 16-output tiles per
    parity in the sine-transform passes (and larger shared-memory tables)."""
    torch = torch_dev
    rmgtd = _rmgtd()
    s = _ring_small(n=(72, 36, 40), h=0.4)
    raw = inputs.smooth_random_orbitals(s).reshape(s.N, s.Ng)
    x, y, z = oham.full_coords(s)
    rho = (np.exp(-((x - 2.1) ** 2 + (y + 0.4) ** 2 + z ** 2) / 2.0)
           + 0.5 * np.exp(-((x + 4.0) ** 2 + (y - 1.0) ** 2 + (z - 0.7) ** 2) / 1.5))
    ref = opoisson.hartree(s, rho, tol=1e-13)
    with rmgtd.Context(s, raw, poisson_tol=1e-13) as ctx:
        rd = torch.from_numpy(rho.ravel()).cuda()
        vh = torch.zeros_like(rd)
        n0, i0 = ctx.profile_counters()
        ctx.hartree(rd, vh)
        n1, i1 = ctx.profile_counters()
        assert _rel(vh.cpu().numpy(), ref.ravel()) < 1e-10
        # the transform preconditioner (not the multigrid fallback) ran: few iterations
        assert n1 - n0 == 1 and i1 - i0 <= 14, (n1 - n0, i1 - i0)


def test_xc_increment_matches_oracle(torch_dev):
    """The mixed path's float32 xc increment V_xc(rho0 + d) - V_xc(rho0) against the float64
    oracle LDA: densities from 1e-16 (below the floor) to 30, around r_s = 1 (rho = 3/(4 pi))
    and across it, increments from 1e-9 to 0.6 of rho0 of both signs, zero increments and
    increments that take the density below the floor.  The bound is a few float32 units of
    the increment itself, plus 2e-13 |V_xc| for the points that take two float64 evaluations
    (near the floor, near r_s = 1): each of those is within 2^-43 relative (one Newton step
    per root, as test_hartree_and_xc checks), the accuracy of the float64 LDA itself."""
    torch = torch_dev
    rmgtd = _rmgtd()
    rng = np.random.default_rng(11)
    n = 400_000
    rs1 = 3.0 / (4.0 * np.pi)
    rho0 = np.concatenate([10 ** rng.uniform(-16, 1.5, n // 2),
                           rs1 * (1 + 10 ** rng.uniform(-9, -1, n // 4) *
                                  np.sign(rng.standard_normal(n // 4))),
                           10 ** rng.uniform(-15, -12, n // 4)])
    rel = np.sign(rng.standard_normal(n)) * 10 ** rng.uniform(-9, np.log10(0.6), n)
    rel[::97] = 0.0
    rel[1::89] = -1.0 - 1e-3            # below the floor (negative density)
    d32 = (rho0 * rel).astype(np.float32)
    d = d32.astype(np.float64)
    v1, _ = olda.lda(rho0 + d)
    v0, _ = olda.lda(rho0)
    ref = v1 - v0
    s = _ring_small(n=(20, 20, 20), h=0.5)
    raw = inputs.smooth_random_orbitals(s).reshape(s.N, s.Ng)
    with rmgtd.Context(s, raw) as ctx:
        r0 = torch.from_numpy(rho0).cuda()
        dd = torch.from_numpy(d32).cuda()
        out = torch.empty(n, dtype=torch.float32, device="cuda")
        ctx.xc_increment(r0, dd, out)
        got = out.cpu().numpy().astype(np.float64)
    err = np.abs(got - ref)
    bound = 2e-6 * np.abs(ref) + 2e-13 * np.abs(v0) + 1e-30
    bad = err > bound
    assert not bad.any(), (np.count_nonzero(bad), rho0[bad][:3], d[bad][:3], ref[bad][:3],
                           got[bad][:3])
    assert np.all(got[rel == 0.0] == 0.0)


def test_kick_matches_oracle(torch_dev):
    rmgtd = _rmgtd()
    s = _ring_small(n=(30, 30, 30), h=0.55, nvirt=20)
    raw = inputs.smooth_random_orbitals(s).reshape(s.N, s.Ng)
    phi = oham.orthonormalize(s, raw)
    pr = tddft.Propagator(s, phi, tddft.Options(dP_thrs=1e-14))
    P = np.diag(s.occupations).astype(complex)
    with rmgtd.Context(s, raw, dP_thrs=1e-14) as ctx:
        for axis, kappa in ((2, 0.05), (0, 0.3)):
            P = pr.kick(P, axis, kappa)
            ctx.kick(0, axis, kappa)
            Pg = ctx.density_matrix(0)
            assert np.max(np.abs(Pg - P)) < 1e-12
        assert abs(np.trace(Pg).real - s.n_electrons) < 1e-12


@pytest.fixture(scope="module")
def small_gs():
    s = inputs.small()
    gs = groundstate.ground_state(s, tol=1e-10)
    return s, gs


def test_trajectory_small_system(torch_dev, small_gs):
    rmgtd = _rmgtd()
    s, gs = small_gs
    nsteps = 40
    o = tddft.Options(H_thrs=1e-10, dP_thrs=1e-13, poisson_tol=1e-13)
    orc = tddft.run(s, gs["phi"], o, nsteps=nsteps, axis=2, kappa=s.kappa)
    with rmgtd.Context(s, gs["phi"], H_thrs=1e-10, dP_thrs=1e-13, poisson_tol=1e-13,
                       orthonormalize=False) as ctx:
        ctx.kick(0, 2, s.kappa)
        d = [ctx.dipole(0)]
        e = [ctx.energy(0)]
        passes = []
        for _ in range(nsteps):
            st = ctx.step(1)
            passes.append(int(st["passes"][0, 0]))
            d.append(ctx.dipole(0))
            e.append(ctx.energy(0))
        P = ctx.density_matrix(0)
    d, e = np.array(d), np.array(e)
    scale = np.max(np.abs(orc["dipole"][:, 2] - orc["dipole"][0, 2]))
    assert np.max(np.abs(d - orc["dipole"])) / scale < 1e-6
    assert np.max(np.abs(e - orc["energy"])) < 1e-9
    assert abs(np.trace(P).real - s.n_electrons) < 1e-11
    assert np.max(np.abs(P - P.conj().T)) < 1e-14
    assert abs(np.mean(passes) - np.mean(orc["passes"])) <= 0.5


def test_trajectory_three_kicks_ragged(torch_dev):
    """Three replicas (kicks x, y, z) in one context on a ragged grid and N = 37."""
    rmgtd = _rmgtd()
    s = _ring_small(n=(30, 34, 38), h=0.5, nvirt=22)
    raw = inputs.smooth_random_orbitals(s).reshape(s.N, s.Ng)
    phi = oham.orthonormalize(s, raw)
    nsteps, dt, kap = 5, 0.02, 1e-2
    o = tddft.Options(dt=dt, H_thrs=1e-10, dP_thrs=1e-13, poisson_tol=1e-13)
    refs = [tddft.run(s, phi, o, nsteps=nsteps, axis=a, kappa=kap) for a in range(3)]
    with rmgtd.Context(s, raw, dt=dt, H_thrs=1e-10, dP_thrs=1e-13, poisson_tol=1e-13,
                       nrep=3) as ctx:
        for a in range(3):
            ctx.kick(a, a, kap)
        d = [[ctx.dipole(a) for a in range(3)]]
        for _ in range(nsteps):
            ctx.step(1)
            d.append([ctx.dipole(a) for a in range(3)])
    d = np.array(d)  # (t, rep, q)
    for a in range(3):
        ref = refs[a]["dipole"]
        scale = np.max(np.abs(ref - ref[0]))
        assert np.max(np.abs(d[:, a, :] - ref)) / scale < 1e-6


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_large_orbital_block(torch_dev, precision):
    """N = 70 (> 64): the commutator series on the cooperative kernel (tile pairs, one grid
    barrier per term) instead of the cluster kernel, and the density and Gram kernels with
    three orbital tiles; two replicas on a small ragged grid against the oracle."""
    rmgtd = _rmgtd()
    s = _ring_small(n=(20, 22, 24), h=0.6, nvirt=55)
    assert s.N > 64
    raw = inputs.smooth_random_orbitals(s).reshape(s.N, s.Ng)
    phi = oham.orthonormalize(s, raw)
    nsteps, dt, kap = 3, 0.02, 1e-2
    o = tddft.Options(dt=dt, H_thrs=1e-10, dP_thrs=1e-13, poisson_tol=1e-13)
    refs = [tddft.run(s, phi, o, nsteps=nsteps, axis=a, kappa=kap) for a in range(2)]
    prec = rmgtd.PREC_FP64 if precision == "fp64" else rmgtd.PREC_MIXED
    with rmgtd.Context(s, raw, dt=dt, H_thrs=1e-10, dP_thrs=1e-13, poisson_tol=1e-13,
                       nrep=2, precision=prec) as ctx:
        for a in range(2):
            ctx.kick(a, a, kap)
        d = [[ctx.dipole(a) for a in range(2)]]
        for _ in range(nsteps):
            ctx.step(1)
            d.append([ctx.dipole(a) for a in range(2)])
    d = np.array(d)
    tol = 1e-6 if precision == "fp64" else 1e-4
    for a in range(2):
        ref = refs[a]["dipole"]
        scale = np.max(np.abs(ref - ref[0]))
        assert np.max(np.abs(d[:, a, :] - ref)) / scale < tol


def test_checkpoint_resume_is_bitwise(torch_dev, small_gs):
    rmgtd = _rmgtd()
    s, gs = small_gs
    kw = dict(H_thrs=1e-9, dP_thrs=1e-12, orthonormalize=False)
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "ck.bin")
        with rmgtd.Context(s, gs["phi"], **kw) as a:
            a.kick(0, 2, 0.01)
            a.step(3)
            a.save(path)
            a.step(3)
            Pa = a.density_matrix(0)
            ta = a.time()
        with rmgtd.Context(s, gs["phi"], **kw) as b:
            b.load(path)
            b.step(3)
            Pb = b.density_matrix(0)
            tb = b.time()
    assert ta == tb
    assert np.array_equal(Pa, Pb)


def test_error_paths_keep_state(torch_dev, small_gs):
    rmgtd = _rmgtd()
    s, gs = small_gs
    with rmgtd.Context(s, gs["phi"], H_thrs=1e-16, max_scf=1, orthonormalize=False) as ctx:
        ctx.kick(0, 2, 0.01)
        P_before = ctx.density_matrix(0)
        with pytest.raises(rmgtd.RmgtdError) as ei:
            ctx.step(1)
        assert ei.value.code == rmgtd.ENOTCONVERGED
        assert np.array_equal(ctx.density_matrix(0), P_before)
        assert ctx.time() == (0.0, 0)
        with pytest.raises(rmgtd.RmgtdError) as ei:
            ctx.kick(0, 3, 0.01)
        assert ei.value.code == rmgtd.EINVAL


def test_full_size_ring_workload(torch_dev):
    """The benchmarked workload (64^3, N = 30, kicks x/y/z) at full size: the oracle
    re-evaluates H = DFT(rho(P)) from the GPU's own P after the steps, and the invariants
    of the propagation hold."""
    rmgtd = _rmgtd()
    s = inputs.ring()
    raw = inputs.smooth_random_orbitals(s).reshape(s.N, s.Ng)
    phi = oham.orthonormalize(s, raw)
    with rmgtd.Context(s, raw, nrep=3, poisson_tol=1e-13, H_thrs=1e-9) as ctx:
        for a in range(3):
            ctx.kick(a, a, s.kappa)
        e0 = [ctx.energy(a) for a in range(3)]
        st = ctx.step(3)
        assert np.all(st["status"] == 0)
        P = [ctx.density_matrix(a) for a in range(3)]
        H0 = [ctx.get_matrix(rmgtd.MAT_H0, a) for a in range(3)]
        e1 = [ctx.energy(a) for a in range(3)]
    pr = tddft.Propagator(s, phi, tddft.Options(poisson_tol=1e-13, full_apply=False))
    for a in range(3):
        assert abs(np.trace(P[a]).real - s.n_electrons) < 1e-10
        assert np.max(np.abs(P[a] - P[a].conj().T)) < 1e-14
        H, _ = pr.dft(P[a])
        assert np.max(np.abs(H - H0[a])) < 1e-8
        assert abs(e1[a] - e0[a]) < 1e-4


def test_graph_step_matches_eager_bitwise(torch_dev):
    """The captured step (device-side SCF and Hartree while loops) runs the same kernels in
    the same order as the host-driven step: identical results."""
    rmgtd = _rmgtd()
    s = _ring_small(n=(30, 34, 38), h=0.5, nvirt=22)
    raw = inputs.smooth_random_orbitals(s).reshape(s.N, s.Ng)
    out = {}
    for mode in (False, True):
        with rmgtd.Context(s, raw, dt=0.02, nrep=3, use_graph=mode, H_thrs=1e-9) as ctx:
            for a in range(3):
                ctx.kick(a, a, 1e-2)
            st = ctx.step(4)
            out[mode] = ([ctx.density_matrix(a) for a in range(3)], st, ctx.time())
    for a in range(3):
        assert np.array_equal(out[False][0][a], out[True][0][a])
    assert np.array_equal(out[False][1]["passes"], out[True][1]["passes"])
    assert out[False][2] == out[True][2]


def test_graph_step_failure_keeps_last_completed_state(torch_dev, small_gs):
    rmgtd = _rmgtd()
    s, gs = small_gs
    with rmgtd.Context(s, gs["phi"], H_thrs=1e-9, orthonormalize=False, use_graph=True) as ctx:
        ctx.kick(0, 2, 0.01)
        ctx.step(2)
        P2 = ctx.density_matrix(0)
    with rmgtd.Context(s, gs["phi"], H_thrs=1e-9, orthonormalize=False, use_graph=True,
                       max_scf=1) as ctx:
        ctx.kick(0, 2, 0.01)
        with pytest.raises(rmgtd.RmgtdError) as ei:
            ctx.step(3)
        assert ei.value.code == rmgtd.ENOTCONVERGED
        assert ctx.time() == (0.0, 0)


# ---- mixed-precision path: float32 contractions around the float64 reference state ------
def test_mixed_trajectory_small_system(torch_dev, small_gs):
    """Mixed path vs the FP64 oracle: the stated target is 1e-4 of the dipole variation."""
    rmgtd = _rmgtd()
    s, gs = small_gs
    nsteps = 40
    o = tddft.Options(H_thrs=1e-9, dP_thrs=1e-12, poisson_tol=1e-13)
    orc = tddft.run(s, gs["phi"], o, nsteps=nsteps, axis=2, kappa=s.kappa)
    with rmgtd.Context(s, gs["phi"], H_thrs=1e-9, dP_thrs=1e-12, orthonormalize=False,
                       precision=rmgtd.PREC_MIXED) as ctx:
        ctx.kick(0, 2, s.kappa)
        d = [ctx.dipole(0)]
        e = [ctx.energy(0)]
        for _ in range(nsteps):
            ctx.step(1)
            d.append(ctx.dipole(0))
            e.append(ctx.energy(0))
        P = ctx.density_matrix(0)
    d, e = np.array(d), np.array(e)
    scale = np.max(np.abs(orc["dipole"][:, 2] - orc["dipole"][0, 2]))
    err = np.max(np.abs(d - orc["dipole"])) / scale
    assert err < 1e-4, err
    assert np.max(np.abs(e - orc["energy"])) < 1e-7
    assert abs(np.trace(P).real - s.n_electrons) < 1e-11


@pytest.mark.parametrize("tuning", [None, (3, 1, 1, 1), (2, 1, 2, 2), "multigrid"])
def test_mixed_three_kicks_ragged(torch_dev, tuning):
    """Three kicks on a ragged grid with two orbital tiles (N = 37): the default launch
    configuration, the tensor-core Gram kernel (diagonal and off-diagonal tile pairs) and the
    multigrid preconditioner of the Hartree solve."""
    rmgtd = _rmgtd()
    s = _ring_small(n=(30, 34, 38), h=0.5, nvirt=22)
    raw = inputs.smooth_random_orbitals(s).reshape(s.N, s.Ng)
    phi = oham.orthonormalize(s, raw)
    nsteps, dt, kap = 5, 0.02, 1e-2
    o = tddft.Options(dt=dt, H_thrs=1e-9, dP_thrs=1e-12, poisson_tol=1e-13)
    refs = [tddft.run(s, phi, o, nsteps=nsteps, axis=a, kappa=kap) for a in range(3)]
    with rmgtd.Context(s, raw, dt=dt, H_thrs=1e-9, dP_thrs=1e-12, nrep=3,
                       precision=rmgtd.PREC_MIXED) as ctx:
        if tuning == "multigrid":
            ctx.set_hartree_preconditioner(rmgtd.PRECOND_MG)
        elif tuning is not None:
            ctx.set_tuning(tuning)
            assert ctx.tuning() == tuning
        for a in range(3):
            ctx.kick(a, a, kap)
        d = [[ctx.dipole(a) for a in range(3)]]
        for _ in range(nsteps):
            ctx.step(1)
            d.append([ctx.dipole(a) for a in range(3)])
    d = np.array(d)
    for a in range(3):
        ref = refs[a]["dipole"]
        scale = np.max(np.abs(ref - ref[0]))
        assert np.max(np.abs(d[:, a, :] - ref)) / scale < 1e-4


def test_mixed_graph_matches_eager_and_resumes_bitwise(torch_dev, small_gs):
    rmgtd = _rmgtd()
    s, gs = small_gs
    kw = dict(H_thrs=1e-9, dP_thrs=1e-12, orthonormalize=False, precision=rmgtd.PREC_MIXED)
    out = {}
    for mode in (False, True):
        with rmgtd.Context(s, gs["phi"], use_graph=mode, **kw) as ctx:
            ctx.kick(0, 2, 0.01)
            ctx.step(4)
            out[mode] = ctx.density_matrix(0)
    assert np.array_equal(out[False], out[True])
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "ck.bin")
        with rmgtd.Context(s, gs["phi"], **kw) as a:
            a.kick(0, 2, 0.01)
            a.step(2)
            a.save(path)
            a.step(2)
            Pa = a.density_matrix(0)
        with rmgtd.Context(s, gs["phi"], **kw) as b:
            b.load(path)
            b.step(2)
            Pb = b.density_matrix(0)
    assert np.array_equal(Pa, Pb)
    assert np.array_equal(Pa, out[True])


def test_subspace_ground_state_matches_oracle(torch_dev):
    """Set-up SCF inside the orbital block (Jacobi eigensolver on the GPU, eigh in the
    oracle): same stationary P_0 and H_0; a step without a kick leaves P_0 in place."""
    rmgtd = _rmgtd()
    s = _ring_small(n=(30, 34, 38), h=0.5, nvirt=22)
    raw = inputs.smooth_random_orbitals(s).reshape(s.N, s.Ng)
    phi = oham.orthonormalize(s, raw)
    pr = tddft.Propagator(s, phi, tddft.Options(poisson_tol=1e-13, H_thrs=1e-9))
    P, H, _, it, err = pr.subspace_ground_state(300, 0.3, 1e-10)
    assert err <= 1e-10
    for prec in (rmgtd.PREC_FP64, rmgtd.PREC_MIXED):
        with rmgtd.Context(s, raw, poisson_tol=1e-13, subspace_scf=300, H_thrs=1e-9,
                           precision=prec, nrep=2) as ctx:
            for rep in range(2):
                assert np.max(np.abs(ctx.get_matrix(rmgtd.MAT_P_RE, rep) - P)) < 1e-8
                assert np.max(np.abs(ctx.get_matrix(rmgtd.MAT_H0, rep) - H)) < 1e-8
            ctx.step(2)
            assert np.max(np.abs(ctx.density_matrix(0) - P)) < 1e-7


@pytest.mark.parametrize("nvirt", [15, 22])
def test_mixed_density_matches_oracle(torch_dev, nvirt):
    """rho of the mixed path (rho_ref + float32 change; N <= 32 on the tensor cores, larger N
    on the float32 SIMT kernel) against the oracle's rho of the same P, three replicas with
    different kicks on a ragged grid (a partial last 128-point tile)."""
    rmgtd = _rmgtd()
    s = _ring_small(n=(30, 34, 38), h=0.5, nvirt=nvirt)
    raw = inputs.smooth_random_orbitals(s).reshape(s.N, s.Ng)
    phi = oham.orthonormalize(s, raw)
    pr = tddft.Propagator(s, phi, tddft.Options())
    torch = torch_dev
    with rmgtd.Context(s, raw, dt=0.02, H_thrs=1e-9, dP_thrs=1e-12, nrep=3,
                       precision=rmgtd.PREC_MIXED) as ctx:
        for a in range(3):
            ctx.kick(a, a, 1e-2)
        ctx.step(2)
        buf = torch.empty(s.Ng, dtype=torch.float64, device="cuda")
        for a in range(3):
            ctx.field_into(rmgtd.FIELD_RHO, a, buf.data_ptr())
            rho = buf.cpu().numpy()
            ref = pr.density(ctx.density_matrix(a))
            assert np.max(np.abs(rho - ref)) <= 1e-7 * np.max(np.abs(ref)), (a, np.max(np.abs(rho - ref)))
