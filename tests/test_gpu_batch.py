"""Several systems of uneven grids stepped by one CUDA graph per time step (rmgtd_batch), and
the launch autotuner: the batch reproduces the separately stepped contexts bit for bit, and
the tuned launch configurations change results only at rounding level."""
import dataclasses

import numpy as np
import pytest

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


SYSTEMS = [dict(index=0, natoms=8, n=32), dict(index=1, natoms=12, n=36),
           dict(index=2, natoms=6, n=28)]


def _make(lib, spec, precision, **kw):
    s = inputs.cluster(spec["index"], natoms=spec["natoms"], n=spec["n"])
    raw = inputs.smooth_random_orbitals(s).reshape(s.N, s.Ng)
    ctx = lib.Context(s, raw, nrep=3, H_thrs=1e-8, dP_thrs=1e-11, precision=precision,
                      use_graph=True, subspace_scf=50, **kw)
    for a in range(3):
        ctx.kick(a, a, 1e-3)
    return ctx


@pytest.mark.parametrize("budget", [0, 48])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_matches_separate_contexts_bitwise(lib, precision, budget):
    """budget 0: the systems run back to back in the graph; budget 48: each context's grids
    are sized to 48 SMs and the three run concurrently on parallel branches (3 x 48 <= the SM
    count); either way every context matches its separately stepped twin bit for bit."""
    prec = lib.PREC_FP64 if precision == "fp64" else lib.PREC_MIXED
    nsteps = 6
    solo = []
    for spec in SYSTEMS:
        ctx = _make(lib, spec, prec, sm_budget=budget)
        st = ctx.step(nsteps)
        solo.append(([ctx.dipole(a) for a in range(3)], st["passes"].copy()))
        ctx.close()
    ctxs = [_make(lib, spec, prec, sm_budget=budget) for spec in SYSTEMS]
    batch = lib.Batch(ctxs)
    with pytest.raises(lib.RmgtdError):
        ctxs[0].step(1)               # a batched context is stepped through its batch
    sts = []
    for _ in range(2):
        sts.append(batch.step(nsteps // 2))
    for i, ctx in enumerate(ctxs):
        d = [ctx.dipole(a) for a in range(3)]
        passes = np.concatenate([s[i]["passes"] for s in sts])
        assert np.array_equal(np.array(d), np.array(solo[i][0])), i
        assert np.array_equal(passes, solo[i][1]), i
        assert ctx.time()[1] == nsteps
    batch.close()
    ctxs[0].step(1)                   # free again once the batch is gone
    for c in ctxs:
        c.close()


def test_batch_rejects_bad_arguments(lib):
    ctx = _make(lib, SYSTEMS[0], lib.PREC_MIXED)
    with pytest.raises(lib.RmgtdError):
        lib.Batch([ctx, ctx])
    b = lib.Batch([ctx])
    with pytest.raises(lib.RmgtdError):
        lib.Batch([ctx])              # already in a batch
    with pytest.raises(lib.RmgtdError):
        ctx.autotune()
    b.close()
    ctx.close()


def test_autotune_changes_results_only_at_rounding_level(lib):
    s = inputs.scaled(inputs.ring(), n=40, h=0.5, nvirt=15)
    raw = inputs.smooth_random_orbitals(s).reshape(s.N, s.Ng)
    kw = dict(nrep=3, H_thrs=1e-9, dP_thrs=1e-12, precision=lib.PREC_MIXED, use_graph=True)
    out = []
    for tune in (False, True):
        ctx = lib.Context(s, raw, **kw)
        for a in range(3):
            ctx.kick(a, a, 1e-3)
        if tune:
            choice = ctx.autotune()
            assert choice[0] in (1, 2, 3, 4) and choice[1] in (0, 1)
            assert choice[2] in (1, 2, 4, 8) and choice[3] in (1, 2, 4)
        ctx.step(8)
        out.append(np.array([ctx.dipole(a) for a in range(3)]))
        ctx.close()
    d0, d1 = out
    scale = np.max(np.abs(d0))
    assert np.max(np.abs(d1 - d0)) <= 1e-7 * scale


def test_tensor_core_gram_matches_simt_gram(lib):
    """The Hamiltonian update on the tensor cores (3xTF32) against the float32 SIMT kernel:
    the same trajectory up to rounding level, also with two CTAs per SM (fewer stages in
    the copy ring) and a ragged last chunk of the grid."""
    # Ng = 41 * 36 * 44 = 64944: a multiple of 4 (bulk copies) but not of 32 (ragged stage)
    s = dataclasses.replace(inputs.scaled(inputs.ring(), n=40, h=0.5, nvirt=15), n=(41, 36, 44))
    raw = inputs.smooth_random_orbitals(s).reshape(s.N, s.Ng)
    kw = dict(nrep=3, H_thrs=1e-9, dP_thrs=1e-12, precision=lib.PREC_MIXED, use_graph=True)
    out = []
    for tuning in ((3, 0, 2, 1), (3, 1, 1, 1), (3, 1, 2, 1)):
        ctx = lib.Context(s, raw, **kw)
        ctx.set_tuning(tuning)
        for a in range(3):
            ctx.kick(a, a, 1e-3)
        ctx.step(6)
        out.append((np.array([ctx.dipole(a) for a in range(3)]),
                    np.array([ctx.get_matrix(lib.MAT_H0, r) for r in range(3)])))
        ctx.close()
    # 3xTF32 keeps ~2^-21 of each product of the update h^3 Phi^T diag(dV) Phi; the float32
    # SIMT sum ~2^-24 per term: the converged H of the two differs by ~1e-8 of |H|
    d0, h0 = out[0]
    scale = np.max(np.abs(d0))
    for d1, h1 in out[1:]:
        assert np.max(np.abs(d1 - d0)) <= 1e-7 * scale
        assert np.max(np.abs(h1 - h0)) <= 5e-8 * np.max(np.abs(h0))


def test_set_tuning_rejects_bad_values(lib):
    s = inputs.scaled(inputs.ring(), n=24, h=0.6, nvirt=4)
    raw = inputs.smooth_random_orbitals(s).reshape(s.N, s.Ng)
    ctx = lib.Context(s, raw, nrep=1, precision=lib.PREC_MIXED)
    before = ctx.tuning()
    for bad in ((0, 0, 1, 1), (3, 2, 1, 1), (3, 0, 3, 1), (3, 0, 1, 3)):
        with pytest.raises(lib.RmgtdError):
            ctx.set_tuning(bad)
        assert ctx.tuning() == before
    for bad in (-1, 2):
        with pytest.raises(lib.RmgtdError):
            ctx.set_hartree_preconditioner(bad)
    ctx.close()
