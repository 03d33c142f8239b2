"""bench.py's algorithmic-byte model of the Hartree solve (the roofline's numerator) and its
copy of the library's multigrid coarsening rule.  CPU only."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_model", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_multigrid_levels_follow_the_library_rule():
    b = _bench()
    # halve while even and >= 4; stop at a level below the finest with <= 64 points
    assert b._mg_levels((64, 64, 64)) == ([262144, 32768, 4096, 512, 64], 2)
    # an odd dimension stops the coarsening at once; no level <= 4096 below the finest
    assert b._mg_levels((41, 36, 44)) == ([41 * 36 * 44], None)
    assert b._mg_levels((48, 48, 48)) == ([110592, 13824, 1728, 216, 27], 2)


def test_hartree_bytes_sine_transform_model():
    b = _bench()
    n0 = 64 ** 3
    for mixed, sv in ((True, 4), (False, 8)):
        # per CG iteration (32 + 17 s_V) B per point; per solve the prologue 9 s_V minus the
        # first iteration's unread p, A p (4 s_V)
        got = b.hartree_bytes((64, 64, 64), solves=3, iters=5, mixed=mixed)
        assert got == 5 * n0 * (32 + 17 * sv) + 3 * n0 * (9 * sv - 4 * sv)


def test_hartree_bytes_multigrid_model():
    b = _bench()
    lv, tail = b._mg_levels((64, 64, 64))
    per_it = lv[0] * (45 + 17 * 4) + 49 * lv[1] + 8 * lv[tail]
    got = b.hartree_bytes((64, 64, 64), solves=1, iters=2, mixed=True, precond="mg")
    assert got == 2 * per_it + lv[0] * (9 * 4 - 4 * 4)


def test_accuracy_against_the_stored_oracle_run():
    """The bench's per-run errors: dipole error relative to the stored run's own variation
    (worst replica), energy and trace errors absolute, over the stored steps the GPU run
    covers (every fifth step here)."""
    import numpy as np
    b = _bench()
    steps = [0, 5, 10, 15]
    ref_d = [[[0.0, 0.0, 1.0 + 0.1 * k] for k in range(4)], [[0.0, 2.0 * k, 0.0] for k in range(4)]]
    g = {"options": {"H_thrs": 1e-10, "dP_thrs": 1e-12},
         "replicas": [{"step": steps, "dipole": ref_d[a], "energy": [-1.0 - a] * 4,
                       "trace": [2.0] * 4} for a in range(2)]}
    d = {k: [np.array(ref_d[0][i]) + [0.0, 0.0, 3e-5 if k == 10 else 0.0],
             np.array(ref_d[1][i])] for i, k in enumerate(steps)}
    e = {k: [-1.0, -2.0 + (1e-9 if k == 5 else 0.0)] for k in steps}
    t = {k: [2.0, 2.0 - 1e-12] for k in steps}
    out = b.accuracy_against_oracle(d, e, t, g, steps_done=10)
    assert abs(out["dipole_rel_err"] - 3e-5 / 0.3) < 1e-12     # replica 0: variation 0.3
    assert abs(out["energy_err"] - 1e-9) < 1e-15
    assert abs(out["trace_err"] - 1e-12) < 1e-15
    assert out["window"].startswith("steps 0..10")
