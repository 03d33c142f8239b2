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
