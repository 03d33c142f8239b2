"""The C ABI library builds, loads without a GPU and exports every declared entry point."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rmgtd.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rmgtd_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2410_09189_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["rmgtd_create", "rmgtd_destroy", "rmgtd_apply_h", "rmgtd_kick", "rmgtd_step",
              "rmgtd_density", "rmgtd_dipole", "rmgtd_energy", "rmgtd_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    from paper_2410_09189_gb300 import rmgtd
    lib = rmgtd.load_library()
    for n in _declared():
        assert getattr(lib, n).restype is not None or n in ("rmgtd_destroy", "rmgtd_net_destroy", "rmgtd_batch_destroy",
                                                              "rmgtd_default_options")


def test_default_options_without_gpu(lib):
    from paper_2410_09189_gb300 import rmgtd
    L = rmgtd.load_library()
    o = rmgtd.COptions()
    L.rmgtd_default_options(ctypes.byref(o))
    assert o.dt == 0.05 and o.H_thrs == 1e-7 and o.dP_thrs == 1e-10 and o.nrep == 1
    assert o.max_scf == 50 and o.max_terms == 200


def test_create_rejects_bad_input_without_touching_the_gpu(lib):
    from paper_2410_09189_gb300 import rmgtd
    L = rmgtd.load_library()
    cs = rmgtd.CSystem()          # all zeros: NULL phi0, empty grid
    ctx = ctypes.c_void_p()
    rc = L.rmgtd_create(ctypes.byref(cs), None, ctypes.byref(ctx))
    assert rc == rmgtd.EINVAL and not ctx.value
    assert b"phi0" in L.rmgtd_last_error(None)
