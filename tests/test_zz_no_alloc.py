"""The allocation-free Gram contraction (rmgtd_gram_noalloc) against the context's own
dipole and overlap matrices.

It is meant for callers that cannot allocate device memory at the time of the call (stream
capture, host-owned memory arenas, synchronisation-free loops): it keeps its scratch in a
fixed array inside the library.  This file is collected last, so a run that stops at the
first failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest

from oracle import hamiltonian as oham
from paper_2410_09189_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_gram_noalloc_matches_context_matrices_on_consecutive_calls():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2410_09189_gb300 import rmgtd
    torch.cuda.set_device(0)
    lib = rmgtd.load_library()

    import dataclasses
    s = dataclasses.replace(inputs.ring(n=32, h=0.5, nvirt=22), n=(30, 34, 38))  # N = 37
    phi = oham.orthonormalize(s, inputs.smooth_random_orbitals(s).reshape(s.N, s.Ng))
    x, y, z = (c.ravel() for c in oham.full_coords(s))
    with rmgtd.Context(s, phi, orthonormalize=False) as ctx:
        ref = {"x": ctx.get_matrix(rmgtd.MAT_MX), "z": ctx.get_matrix(rmgtd.MAT_MZ),
               "S": ctx.get_matrix(rmgtd.MAT_S)}
    phi_d = torch.from_numpy(phi).cuda()
    w = {"x": torch.from_numpy(x).cuda(), "z": torch.from_numpy(z).cuda(), "S": None}
    stream = torch.cuda.current_stream().cuda_stream
    h3 = s.h ** 3
    outs = []
    for key in ("x", "z", "S", "x"):          # consecutive calls share the scratch array
        out = torch.empty((s.N, s.N), dtype=torch.float64, device="cuda")
        wp = ctypes.c_void_p(w[key].data_ptr()) if w[key] is not None else None
        rc = lib.rmgtd_gram_noalloc(ctypes.c_void_p(phi_d.data_ptr()),
                                    ctypes.c_void_p(phi_d.data_ptr()), wp, s.N, s.Ng, h3,
                                    ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
        assert rc == rmgtd.OK, lib.rmgtd_last_error(None)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.max(np.abs(got - ref[key])) < 1e-10, key
        outs.append(got)
    assert np.array_equal(outs[0], outs[3])

    # sizes beyond the fixed scratch are rejected without touching the device
    rc = lib.rmgtd_gram_noalloc(ctypes.c_void_p(phi_d.data_ptr()),
                                ctypes.c_void_p(phi_d.data_ptr()), None, 1025, s.Ng, 1.0,
                                ctypes.c_void_p(phi_d.data_ptr()), None)
    assert rc == rmgtd.EINVAL
    assert b"1024" in lib.rmgtd_last_error(None)
