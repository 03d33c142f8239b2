"""Thin ctypes binding of librmgtd (the C ABI of include/rmgtd.h).

Argument marshalling only: every step of the propagation runs in the CUDA library.  If the
library is missing the binding raises -- there is no CPU fallback.  Device memory for the
context comes from PyTorch's caching allocator (through the ABI's allocator hook) and work
runs on the current PyTorch CUDA stream unless another stream is given.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from .inputs import System

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "librmgtd.so")

OK, EINVAL, ENOMEM, ECUDA, ENOTCONVERGED, EDIVERGED, ETIMEOUT, ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
PREC_FP64, PREC_MIXED = 0, 1
PRECOND_DST, PRECOND_MG = 0, 1      # Hartree CG preconditioner (rmgtd_set_hartree_preconditioner)
F64, F32, C128, C64 = 0, 1, 2, 3
MAT_P_RE, MAT_P_IM, MAT_H0, MAT_HM1, MAT_HCORE, MAT_MX, MAT_MY, MAT_MZ, MAT_S = range(9)
NPHASES = 6
PHASES = ("eldyn", "rho", "hartree", "xc", "hupdate", "other")

_c_double_p = ctypes.POINTER(ctypes.c_double)
_c_int_p = ctypes.POINTER(ctypes.c_int)
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class RmgtdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"rmgtd error {code}: {msg}")
        self.code = code


class CSystem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("h", ctypes.c_double),
        ("natoms", ctypes.c_int), ("pos", _c_double_p), ("Z", _c_double_p),
        ("rc_loc", _c_double_p),
        ("nproj", ctypes.c_int), ("proj_atom", _c_int_p), ("proj_l", _c_int_p),
        ("proj_m", _c_int_p), ("proj_rc", _c_double_p), ("E_kb", _c_double_p),
        ("nocc", ctypes.c_int), ("nvirt", ctypes.c_int), ("f", _c_double_p),
        ("phi0", _c_double_p), ("v_ext_omega", ctypes.c_double), ("hartree_xc", ctypes.c_int),
        ("rho_core", _c_double_p),
    ]


class COptions(ctypes.Structure):
    _fields_ = [
        ("dt", ctypes.c_double), ("H_thrs", ctypes.c_double), ("dP_thrs", ctypes.c_double),
        ("max_scf", ctypes.c_int), ("max_terms", ctypes.c_int), ("precision", ctypes.c_int),
        ("nrep", ctypes.c_int), ("orthonormalize", ctypes.c_int),
        ("poisson_tol", ctypes.c_double), ("poisson_max_iter", ctypes.c_int),
        ("use_graph", ctypes.c_int), ("stream", ctypes.c_void_p),
        ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", ctypes.c_void_p),
        ("subspace_scf", ctypes.c_int), ("subspace_mix", ctypes.c_double),
        ("subspace_tol", ctypes.c_double), ("mixed_poisson_tol", ctypes.c_double),
        ("magnus_order", ctypes.c_int), ("nonorthogonal", ctypes.c_int),
        ("grid_basis", ctypes.c_int), ("ground_state_scf", ctypes.c_int),
        ("ground_state_tol", ctypes.c_double), ("seed_order", ctypes.c_int),
        ("sm_budget", ctypes.c_int),
    ]


class CStats(ctypes.Structure):
    _fields_ = [("passes", ctypes.c_int), ("terms_max", ctypes.c_int),
                ("terms_sum", ctypes.c_int), ("status", ctypes.c_int), ("H_err", ctypes.c_double)]


_lib = None


def load_library(path: Optional[str] = None):
    """Load librmgtd.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} not found: build it with `python -m paper_2410_09189_gb300.build`")
    lib = ctypes.CDLL(path)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "rmgtd_default_options": (None, [ctypes.POINTER(COptions)]),
        "rmgtd_create": (i, [ctypes.POINTER(CSystem), ctypes.POINTER(COptions), ctypes.POINTER(vp)]),
        "rmgtd_destroy": (None, [vp]),
        "rmgtd_apply_h": (i, [vp, vp, vp, i, i, i]),
        "rmgtd_kick": (i, [vp, i, i, d]),
        "rmgtd_step": (i, [vp, i, ctypes.POINTER(CStats)]),
        "rmgtd_density": (i, [vp, i, _c_double_p]),
        "rmgtd_dipole": (i, [vp, i, _c_double_p]),
        "rmgtd_energy": (i, [vp, i, _c_double_p]),
        "rmgtd_get_matrix": (i, [vp, i, i, _c_double_p]),
        "rmgtd_set_matrix": (i, [vp, i, i, _c_double_p]),
        "rmgtd_hartree": (i, [vp, vp, vp]),
        "rmgtd_xc": (i, [vp, vp, vp, vp, ctypes.c_size_t]),
        "rmgtd_xc_increment": (i, [vp, vp, vp, vp, ctypes.c_size_t]),
        "rmgtd_save": (i, [vp, ctypes.c_char_p]),
        "rmgtd_load": (i, [vp, ctypes.c_char_p]),
        "rmgtd_time": (i, [vp, _c_double_p, ctypes.POINTER(ctypes.c_longlong)]),
        "rmgtd_last_error": (ctypes.c_char_p, [vp]),
        "rmgtd_profile": (i, [vp, i]),
        "rmgtd_profile_counters": (i, [vp, ctypes.POINTER(ctypes.c_longlong),
                                       ctypes.POINTER(ctypes.c_longlong)]),
        "rmgtd_gram_noalloc": (i, [vp, vp, vp, i, ctypes.c_longlong, d, vp, vp]),
        "rmgtd_net_num_params": (ctypes.c_longlong, []),
        "rmgtd_net_create": (i, [i, i, i, i, vp, ctypes.POINTER(vp)]),
        "rmgtd_net_destroy": (None, [vp]),
        "rmgtd_net_set_params": (i, [vp, ctypes.POINTER(ctypes.c_float)]),
        "rmgtd_net_get_params": (i, [vp, ctypes.POINTER(ctypes.c_float)]),
        "rmgtd_net_set_scales": (i, [vp, _c_double_p, d]),
        "rmgtd_net_get_scales": (i, [vp, _c_double_p, _c_double_p]),
        "rmgtd_net_features": (i, [vp, vp, vp, vp, vp]),
        "rmgtd_net_targets": (i, [vp, vp, vp, vp, vp]),
        "rmgtd_net_forward": (i, [vp, vp, vp, i]),
        "rmgtd_net_forward_tc": (i, [vp, vp, vp, i]),
        "rmgtd_net_backward": (i, [vp, vp, vp, i, _c_double_p, ctypes.POINTER(ctypes.c_float)]),
        "rmgtd_net_adam": (i, [vp, d]),
        "rmgtd_attach_net": (i, [vp, vp]),
        "rmgtd_get_field": (i, [vp, i, i, vp]),
        "rmgtd_autotune": (i, [vp, _c_int_p]),
        "rmgtd_set_tuning": (i, [vp, _c_int_p]),
        "rmgtd_get_tuning": (i, [vp, _c_int_p]),
        "rmgtd_set_hartree_preconditioner": (i, [vp, i]),
        "rmgtd_batch_create": (i, [ctypes.POINTER(vp), i, ctypes.POINTER(vp)]),
        "rmgtd_batch_destroy": (None, [vp]),
        "rmgtd_batch_step": (i, [vp, i, ctypes.POINTER(ctypes.POINTER(CStats))]),
        "rmgtd_profile_read": (i, [vp, _c_double_p, ctypes.POINTER(ctypes.c_longlong),
                                   ctypes.POINTER(ctypes.c_longlong)]),
        "rmgtd_selftest_barrier_timeout": (i, [vp, ctypes.c_uint, _c_int_p]),
        "rmgtd_get_hartree_preconditioner": (i, [vp, _c_int_p]),
        "rmgtd_net_save": (i, [vp, ctypes.c_char_p]),
        "rmgtd_net_load": (i, [vp, ctypes.c_char_p]),
        "rmgtd_surrogate_load": (i, [vp, ctypes.c_char_p, ctypes.POINTER(vp)]),
        "rmgtd_ground_state_info": (i, [vp, ctypes.POINTER(i), _c_double_p, _c_double_p, _c_double_p]),
        "rmgtd_set_field": (i, [vp, i, _c_double_p, i]),
        "rmgtd_spectrum": (i, [_c_double_p, i, ctypes.c_long, d, d, d, _c_double_p, i,
                               _c_double_p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_c_double_p)


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(_c_int_p)


class Context:
    """One propagation context on the current CUDA device (owns its device memory)."""

    def __init__(self, sys: System, phi0: np.ndarray, *, dt: Optional[float] = None,
                 H_thrs: float = 1e-7, dP_thrs: float = 1e-10, max_scf: int = 50,
                 max_terms: int = 200, precision: int = PREC_FP64, nrep: int = 1,
                 orthonormalize: bool = True, poisson_tol: float = 1e-12,
                 poisson_max_iter: int = 200, use_graph: bool = True,
                 stream: Optional[int] = None, torch_alloc: bool = True,
                 subspace_scf: int = 0, subspace_mix: float = 0.3, subspace_tol: float = 1e-10,
                 mixed_poisson_tol: float = 0.0, magnus_order: int = 1,
                 nonorthogonal: bool = False, grid_basis: bool = False,
                 ground_state_scf: int = 0, ground_state_tol: float = 1e-8,
                 seed_order: int = 1, sm_budget: int = 0):
        import torch

        lib = load_library()
        self._lib = lib
        self._torch = torch
        self.sys = sys
        self.N = sys.N
        self.Ng = sys.Ng
        self.nrep = nrep
        self._keep = []
        phi = np.ascontiguousarray(phi0, dtype=np.float64).reshape(sys.N, sys.Ng)
        arrs = {
            "pos": np.ascontiguousarray(sys.pos, dtype=np.float64).reshape(-1),
            "Z": np.ascontiguousarray(sys.Z, dtype=np.float64),
            "rc": np.ascontiguousarray(sys.rc_loc, dtype=np.float64),
            "pa": np.ascontiguousarray(sys.proj_atom, dtype=np.int32),
            "pl": np.ascontiguousarray(sys.proj_l, dtype=np.int32),
            "pm": np.ascontiguousarray(sys.proj_m, dtype=np.int32),
            "prc": np.ascontiguousarray(sys.proj_rc, dtype=np.float64),
            "ekb": np.ascontiguousarray(sys.E_kb, dtype=np.float64),
            "f": np.ascontiguousarray(sys.occupations, dtype=np.float64),
            "phi": phi,
        }
        self._keep.append(arrs)
        cs = CSystem()
        cs.nx, cs.ny, cs.nz = (int(v) for v in sys.n)
        cs.h = float(sys.h)
        cs.natoms = int(len(sys.Z))
        cs.pos, cs.Z, cs.rc_loc = _dptr(arrs["pos"]), _dptr(arrs["Z"]), _dptr(arrs["rc"])
        cs.nproj = int(sys.nproj)
        cs.proj_atom, cs.proj_l, cs.proj_m = _iptr(arrs["pa"]), _iptr(arrs["pl"]), _iptr(arrs["pm"])
        cs.proj_rc, cs.E_kb = _dptr(arrs["prc"]), _dptr(arrs["ekb"])
        cs.nocc, cs.nvirt = int(sys.nocc), int(sys.nvirt)
        cs.f = _dptr(arrs["f"])
        cs.phi0 = _dptr(phi)
        cs.v_ext_omega = float(sys.v_ext_omega)
        cs.hartree_xc = 1 if sys.hartree_xc else 0
        if getattr(sys, "rho_core", None) is not None:
            core = np.ascontiguousarray(np.asarray(sys.rho_core, dtype=np.float64).reshape(-1))
            if core.size != sys.Ng:
                raise ValueError("rho_core must have one value per grid point")
            arrs["core"] = core
            cs.rho_core = _dptr(core)
        opt = COptions()
        lib.rmgtd_default_options(ctypes.byref(opt))
        opt.dt = float(sys.dt if dt is None else dt)
        opt.H_thrs, opt.dP_thrs = float(H_thrs), float(dP_thrs)
        opt.max_scf, opt.max_terms = int(max_scf), int(max_terms)
        opt.precision, opt.nrep = int(precision), int(nrep)
        opt.orthonormalize = 1 if orthonormalize else 0
        opt.poisson_tol, opt.poisson_max_iter = float(poisson_tol), int(poisson_max_iter)
        opt.use_graph = 1 if use_graph else 0
        opt.subspace_scf, opt.subspace_mix = int(subspace_scf), float(subspace_mix)
        opt.subspace_tol = float(subspace_tol)
        opt.mixed_poisson_tol = float(mixed_poisson_tol)
        opt.magnus_order = int(magnus_order)
        opt.nonorthogonal = 1 if nonorthogonal else 0
        opt.grid_basis = 1 if grid_basis else 0
        opt.ground_state_scf = int(ground_state_scf)
        opt.ground_state_tol = float(ground_state_tol)
        opt.seed_order = int(seed_order)
        opt.sm_budget = int(sm_budget)
        if nonorthogonal:
            opt.orthonormalize = 0
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = int(stream)
        opt.stream = ctypes.c_void_p(self.stream)
        if torch_alloc:
            dev = torch.cuda.current_device()

            def _alloc(nbytes, strm, user):
                try:
                    return int(torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(strm or 0)))
                except Exception:  # reported to the library as an allocation failure
                    return None

            def _free(ptr, user):
                torch.cuda.caching_allocator_delete(int(ptr))

            self._alloc_cb = ALLOC_FN(_alloc)
            self._free_cb = FREE_FN(_free)
            opt.alloc, opt.free = self._alloc_cb, self._free_cb
        self._ctx = ctypes.c_void_p()
        rc = lib.rmgtd_create(ctypes.byref(cs), ctypes.byref(opt), ctypes.byref(self._ctx))
        if rc != OK:
            msg = lib.rmgtd_last_error(None).decode()
            raise RmgtdError(rc, msg)

    def _stats_array(self, st, nsteps):
        out = np.zeros((nsteps, self.nrep), dtype=[("passes", "i4"), ("terms_max", "i4"),
                                                   ("terms_sum", "i4"), ("status", "i4"),
                                                   ("H_err", "f8")])
        for s in range(nsteps):
            for r in range(self.nrep):
                c = st[s * self.nrep + r]
                out[s, r] = (c.passes, c.terms_max, c.terms_sum, c.status, c.H_err)
        return out

    # --- helpers -----------------------------------------------------------------------
    def _check(self, rc: int):
        if rc != OK:
            raise RmgtdError(rc, self._lib.rmgtd_last_error(self._ctx).decode())

    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            self._lib.rmgtd_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # --- ABI -----------------------------------------------------------------------------
    def ground_state_info(self):
        """(iterations, max|rho_out - rho_in|, largest Ritz residual, orbital energies) of the
        ground-state SCF run at creation (rmgtd_ground_state_info)."""
        it = ctypes.c_int()
        d, r = ctypes.c_double(), ctypes.c_double()
        eps = np.empty(self.N)
        self._check(self._lib.rmgtd_ground_state_info(
            self._ctx, ctypes.byref(it), ctypes.cast(ctypes.byref(d), _c_double_p),
            ctypes.cast(ctypes.byref(r), _c_double_p), _dptr(eps)))
        return int(it.value), float(d.value), float(r.value), eps

    def set_field(self, rep: int, E):
        """Samples E[j] = (E_x, E_y, E_z)(j dt) of replica `rep`'s external field
        (rmgtd_set_field); an empty array clears it."""
        E = np.ascontiguousarray(np.asarray(E, dtype=np.float64).reshape(-1, 3))
        self._keep.append(E)
        self._check(self._lib.rmgtd_set_field(self._ctx, int(rep), _dptr(E), int(E.shape[0])))

    def kick(self, rep: int, axis: int, kappa: float):
        self._check(self._lib.rmgtd_kick(self._ctx, rep, axis, float(kappa)))

    def step(self, nsteps: int = 1, stats: bool = True, raise_on_error: bool = True):
        st = (CStats * max(1, nsteps * self.nrep))() if stats else None
        rc = self._lib.rmgtd_step(self._ctx, int(nsteps), st)
        if raise_on_error:
            self._check(rc)
        if not stats:
            return rc
        out = np.zeros((nsteps, self.nrep), dtype=[("passes", "i4"), ("terms_max", "i4"),
                                                   ("terms_sum", "i4"), ("status", "i4"),
                                                   ("H_err", "f8")])
        for s in range(nsteps):
            for r in range(self.nrep):
                c = st[s * self.nrep + r]
                out[s, r] = (c.passes, c.terms_max, c.terms_sum, c.status, c.H_err)
        return out if raise_on_error else (rc, out)

    def autotune(self):
        """Time the launch alternatives and keep the fastest; returns the choice
        (density CTAs/SM, Gram on tensor cores, Gram CTAs/SM, Hartree block divisor)."""
        c = np.zeros(4, dtype=np.int32)
        self._check(self._lib.rmgtd_autotune(self._ctx, _iptr(c)))
        return tuple(int(v) for v in c)

    def set_tuning(self, choice):
        """Set the launch configuration (same order as autotune's result)."""
        c = np.ascontiguousarray(choice, dtype=np.int32)
        assert c.shape == (4,)
        self._check(self._lib.rmgtd_set_tuning(self._ctx, _iptr(c)))

    def set_hartree_preconditioner(self, kind: int):
        """PRECOND_DST (sine transform, the default where it fits) or PRECOND_MG (V-cycle)."""
        self._check(self._lib.rmgtd_set_hartree_preconditioner(self._ctx, int(kind)))

    def tuning(self):
        c = np.zeros(4, dtype=np.int32)
        self._check(self._lib.rmgtd_get_tuning(self._ctx, _iptr(c)))
        return tuple(int(v) for v in c)

    def attach_net(self, net: Optional["Net"]):
        """Seed every step's SCF loop with the network's correction (None detaches)."""
        self._net = net
        self._check(self._lib.rmgtd_attach_net(self._ctx, net._net if net is not None else None))

    def surrogate_load(self, path: str) -> "Net":
        """Create a network on this grid, load the weight file and attach it
        (rmgtd_surrogate_load); returns the attached network."""
        handle = ctypes.c_void_p()
        self._check(self._lib.rmgtd_surrogate_load(self._ctx, os.fsencode(path), ctypes.byref(handle)))
        net = Net.__new__(Net)
        net._lib = self._lib
        net.n = tuple(int(v) for v in self.sys.n)
        net.Ng = self.Ng
        net.max_batch = self.nrep
        net.P = int(self._lib.rmgtd_net_num_params())
        net._net = handle
        self._net = net
        return net

    def field_into(self, which: int, rep: int, dev_ptr: int):
        """Copy rho (FIELD_RHO) or V_H + V_xc (FIELD_VHXC) of replica `rep` to device memory."""
        self._check(self._lib.rmgtd_get_field(self._ctx, int(which), int(rep), ctypes.c_void_p(dev_ptr)))

    def density(self, rep: int = 0) -> np.ndarray:
        out = np.empty(self.Ng)
        self._check(self._lib.rmgtd_density(self._ctx, rep, _dptr(out)))
        return out

    def dipole(self, rep: int = 0) -> np.ndarray:
        out = np.empty(3)
        self._check(self._lib.rmgtd_dipole(self._ctx, rep, _dptr(out)))
        return out

    def energy(self, rep: int = 0) -> float:
        out = np.empty(1)
        self._check(self._lib.rmgtd_energy(self._ctx, rep, _dptr(out)))
        return float(out[0])

    def get_matrix(self, which: int, rep: int = 0) -> np.ndarray:
        out = np.empty((self.N, self.N))
        self._check(self._lib.rmgtd_get_matrix(self._ctx, which, rep, _dptr(out)))
        return out

    def set_matrix(self, which: int, rep: int, M: np.ndarray):
        a = np.ascontiguousarray(M, dtype=np.float64)
        self._check(self._lib.rmgtd_set_matrix(self._ctx, which, rep, _dptr(a)))

    def density_matrix(self, rep: int = 0) -> np.ndarray:
        return self.get_matrix(MAT_P_RE, rep) + 1j * self.get_matrix(MAT_P_IM, rep)

    def apply_h(self, x, hx, rep: int = -1):
        """hx = H x for CUDA tensors of shape (ncols, Ng) (float64/float32/complex128/complex64)."""
        torch = self._torch
        codes = {torch.float64: F64, torch.float32: F32, torch.complex128: C128,
                 torch.complex64: C64}
        assert x.is_cuda and hx.is_cuda and x.dtype == hx.dtype and x.is_contiguous()
        ncols = x.numel() // self.Ng
        self._check(self._lib.rmgtd_apply_h(self._ctx, ctypes.c_void_p(x.data_ptr()),
                                            ctypes.c_void_p(hx.data_ptr()), ncols,
                                            codes[x.dtype], rep))

    def hartree(self, rho, vh):
        self._check(self._lib.rmgtd_hartree(self._ctx, ctypes.c_void_p(rho.data_ptr()),
                                            ctypes.c_void_p(vh.data_ptr())))

    def xc(self, rho, vxc, exc):
        self._check(self._lib.rmgtd_xc(self._ctx, ctypes.c_void_p(rho.data_ptr()),
                                       ctypes.c_void_p(vxc.data_ptr()),
                                       ctypes.c_void_p(exc.data_ptr()), rho.numel()))

    def xc_increment(self, rho0, drho, dvxc):
        """dvxc <- V_xc(rho0 + drho) - V_xc(rho0) (float64 rho0, float32 drho and dvxc)."""
        self._check(self._lib.rmgtd_xc_increment(self._ctx, ctypes.c_void_p(rho0.data_ptr()),
                                                 ctypes.c_void_p(drho.data_ptr()),
                                                 ctypes.c_void_p(dvxc.data_ptr()),
                                                 rho0.numel()))

    def save(self, path: str):
        self._check(self._lib.rmgtd_save(self._ctx, path.encode()))

    def load(self, path: str):
        self._check(self._lib.rmgtd_load(self._ctx, path.encode()))

    def profile(self, enable: bool = True):
        """Start / stop per-phase CUDA-event timing (resets totals and the launch count)."""
        self._check(self._lib.rmgtd_profile(self._ctx, 1 if enable else 0))

    def profile_read(self):
        """(phase -> ms, phase -> calls, kernel launches) since the last profile() call."""
        ms = np.zeros(NPHASES)
        calls = (ctypes.c_longlong * NPHASES)()
        n = ctypes.c_longlong()
        self._check(self._lib.rmgtd_profile_read(self._ctx, _dptr(ms), calls, ctypes.byref(n)))
        return (dict(zip(PHASES, ms.tolist())), dict(zip(PHASES, list(calls))), int(n.value))

    def hartree_preconditioner(self) -> int:
        """PRECOND_DST or PRECOND_MG: the preconditioner the Hartree solves use now."""
        k = ctypes.c_int(-1)
        self._check(self._lib.rmgtd_get_hartree_preconditioner(self._ctx, ctypes.byref(k)))
        return int(k.value)

    def selftest_barrier_timeout(self, polls: int) -> int:
        """Status recorded by blocks whose grid-barrier wait (limited to `polls` polls) had
        to give up (rmgtd_selftest_barrier_timeout)."""
        st = ctypes.c_int(0)
        self._check(self._lib.rmgtd_selftest_barrier_timeout(self._ctx, int(polls), ctypes.byref(st)))
        return int(st.value)

    def profile_counters(self):
        """(Hartree replica solves, CG iterations summed over them) since profile()."""
        ns = ctypes.c_longlong()
        ni = ctypes.c_longlong()
        self._check(self._lib.rmgtd_profile_counters(self._ctx, ctypes.byref(ns), ctypes.byref(ni)))
        return int(ns.value), int(ni.value)

    def time(self):
        t = ctypes.c_double()
        n = ctypes.c_longlong()
        self._check(self._lib.rmgtd_time(self._ctx, ctypes.byref(t), ctypes.byref(n)))
        return t.value, n.value


FIELD_RHO, FIELD_VHXC = 0, 1


class Net:
    """The learned SCF-seed network (rmgtd_net): parameters, scales, features, forward,
    backward and Adam all run in the library; arrays passed as device pointers (ints)."""

    def __init__(self, n, max_batch: int = 1, stream: Optional[int] = None):
        import torch

        self._lib = load_library()
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.n = tuple(int(v) for v in n)
        self.Ng = self.n[0] * self.n[1] * self.n[2]
        self.max_batch = int(max_batch)
        self.P = int(self._lib.rmgtd_net_num_params())
        self._net = ctypes.c_void_p()
        self._check(self._lib.rmgtd_net_create(self.n[0], self.n[1], self.n[2], self.max_batch,
                                               ctypes.c_void_p(int(stream)), ctypes.byref(self._net)))

    def _check(self, rc: int):
        if rc != OK:
            raise RmgtdError(rc, self._lib.rmgtd_last_error(None).decode())

    def save(self, path: str):
        """Write the parameters and scales to a weight file (rmgtd_net_save)."""
        self._check(self._lib.rmgtd_net_save(self._net, os.fsencode(path)))

    def load(self, path: str):
        """Read parameters and scales from a weight file (rmgtd_net_load)."""
        self._check(self._lib.rmgtd_net_load(self._net, os.fsencode(path)))

    def close(self):
        if getattr(self, "_net", None) and self._net.value:
            self._lib.rmgtd_net_destroy(self._net)
            self._net = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, theta: np.ndarray):
        t = np.ascontiguousarray(theta, dtype=np.float32)
        assert t.size == self.P
        self._check(self._lib.rmgtd_net_set_params(self._net, t.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def params(self) -> np.ndarray:
        t = np.empty(self.P, dtype=np.float32)
        self._check(self._lib.rmgtd_net_get_params(self._net, t.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return t

    def set_scales(self, in_scales, out_scale: float):
        s = np.ascontiguousarray(in_scales, dtype=np.float64)
        self._check(self._lib.rmgtd_net_set_scales(self._net, _dptr(s), float(out_scale)))

    def scales(self):
        s = np.empty(3)
        o = ctypes.c_double()
        self._check(self._lib.rmgtd_net_get_scales(self._net, _dptr(s), ctypes.byref(o)))
        return s, float(o.value)

    def features(self, rho_t: int, rho_tm1: int, rho_tm2: int, x: int):
        v = ctypes.c_void_p
        self._check(self._lib.rmgtd_net_features(self._net, v(rho_t), v(rho_tm1), v(rho_tm2), v(x)))

    def targets(self, v_tp1: int, v_t: int, v_tm1: int, t: int):
        v = ctypes.c_void_p
        self._check(self._lib.rmgtd_net_targets(self._net, v(v_tp1), v(v_t), v(v_tm1), v(t)))

    def forward(self, x: int, y: int, batch: int):
        self._check(self._lib.rmgtd_net_forward(self._net, ctypes.c_void_p(x), ctypes.c_void_p(y), int(batch)))

    def forward_tc(self, x: int, y: int, batch: int):
        """Forward with the middle layers on the tensor cores (bfloat16 activations)."""
        self._check(self._lib.rmgtd_net_forward_tc(self._net, ctypes.c_void_p(x), ctypes.c_void_p(y), int(batch)))

    def backward(self, x: int, t: int, batch: int, want_grad: bool = False):
        loss = ctypes.c_double()
        g = np.empty(self.P, dtype=np.float32) if want_grad else None
        gp = g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) if want_grad else None
        self._check(self._lib.rmgtd_net_backward(self._net, ctypes.c_void_p(x), ctypes.c_void_p(t),
                                                 int(batch), ctypes.byref(loss), gp))
        return (float(loss.value), g) if want_grad else float(loss.value)

    def adam(self, lr: float):
        self._check(self._lib.rmgtd_net_adam(self._net, float(lr)))


class Batch:
    """Several contexts stepped by one CUDA graph per time step (rmgtd_batch)."""

    def __init__(self, ctxs):
        self._lib = load_library()
        self.ctxs = list(ctxs)
        arr = (ctypes.c_void_p * len(self.ctxs))(*[c._ctx.value for c in self.ctxs])
        self._b = ctypes.c_void_p()
        rc = self._lib.rmgtd_batch_create(arr, len(self.ctxs), ctypes.byref(self._b))
        if rc != OK:
            raise RmgtdError(rc, self._lib.rmgtd_last_error(None).decode())

    def step(self, nsteps: int = 1):
        bufs = [(CStats * max(1, nsteps * c.nrep))() for c in self.ctxs]
        ptrs = (ctypes.POINTER(CStats) * len(bufs))(*[ctypes.cast(b, ctypes.POINTER(CStats)) for b in bufs])
        rc = self._lib.rmgtd_batch_step(self._b, int(nsteps), ptrs)
        if rc != OK:
            raise RmgtdError(rc, self._lib.rmgtd_last_error(None).decode())
        return [c._stats_array(b, nsteps) for c, b in zip(self.ctxs, bufs)]

    def close(self):
        if getattr(self, "_b", None) and self._b.value:
            self._lib.rmgtd_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def spectrum(dipole, dt: float, kappa: float, gamma: float, omega) -> np.ndarray:
    """Dipole strength function S(omega) of the kicked runs (rmgtd_spectrum): `dipole` is
    (nq, nt), row q the component along the kick of the run kicked along q."""
    lib = load_library()
    d = np.ascontiguousarray(np.atleast_2d(np.asarray(dipole, dtype=np.float64)))
    om = np.ascontiguousarray(np.asarray(omega, dtype=np.float64).reshape(-1))
    out = np.empty(om.size, dtype=np.float64)
    rc = lib.rmgtd_spectrum(_dptr(d), int(d.shape[0]), int(d.shape[1]), float(dt), float(kappa),
                            float(gamma), _dptr(om), int(om.size), _dptr(out))
    if rc != OK:
        raise RmgtdError(rc, lib.rmgtd_last_error(None).decode())
    return out
