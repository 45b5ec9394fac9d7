"""Thin ctypes binding of libhfx.so (the C ABI in include/hfx.h).

Argument marshalling only: every step of the evaluation runs in the
library's CUDA kernels.  The binding refuses to run if libhfx.so has not
been built (no fallback of any kind).
"""
from __future__ import annotations

import ctypes as ct
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhfx.so")

HFX_OK = 0
HFX_FP64, HFX_BF16X3, HFX_BF16X6 = 0, 2, 3
STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "CUDA error", 4: "timeout",
          5: "pair list stale", 6: "unsupported"}

_dp = ct.POINTER(ct.c_double)
_ip = ct.POINTER(ct.c_int)
_llp = ct.POINTER(ct.c_longlong)


class HfxSystem(ct.Structure):
    _fields_ = [("n_atoms", ct.c_int), ("species", _ip), ("lattice", ct.c_double * 9), ("positions", _dp)]


class HfxModel(ct.Structure):
    _fields_ = [("n_species", ct.c_int), ("n_ao", _ip), ("n_abf", _ip), ("r_c", ct.c_double),
                ("omega", ct.c_double), ("G", ct.POINTER(_dp)), ("M", ct.POINTER(_dp)),
                ("G_aniso", ct.POINTER(_dp)), ("aniso_dir", ct.c_double * 3), ("n_d", ct.c_longlong),
                ("d_index", _ip), ("d_offset", _llp), ("d_values", _dp)]


ALLOC_FN = ct.CFUNCTYPE(ct.c_void_p, ct.c_size_t, ct.c_void_p, ct.c_void_p)
FREE_FN = ct.CFUNCTYPE(None, ct.c_void_p, ct.c_size_t, ct.c_void_p, ct.c_void_p)


class HfxOptions(ct.Structure):
    _fields_ = [("theta_C", ct.c_double), ("theta_dC", ct.c_double), ("theta_V", ct.c_double),
                ("theta_dV", ct.c_double), ("theta_D", ct.c_double), ("theta_CS", ct.c_double),
                ("precision", ct.c_int), ("terms", ct.c_int), ("skin", ct.c_double),
                ("freeze_lists", ct.c_int), ("home_begin", ct.c_int), ("home_end", ct.c_int),
                ("home_chunk", ct.c_int), ("graph", ct.c_int), ("stream", ct.c_void_p), ("device", ct.c_int),
                ("alloc", ALLOC_FN),
                ("free", FREE_FN), ("alloc_ctx", ct.c_void_p), ("deterministic", ct.c_int)]


class HfxTuneReport(ct.Structure):
    _fields_ = [("candidates", ct.c_int), ("t1_rows_per_slot", ct.c_int), ("t1_slots", ct.c_int),
                ("default_ms", ct.c_double), ("best_ms", ct.c_double), ("t1_home_order", ct.c_int),
                ("y_tiles_per_cta", ct.c_int), ("q2_tiles_per_cta", ct.c_int)]


class HfxStats(ct.Structure):
    _fields_ = [("c_pairs", ct.c_longlong), ("v_pairs", ct.c_longlong), ("d_blocks", ct.c_longlong),
                ("triplets", ct.c_longlong), ("term1_pairs", ct.c_longlong), ("term2_pairs", ct.c_longlong),
                ("y_blocks", ct.c_longlong), ("flops_y", ct.c_double), ("flops_term1", ct.c_double),
                ("flops_term2", ct.c_double), ("flops_total", ct.c_double), ("ms_blocks", ct.c_double),
                ("ms_screen", ct.c_double), ("ms_y", ct.c_double), ("ms_term1", ct.c_double),
                ("ms_term2", ct.c_double), ("ms_reduce", ct.c_double), ("ms_total", ct.c_double),
                ("device_bytes", ct.c_longlong), ("kernel_launches", ct.c_longlong), ("passes", ct.c_int),
                ("graph_replayed", ct.c_int),
                ("ms_term1_kernel", ct.c_double), ("ms_term2_kernel", ct.c_double),
                ("ref_err_E", ct.c_double), ("ref_err_F", ct.c_double), ("ref_err_sigma", ct.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# Every symbol include/hfx.h declares, with its ctypes signature.
_SIGNATURES = {
    "hfx_default_options": (ct.c_int, [ct.POINTER(HfxOptions)]),
    "hfx_plan_create": (ct.c_int, [ct.POINTER(HfxSystem), ct.POINTER(HfxModel), ct.POINTER(HfxOptions),
                                   ct.POINTER(ct.c_void_p)]),
    "hfx_energy_force_stress": (ct.c_int, [ct.c_void_p, _dp, _dp, _dp, _dp, _dp, ct.POINTER(HfxStats)]),
    "hfx_energy_force_stress_device": (ct.c_int, [ct.c_void_p, _dp, ct.c_void_p, ct.c_void_p,
                                                  ct.POINTER(HfxStats)]),
    "hfx_energy_force_stress_noalloc": (ct.c_int, [ct.c_void_p, _dp, _dp, _dp, _dp, _dp]),
    "hfx_set_timing": (ct.c_int, [ct.c_void_p, ct.c_int]),
    "hfx_set_reference": (ct.c_int, [ct.c_void_p, _dp, _dp, _dp]),
    "hfx_plan_autotune": (ct.c_int, [ct.c_void_p, _dp, _dp, ct.c_int, ct.c_void_p]),
    "hfx_lri_fit": (ct.c_int, [ct.c_int, ct.c_int, ct.c_int, _dp, _dp, _dp, _dp, _dp, _dp, ct.c_int]),
    "hfx_plan_destroy": (ct.c_int, [ct.c_void_p]),
    "hfx_status_string": (ct.c_char_p, [ct.c_int]),
    "hfx_last_error": (ct.c_char_p, [ct.c_void_p]),
}

_lib: Optional[ct.CDLL] = None


def load_library(path: str = LIB_PATH) -> ct.CDLL:
    """Load libhfx.so and bind its signatures.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libhfx.so is not built at {path}; run paper_2412_11081_gb300.build.build()")
    lib = ct.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class HfxError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _check(lib, status, plan=None):
    if status != HFX_OK:
        msg = lib.hfx_last_error(plan)
        raise HfxError(status, msg.decode() if msg else "")


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def default_options(**kw) -> HfxOptions:
    lib = load_library()
    o = HfxOptions()
    _check(lib, lib.hfx_default_options(ct.byref(o)))
    for k, v in kw.items():
        if k == "stream":
            v = int(v) if v else None
        setattr(o, k, v)
    return o


class Plan:
    """A device-resident plan for one structure (hfx_plan_create).

    `w` is any object with the workload attributes species, lattice,
    positions, n_ao, n_abf, r_c, omega, G, M, d_index, d_offset, d_values
    and theta (dict with keys C, dC, V, dV, D, CS).
    """

    def __init__(self, w, *, precision: int = HFX_FP64, terms: int = 3, skin: float = 0.5,
                 freeze_lists: bool = False, stream: Optional[int] = None, device: int = 0,
                 theta: Optional[dict] = None, aniso=None, allocator=None, home=None, home_chunk: int = 0,
                 graph: bool = False, deterministic: bool = False):
        self.lib = load_library()
        th = dict(w.theta) if theta is None else dict(theta)
        if stream is None:
            stream = _current_stream()
        hb, he = (0, 0) if home is None else (int(home[0]), int(home[1]))
        self.opts = default_options(theta_C=th["C"], theta_dC=th["dC"], theta_V=th["V"], theta_dV=th["dV"],
                                    theta_D=th["D"], theta_CS=th["CS"], precision=precision, terms=terms,
                                    skin=skin, freeze_lists=int(freeze_lists), stream=stream, device=device,
                                    home_begin=hb, home_end=he, home_chunk=int(home_chunk), graph=int(graph),
                                    deterministic=int(deterministic))
        # allocator="torch": the plan's device memory comes from PyTorch's
        # caching allocator (hfx_options alloc / free); a pair of callables
        # (alloc(nbytes) -> device address or 0, free(address, nbytes)) is
        # wrapped the same way.  The callbacks live as long as the plan.
        self._hooks = None
        if allocator == "torch":
            self._hooks = _torch_hooks(device)
        elif isinstance(allocator, tuple) and len(allocator) == 2:
            a_fn, f_fn = allocator
            self._hooks = (ALLOC_FN(lambda n, s, c: a_fn(int(n)) or None),
                           FREE_FN(lambda p, n, s, c: f_fn(int(p), int(n))))
        elif allocator is not None:
            raise ValueError("allocator must be None, 'torch' or (alloc, free)")
        if self._hooks is not None:
            self.opts.alloc, self.opts.free = self._hooks
        self.n_atoms = int(np.asarray(w.species).shape[0])
        # keep every marshalled array alive for the duration of the create call
        self._keep = []
        species = np.ascontiguousarray(w.species, dtype=np.int32)
        pos = _f64(w.positions)
        sysm = HfxSystem()
        sysm.n_atoms = self.n_atoms
        sysm.species = species.ctypes.data_as(_ip)
        sysm.lattice = (ct.c_double * 9)(*_f64(w.lattice).ravel())
        sysm.positions = pos.ctypes.data_as(_dp)
        S = int(np.asarray(w.n_ao).shape[0])
        n_ao = np.ascontiguousarray(w.n_ao, dtype=np.int32)
        n_abf = np.ascontiguousarray(w.n_abf, dtype=np.int32)
        G = [_f64(g) for g in w.G]
        M = [_f64(m) for m in w.M]
        Gptr = (_dp * (S * S))(*[g.ctypes.data_as(_dp) for g in G])
        Mptr = (_dp * (S * S))(*[m.ctypes.data_as(_dp) for m in M])
        model = HfxModel()
        model.n_species = S
        model.n_ao = n_ao.ctypes.data_as(_ip)
        model.n_abf = n_abf.ctypes.data_as(_ip)
        model.r_c = float(w.r_c)
        model.omega = float(w.omega)
        model.G = Gptr
        model.M = Mptr
        Gp = None
        if aniso is not None:
            Gp = [_f64(g) for g in aniso[0]]
            model.G_aniso = (_dp * (S * S))(*[g.ctypes.data_as(_dp) for g in Gp])
            model.aniso_dir = (ct.c_double * 3)(*_f64(aniso[1]))
        d_index = np.ascontiguousarray(w.d_index, dtype=np.int32)
        d_offset = np.ascontiguousarray(w.d_offset, dtype=np.int64)
        d_values = _f64(w.d_values)
        model.n_d = int(d_index.shape[0])
        model.d_index = d_index.ctypes.data_as(_ip)
        model.d_offset = d_offset.ctypes.data_as(_llp)
        model.d_values = d_values.ctypes.data_as(_dp)
        self._keep = [species, pos, n_ao, n_abf, G, M, Gp, d_index, d_offset, d_values, Gptr, Mptr]
        handle = ct.c_void_p()
        st = self.lib.hfx_plan_create(ct.byref(sysm), ct.byref(model), ct.byref(self.opts), ct.byref(handle))
        self._keep = None
        _check(self.lib, st, None)
        self.handle = handle
        self.stats = HfxStats()

    def set_timing(self, on: bool = True):
        _check(self.lib, self.lib.hfx_set_timing(self.handle, int(on)), self.handle)

    def set_reference(self, E=None, F=None, sigma=None):
        """hfx_set_reference: later stats report their error against (E, F,
        sigma); no arguments clear it."""
        if E is None and F is None and sigma is None:
            st = self.lib.hfx_set_reference(self.handle, None, None, None)
        else:
            e = np.array([float(E)])
            f, s = _f64(F).ravel(), _f64(sigma).ravel()
            if f.size != 3 * self.n_atoms or s.size != 9:
                raise ValueError("F must be n_atoms x 3 and sigma 3 x 3")
            st = self.lib.hfx_set_reference(self.handle, e.ctypes.data_as(_dp), f.ctypes.data_as(_dp),
                                            s.ctypes.data_as(_dp))
        _check(self.lib, st, self.handle)

    def evaluate(self, lattice, positions, stats: bool = False):
        """E, F (n x 3), sigma (3 x 3) at the given geometry (host arrays)."""
        lat = _f64(lattice).ravel()
        pos = _f64(positions).ravel()
        if pos.size != 3 * self.n_atoms:
            raise ValueError("positions must be n_atoms x 3")
        E = ct.c_double()
        F = np.zeros((self.n_atoms, 3))
        sig = np.zeros((3, 3))
        st = self.lib.hfx_energy_force_stress(self.handle, lat.ctypes.data_as(_dp), pos.ctypes.data_as(_dp),
                                              ct.byref(E), F.ctypes.data_as(_dp), sig.ctypes.data_as(_dp),
                                              ct.byref(self.stats) if stats else None)
        _check(self.lib, st, self.handle)
        return float(E.value), F, sig

    def autotune(self, lattice, positions, reps: int = 3) -> dict:
        """hfx_plan_autotune: time the launch configurations that leave the
        arithmetic unchanged at this geometry and keep the fastest."""
        lat = _f64(lattice).ravel()
        pos = _f64(positions).ravel()
        if pos.size != 3 * self.n_atoms:
            raise ValueError("positions must be n_atoms x 3")
        rep = HfxTuneReport()
        st = self.lib.hfx_plan_autotune(self.handle, lat.ctypes.data_as(_dp), pos.ctypes.data_as(_dp), int(reps),
                                        ct.byref(rep))
        _check(self.lib, st, self.handle)
        return {k: getattr(rep, k) for k, _ in rep._fields_}

    def evaluate_noalloc(self, lattice, positions):
        """hfx_energy_force_stress_noalloc: the FP64 evaluation with its
        scratch in the library's fixed device array (no device allocation)."""
        lat = _f64(lattice).ravel()
        pos = _f64(positions).ravel()
        if pos.size != 3 * self.n_atoms:
            raise ValueError("positions must be n_atoms x 3")
        E = ct.c_double()
        F = np.zeros((self.n_atoms, 3))
        sig = np.zeros((3, 3))
        st = self.lib.hfx_energy_force_stress_noalloc(self.handle, lat.ctypes.data_as(_dp), pos.ctypes.data_as(_dp),
                                                      ct.byref(E), F.ctypes.data_as(_dp), sig.ctypes.data_as(_dp))
        _check(self.lib, st, self.handle)
        return float(E.value), F, sig

    def evaluate_device(self, lattice, d_positions_ptr: int, d_out_ptr: int, stats: bool = False):
        """Device-memory variant: positions and [E, F, sigma] live in device memory."""
        lat = _f64(lattice).ravel()
        st = self.lib.hfx_energy_force_stress_device(self.handle, lat.ctypes.data_as(_dp),
                                                     ct.c_void_p(d_positions_ptr), ct.c_void_p(d_out_ptr),
                                                     ct.byref(self.stats) if stats else None)
        _check(self.lib, st, self.handle)

    def close(self):
        if getattr(self, "handle", None):
            self.lib.hfx_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def lri_fit(A, B, dA=None, dB=None, device: int = 0):
    """hfx_lri_fit: X = A^-1 B per pair (Eq. C_VA) and, with dA and dB,
    dX[c] = A^-1 (dB[c] - dA[c] X).  A [batch, n, n], B [batch, n, w],
    dA [batch, 3, n, n], dB [batch, 3, n, w]; returns X (and dX)."""
    lib = load_library()
    A, B = _f64(A), _f64(B)
    if A.ndim != 3 or B.ndim != 3 or A.shape[1] != A.shape[2] or B.shape[:2] != A.shape[:2]:
        raise ValueError("A must be [batch, n, n] and B [batch, n, w]")
    batch, n, w = B.shape
    X = np.zeros((batch, n, w))
    grad = dA is not None or dB is not None
    if grad:
        dA, dB = _f64(dA), _f64(dB)
        if dA.shape != (batch, 3, n, n) or dB.shape != (batch, 3, n, w):
            raise ValueError("dA must be [batch, 3, n, n] and dB [batch, 3, n, w]")
        dX = np.zeros((batch, 3, n, w))
    ptr = lambda a: a.ctypes.data_as(_dp) if a is not None else None
    st = lib.hfx_lri_fit(batch, n, w, ptr(A), ptr(B), ptr(dA) if grad else None, ptr(dB) if grad else None,
                         ptr(X), ptr(dX) if grad else None, device)
    _check(lib, st, None)
    return (X, dX) if grad else X


def _torch_hooks(device: int):
    """hfx_options alloc / free over torch.cuda's caching allocator."""
    import torch

    def alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device, int(stream or 0))
        except RuntimeError:
            return None

    def free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    return ALLOC_FN(alloc), FREE_FN(free)


def _current_stream() -> int:
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return 0
