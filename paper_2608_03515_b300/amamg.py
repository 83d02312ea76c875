"""Thin ctypes binding of libamamg.so (include/amamg.h).

Argument marshalling only: every function here forwards to the C entry point of
the same name, passing device pointers of caller-owned PyTorch tensors and the
current CUDA stream.  There is no fallback: if the library cannot be loaded,
importing this module raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import List, Optional, Sequence

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libamamg.so")

OK = 0
NOT_CONVERGED = 1
ERR_INVALID_ARG = -1
ERR_OOM = -2
ERR_CUDA = -3
ERR_SINGULAR = -4
ERR_NONFINITE = -5
ERR_TIMEOUT = -6
F64 = 0
F32 = 1
SOLVE_FP64 = 0
SOLVE_MIXED = 1
MAX_LEVELS = 4
NORM_NONE = 0
NORM_ROWSUM = 1
OWNER_TILE = 0
OWNER_FIRST_LEX = 1
COARSEST_DIRECT = 0
COARSEST_GMRES = 1
F32_F64 = 2
GS_FP64 = 0
GS_DF64 = 1
GS_CGS2 = 0
GS_MGS = 1

EXPORTED = [
    "amamg_default_params", "amamg_query_bytes", "amamg_setup", "amamg_solve", "amamg_apply_D",
    "amamg_apply_Ddag", "amamg_cgnr", "amamg_coarsest_apply", "amamg_query_smoother",
    "amamg_apply_P", "amamg_apply_PH", "amamg_apply_coarse", "amamg_smooth", "amamg_coarsest_solve",
    "amamg_vcycle", "amamg_vcycle_noalloc", "amamg_selftest_sync_timeout", "amamg_sync_status", "amamg_export_structure", "amamg_level_info", "amamg_export_P", "amamg_export_coarse",
    "amamg_profile_enable", "amamg_profile_reset", "amamg_profile_get", "amamg_launch_count",
    "amamg_setup_seconds", "amamg_destroy", "amamg_status_string", "amamg_last_error",
    "amamg_batch_create", "amamg_batch_admit", "amamg_batch_cycle", "amamg_batch_retire", "amamg_batch_destroy",
]


class Params(ctypes.Structure):
    _fields_ = [
        ("nlevels", ctypes.c_int),
        ("agg", ctypes.c_int * MAX_LEVELS),
        ("precision", ctypes.c_int),
        ("restart", ctypes.c_int),
        ("max_iter", ctypes.c_int),
        ("post_smooth", ctypes.c_int),
        ("tol", ctypes.c_double),
        ("spin_split", ctypes.c_int),
        ("normalization", ctypes.c_int),
        ("edge_owner", ctypes.c_int),
        ("coarsest", ctypes.c_int),
        ("gs_arith", ctypes.c_int),
        ("autotune", ctypes.c_int),
        ("gs_method", ctypes.c_int),
    ]


class SlotInfo(ctypes.Structure):
    _fields_ = [("active", ctypes.c_int), ("done", ctypes.c_int), ("status", ctypes.c_int),
                ("iterations", ctypes.c_int), ("true_relres", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("status", ctypes.c_int), ("true_relres", ctypes.c_double)]


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libamamg.so is not built ({LIB_PATH}); run paper_2608_03515_b300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, ci, cd = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "amamg_default_params": ([ctypes.POINTER(Params)], ci),
        "amamg_query_bytes": ([ctypes.POINTER(Params), ci, ci, ci, ctypes.POINTER(ctypes.c_size_t),
                               ctypes.POINTER(ctypes.c_size_t)], ci),
        "amamg_setup": ([ctypes.POINTER(Params), vp, ci, ci, cd, vp, ctypes.POINTER(vp)], ci),
        "amamg_solve": ([vp, vp, vp, ci, vp, ctypes.POINTER(SolveInfo)], ci),
        "amamg_apply_D": ([vp, vp, vp, ci, ci, vp], ci),
        "amamg_apply_Ddag": ([vp, vp, vp, ci, vp], ci),
        "amamg_cgnr": ([vp, vp, vp, ci, ci, cd, vp, ctypes.POINTER(SolveInfo)], ci),
        "amamg_apply_P": ([vp, ci, vp, vp, ci, ci, vp], ci),
        "amamg_apply_PH": ([vp, ci, vp, vp, ci, ci, vp], ci),
        "amamg_apply_coarse": ([vp, ci, vp, vp, ci, ci, vp], ci),
        "amamg_smooth": ([vp, ci, vp, vp, ci, ci, ci, vp], ci),
        "amamg_coarsest_solve": ([vp, vp, vp, ci, vp], ci),
        "amamg_coarsest_apply": ([vp, vp, vp, ci, ci, vp], ci),
        "amamg_query_smoother": ([vp, ci, ci, ci, ctypes.POINTER(ci), ctypes.POINTER(ci)], ci),
        "amamg_vcycle": ([vp, vp, vp, ci, ci, vp], ci),
        "amamg_vcycle_noalloc": ([vp, vp, vp, ci, ci, vp], ci),
        "amamg_selftest_sync_timeout": ([vp, ci, ci, vp], ci),
        "amamg_sync_status": ([vp, vp], ci),
        "amamg_export_structure": ([vp, ci, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                    ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)], ci),
        "amamg_level_info": ([vp, ci, ctypes.POINTER(ci), ctypes.POINTER(ci), ctypes.POINTER(ci)], ci),
        "amamg_export_P": ([vp, ci, vp, vp], ci),
        "amamg_export_coarse": ([vp, ci, vp, vp], ci),
        "amamg_profile_enable": ([vp, ci], ci),
        "amamg_profile_reset": ([vp], ci),
        "amamg_profile_get": ([vp, ci, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_longlong),
                               ctypes.POINTER(cd), ctypes.POINTER(cd), ctypes.POINTER(cd)], ci),
        "amamg_launch_count": ([vp], ctypes.c_longlong),
        "amamg_setup_seconds": ([vp], cd),
        "amamg_destroy": ([vp], ci),
        "amamg_status_string": ([ci], ctypes.c_char_p),
        "amamg_last_error": ([vp], ctypes.c_char_p),
        "amamg_batch_create": ([vp, ci, ctypes.POINTER(vp)], ci),
        "amamg_batch_admit": ([vp, ci, vp, cd, vp], ci),
        "amamg_batch_cycle": ([vp, vp, ctypes.POINTER(SlotInfo)], ci),
        "amamg_batch_retire": ([vp, ci, vp, vp], ci),
        "amamg_batch_destroy": ([vp], ci),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_lib = _load()


class AmamgError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where}: {_lib.amamg_status_string(status).decode()} ({status})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


def lib() -> ctypes.CDLL:
    return _lib


def _stream(stream=None) -> ctypes.c_void_p:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t) -> ctypes.c_void_p:
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _prec(t) -> int:
    import torch
    if t.dtype == torch.complex128:
        return F64
    if t.dtype == torch.complex64:
        return F32
    raise ValueError(f"vectors must be complex128 or complex64, got {t.dtype}")


def default_params() -> Params:
    p = Params()
    _lib.amamg_default_params(ctypes.byref(p))
    return p


def make_params(aggs: Sequence[int], precision: int = SOLVE_FP64, restart: int = 30, max_iter: int = 3000,
                post_smooth: int = 2, tol: float = 1e-10, spin_split: bool = False,
                normalization: str = "none", ownership: str = "tile", coarsest: str = "direct",
                gs: str = "fp64", autotune: bool = False, gs_method: str = "cgs2") -> Params:
    """Parameters of amamg_setup; normalization "none" | "rowsum" and ownership
    "tile" | "first_lex" name the readings the oracle's build_hierarchy takes;
    coarsest "direct" | "gmres" the coarsest solver (the oracle's vcycle
    coarsest="lu" | "gmres"); gs "fp64" | "df64" the outer Gram-Schmidt's
    arithmetic (df64 with mixed precision only); gs_method "cgs2" | "mgs" its
    variant (classical with DGKS-gated second pass, or modified as in the
    oracle; mgs with fp64 arithmetic only); autotune: time the coarse
    Gauss-Seidel candidates at the first solve of each right-hand-side count."""
    p = default_params()
    p.nlevels = len(aggs) + 1
    for i, a in enumerate(aggs):
        p.agg[i] = int(a)
    p.precision = precision
    p.restart = restart
    p.max_iter = max_iter
    p.post_smooth = post_smooth
    p.tol = tol
    p.spin_split = 1 if spin_split else 0
    p.normalization = {"none": NORM_NONE, "rowsum": NORM_ROWSUM}[normalization]
    p.edge_owner = {"tile": OWNER_TILE, "first_lex": OWNER_FIRST_LEX}[ownership]
    p.coarsest = {"direct": COARSEST_DIRECT, "gmres": COARSEST_GMRES}[coarsest]
    p.gs_arith = {"fp64": GS_FP64, "df64": GS_DF64}[gs]
    p.autotune = 1 if autotune else 0
    p.gs_method = {"cgs2": GS_CGS2, "mgs": GS_MGS}[gs_method]
    return p


def query_bytes(params: Params, Nt: int, Nx: int, max_rhs: int = 1):
    sb, rb = ctypes.c_size_t(), ctypes.c_size_t()
    st = _lib.amamg_query_bytes(ctypes.byref(params), Nt, Nx, max_rhs, ctypes.byref(sb), ctypes.byref(rb))
    if st != OK:
        raise AmamgError(st, "amamg_query_bytes")
    return sb.value, rb.value


@dataclass
class Info:
    iterations: int
    status: int
    true_relres: float


class Hierarchy:
    """Owns one amamg_handle (setup result); destroyed with the object."""

    def __init__(self, handle: ctypes.c_void_p, params: Params, Nt: int, Nx: int, m0: float):
        self.h = handle
        self.params = params
        self.Nt, self.Nx, self.m0 = Nt, Nx, m0

    def _check(self, st: int, where: str):
        if st < 0:
            raise AmamgError(st, where, _lib.amamg_last_error(self.h).decode())
        return st

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            try:
                _lib.amamg_destroy(h)
            except Exception:
                pass
            self.h = ctypes.c_void_p()

    def destroy(self):
        self.__del__()

    # ---- levels
    def level_info(self, level: int):
        nt, nx, k = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(_lib.amamg_level_info(self.h, level, ctypes.byref(nt), ctypes.byref(nx), ctypes.byref(k)),
                    "amamg_level_info")
        return nt.value, nx.value, k.value

    @property
    def nlevels(self) -> int:
        return self.params.nlevels


def setup(U, m0: float, params: Params, stream=None) -> Hierarchy:
    """amamg_setup: U complex128 [2, Nt, Nx] on the device."""
    import torch
    if U.dtype != torch.complex128 or U.dim() != 3 or U.shape[0] != 2:
        raise ValueError("U must be complex128 [2, Nt, Nx]")
    Nt, Nx = int(U.shape[1]), int(U.shape[2])
    h = ctypes.c_void_p()
    st = _lib.amamg_setup(ctypes.byref(params), _ptr(U), Nt, Nx, float(m0), _stream(stream), ctypes.byref(h))
    if st != OK:
        raise AmamgError(st, "amamg_setup")
    return Hierarchy(h, params, Nt, Nx, float(m0))


def apply_Ddag(hier: Hierarchy, inp, out, stream=None):
    """amamg_apply_Ddag: out = sigma_3 D sigma_3 in (complex128)."""
    hier._check(_lib.amamg_apply_Ddag(hier.h, _ptr(inp), _ptr(out), int(inp.shape[0]), _stream(stream)),
                "amamg_apply_Ddag")


def cgnr(hier: Hierarchy, psi, x, max_iter: int = 100000, tol: float = 1e-10, stream=None) -> List["Info"]:
    """amamg_cgnr: CG on the normal equations; psi, x complex128 [R, 2, Nt, Nx]."""
    R = int(psi.shape[0])
    info = (SolveInfo * R)()
    st = _lib.amamg_cgnr(hier.h, _ptr(psi), _ptr(x), R, int(max_iter), float(tol), _stream(stream), info)
    hier._check(st, "amamg_cgnr")
    return [Info(i.iterations, i.status, i.true_relres) for i in info]


def solve(hier: Hierarchy, psi, x, stream=None) -> List[Info]:
    """amamg_solve: psi, x complex128 [R, 2, Nt, Nx]; returns per-RHS info."""
    R = int(psi.shape[0])
    info = (SolveInfo * R)()
    st = _lib.amamg_solve(hier.h, _ptr(psi), _ptr(x), R, _stream(stream), info)
    hier._check(st, "amamg_solve")
    return [Info(i.iterations, i.status, i.true_relres) for i in info]


def apply_D(hier: Hierarchy, inp, out, stream=None):
    """out = D inp; complex64 inp with complex128 out is the FP64 stencil of the
    widened input (AMAMG_F32_F64), else both of one precision."""
    import torch
    R = int(inp.shape[0])
    prec = F32_F64 if (inp.dtype == torch.complex64 and out.dtype == torch.complex128) else _prec(inp)
    hier._check(_lib.amamg_apply_D(hier.h, _ptr(inp), _ptr(out), R, prec, _stream(stream)), "amamg_apply_D")


def apply_P(hier: Hierarchy, level: int, coarse_in, fine_out, stream=None):
    R = int(coarse_in.shape[0])
    hier._check(_lib.amamg_apply_P(hier.h, level, _ptr(coarse_in), _ptr(fine_out), R, _prec(coarse_in),
                                   _stream(stream)), "amamg_apply_P")


def apply_PH(hier: Hierarchy, level: int, fine_in, coarse_out, stream=None):
    R = int(fine_in.shape[0])
    hier._check(_lib.amamg_apply_PH(hier.h, level, _ptr(fine_in), _ptr(coarse_out), R, _prec(fine_in),
                                    _stream(stream)), "amamg_apply_PH")


def apply_coarse(hier: Hierarchy, level: int, inp, out, stream=None):
    R = int(inp.shape[0])
    hier._check(_lib.amamg_apply_coarse(hier.h, level, _ptr(inp), _ptr(out), R, _prec(inp), _stream(stream)),
                "amamg_apply_coarse")


def smooth(hier: Hierarchy, level: int, r, e, sweeps: int, stream=None):
    R = int(r.shape[0])
    hier._check(_lib.amamg_smooth(hier.h, level, _ptr(r), _ptr(e), R, sweeps, _prec(r), _stream(stream)),
                "amamg_smooth")


def coarsest_solve(hier: Hierarchy, r, e, stream=None):
    R = int(r.shape[0])
    hier._check(_lib.amamg_coarsest_solve(hier.h, _ptr(r), _ptr(e), R, _stream(stream)), "amamg_coarsest_solve")


def coarsest_apply(hier: Hierarchy, r, e, stream=None):
    """amamg_coarsest_apply in the precision of r (complex128 or complex64)."""
    R = int(r.shape[0])
    hier._check(_lib.amamg_coarsest_apply(hier.h, _ptr(r), _ptr(e), R, _prec(r), _stream(stream)),
                "amamg_coarsest_apply")


def vcycle(hier: Hierarchy, r, e, stream=None):
    R = int(r.shape[0])
    hier._check(_lib.amamg_vcycle(hier.h, _ptr(r), _ptr(e), R, _prec(r), _stream(stream)), "amamg_vcycle")


def vcycle_noalloc(hier: Hierarchy, r, e, stream=None):
    """amamg_vcycle_noalloc: the V-cycle without device allocation (fixed scratch array)."""
    R = int(r.shape[0])
    hier._check(_lib.amamg_vcycle_noalloc(hier.h, _ptr(r), _ptr(e), R, _prec(r), _stream(stream)),
                "amamg_vcycle_noalloc")


def selftest_sync_timeout(hier: Hierarchy, level: int, precision: int = None, stream=None) -> int:
    """amamg_selftest_sync_timeout: enqueues one coarse smoothing in which one
    owner block withholds its phase counter; returns the raw status (OK once
    enqueued; sync_status then reports the time-out)."""
    prec = F64 if precision is None else precision
    return int(_lib.amamg_selftest_sync_timeout(hier.h, level, prec, _stream(stream)))


SMOOTHER_NAMES = {0: "colour", 1: "cluster", 2: "dsmem", 3: "grid", 4: "owner"}


def query_smoother(hier: Hierarchy, level: int, precision: int, R: int = 1):
    """amamg_query_smoother: (kernel name, owner-shape variant) that a smoothing
    of `level` with R right-hand sides in `precision` (F64 / F32) uses now."""
    k, v = ctypes.c_int(), ctypes.c_int()
    hier._check(_lib.amamg_query_smoother(hier.h, level, precision, R, ctypes.byref(k), ctypes.byref(v)),
                "amamg_query_smoother")
    return SMOOTHER_NAMES[k.value], v.value


def sync_status(hier: Hierarchy, stream=None) -> int:
    """amamg_sync_status: the raw status of the bounded-wait check (OK or
    ERR_TIMEOUT), re-arming the counters after a time-out."""
    return int(_lib.amamg_sync_status(hier.h, _stream(stream)))


def export_structure(hier: Hierarchy, level: int):
    import numpy as np
    nt, nx, _ = hier.level_info(level)
    role = np.zeros(nt * nx, dtype=np.int32)
    owner = np.zeros(nt * nx, dtype=np.int32)
    offs = np.zeros(96, dtype=np.int32)
    cnt = ctypes.c_int32()
    P = ctypes.POINTER(ctypes.c_int32)
    hier._check(_lib.amamg_export_structure(hier.h, level, role.ctypes.data_as(P), owner.ctypes.data_as(P),
                                            offs.ctypes.data_as(P), ctypes.byref(cnt)), "amamg_export_structure")
    K = cnt.value
    return role.reshape(nt, nx), owner.reshape(nt, nx), [(int(offs[2 * k]), int(offs[2 * k + 1])) for k in range(K)]


def export_P(hier: Hierarchy, level: int, out, stream=None):
    hier._check(_lib.amamg_export_P(hier.h, level, _ptr(out), _stream(stream)), "amamg_export_P")


def export_coarse(hier: Hierarchy, level: int, out, stream=None):
    hier._check(_lib.amamg_export_coarse(hier.h, level, _ptr(out), _stream(stream)), "amamg_export_coarse")


def profile_enable(hier: Hierarchy, on: bool):
    hier._check(_lib.amamg_profile_enable(hier.h, int(bool(on))), "amamg_profile_enable")


def profile_reset(hier: Hierarchy):
    hier._check(_lib.amamg_profile_reset(hier.h), "amamg_profile_reset")


def profile_get(hier: Hierarchy):
    """[(name, launches, total_ms, bytes, flops)] for every kernel category seen."""
    out = []
    i = 0
    while True:
        name = ctypes.c_char_p()
        n = ctypes.c_longlong()
        ms = ctypes.c_double()
        by = ctypes.c_double()
        fl = ctypes.c_double()
        st = _lib.amamg_profile_get(hier.h, i, ctypes.byref(name), ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by),
                                    ctypes.byref(fl))
        if st != OK:
            break
        out.append((name.value.decode(), n.value, ms.value, by.value, fl.value))
        i += 1
    return out


def launch_count(hier: Hierarchy) -> int:
    return int(_lib.amamg_launch_count(hier.h))


def setup_seconds(hier: Hierarchy) -> float:
    return float(_lib.amamg_setup_seconds(hier.h))


def destroy(hier: Hierarchy):
    hier.destroy()


class Batch:
    """amamg_batch_*: S right-hand-side slots on one hierarchy (continuous batching).

    admit() puts a right-hand side (device complex128 [2, Nt, Nx]) with its own
    mass into a free slot, cycle() runs one FGMRES restart cycle over all
    occupied slots, retire() copies a slot's solution out and frees the slot."""

    def __init__(self, hier: Hierarchy, slots: int):
        self.hier = hier
        self.slots = slots
        self.b = ctypes.c_void_p()
        hier._check(_lib.amamg_batch_create(hier.h, slots, ctypes.byref(self.b)), "amamg_batch_create")

    def admit(self, slot: int, psi, m0: float, stream=None):
        self.hier._check(_lib.amamg_batch_admit(self.b, slot, _ptr(psi), float(m0), _stream(stream)),
                         "amamg_batch_admit")

    def cycle(self, stream=None):
        info = (SlotInfo * self.slots)()
        self.hier._check(_lib.amamg_batch_cycle(self.b, _stream(stream), info), "amamg_batch_cycle")
        return [(i.active, i.done, i.status, i.iterations, i.true_relres) for i in info]

    def retire(self, slot: int, x=None, stream=None):
        self.hier._check(_lib.amamg_batch_retire(self.b, slot, _ptr(x) if x is not None else None,
                                                 _stream(stream)), "amamg_batch_retire")

    def destroy(self):
        if self.b is not None and self.b.value:
            _lib.amamg_batch_destroy(self.b)
            self.b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
