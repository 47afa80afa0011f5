"""ctypes binding of libspg (include/spg.h).

Argument marshalling only: every step of the method runs in the CUDA library.
The module fails at import when the library cannot be loaded; there is no
other implementation behind it.
"""
from __future__ import annotations

import atexit
import ctypes as C
import os
import weakref

import numpy as np

from . import build as _build

SPG_OK = 0
SPG_EINVAL = -1
SPG_EINEXACT = -2
SPG_ENOMEM = -3
SPG_ECUDA = -4
SPG_ETIMEOUT = -5
SPG_ENUMERIC = -6
SPG_EUNSUPPORTED = -7
SPG_SQUARE = 0
SPG_KING = 1
SPG_FP64 = 0
SPG_MIXED = 1

_ERRNAMES = {v: k for k, v in dict(SPG_EINVAL=-1, SPG_EINEXACT=-2, SPG_ENOMEM=-3, SPG_ECUDA=-4,
                                   SPG_ETIMEOUT=-5, SPG_ENUMERIC=-6, SPG_EUNSUPPORTED=-7).items()}


class spg_params(C.Structure):
    _fields_ = [("beta", C.c_double), ("chi", C.c_int32), ("num_sweeps", C.c_int32),
                ("beam", C.c_int32), ("precision", C.c_int32), ("cut_off_prob", C.c_double),
                ("svd_iters", C.c_int32), ("warm_start", C.c_int32), ("seed", C.c_uint64),
                ("merge", C.c_int32), ("reserved", C.c_int32 * 7)]


class spg_info(C.Structure):
    _fields_ = [("n_states", C.c_int32), ("near_ties", C.c_int32), ("degenerate_cuts", C.c_int32),
                ("error_flags", C.c_int32), ("ms_boundary", C.c_double), ("ms_search", C.c_double),
                ("candidates", C.c_double), ("boundary_lognorm", C.c_double),
                ("kernel_launches", C.c_int64), ("jacobi_sweeps_max", C.c_int32), ("reserved", C.c_int32)]


def _load():
    path = _build.LIB
    if _build.needs_build():
        path = _build.build()
    if not os.path.exists(path):
        raise ImportError("libspg.so is not built (run __graft_entry__.build())")
    lib = C.CDLL(path)
    P, I32, I64, D, U16 = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_uint16
    pI32, pI64, pD, pU16 = C.POINTER(I32), C.POINTER(I64), C.POINTER(D), C.POINTER(U16)
    sig = {
        "spg_version": (C.c_int, []),
        "spg_lattice_site_map": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_int32),
                                           C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
        "spg_params_default": (C.c_int, [C.POINTER(spg_params)]),
        "spg_create": (C.c_int, [C.POINTER(P), C.c_int, P]),
        "spg_destroy": (None, [P]),
        "spg_last_error": (C.c_char_p, [P]),
        "spg_problem_ising": (C.c_int, [P, I32, I32, pI32, pI32, pD, pD, pI32, I32, I32, pI32, pI32, I32, I32,
                                        C.POINTER(P)]),
        "spg_problem_potts": (C.c_int, [P, I32, I32, pI32, pI64, I32, pI32, pI32, pI64, I32, I32, C.POINTER(P)]),
        "spg_problem_destroy": (None, [P]),
        "spg_problem_shape": (C.c_int, [P, pI32, pI32, pI32]),
        "spg_solve": (C.c_int, [P, P, C.POINTER(spg_params), C.POINTER(P)]),
        "spg_solve_batch": (C.c_int, [P, I32, C.POINTER(P), C.POINTER(spg_params), C.POINTER(P)]),
        "spg_result_get": (C.c_int, [P, pI32, pI32, pU16, pI64, pD, pD]),
        "spg_result_info": (C.c_int, [P, C.POINTER(spg_info)]),
        "spg_result_destroy": (None, [P]),
        "spg_debug_marginals": (C.c_int, [P, P, C.POINTER(spg_params), I32, I32, pU16, pD]),
        "spg_log_partition": (C.c_int, [P, P, C.POINTER(spg_params), pD]),
        "spg_truncate": (C.c_int, [P, P, I32, I32, I32, I32, P, P, P]),
        "spg_truncate_static": (C.c_int, [P, I32, I32, I32, I32, P, P, P, P]),
        "spg_tc_product": (C.c_int, [P, P, I32, I32, P, I32, I32, P]),
        "spg_profile": (C.c_int, [P, C.c_int]),
        "spg_profile_report": (C.c_int, [P, C.c_char_p, C.c_size_t]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


# Handles still open at interpreter exit are released results -> problems ->
# contexts, before the CUDA runtime is torn down.
_LIVE = {"result": weakref.WeakSet(), "problem": weakref.WeakSet(), "ctx": weakref.WeakSet()}


@atexit.register
def _close_all():
    for kind in ("result", "problem", "ctx"):
        for obj in list(_LIVE[kind]):
            try:
                obj.close()
            except Exception:
                pass


class SpgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct)) if a is not None else None


def spg_lattice_site_map(rows: int, cols: int, k: int):
    """(site_map [rows*cols] int32, new_rows, new_cols) of lattice
    transformation k (include/spg.h)."""
    out = np.zeros(rows * cols, np.int32)
    r, c = C.c_int32(), C.c_int32()
    rc = lib.spg_lattice_site_map(rows, cols, k, _ptr(out, C.c_int32), C.byref(r), C.byref(c))
    if rc != SPG_OK:
        raise SpgError(rc, "spg_lattice_site_map: invalid arguments")
    return out, r.value, c.value


def params(**kw) -> spg_params:
    p = spg_params()
    lib.spg_params_default(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


class Context:
    """spg_create / spg_destroy.  ``stream`` is a cudaStream_t as an int
    (e.g. ``torch.cuda.current_stream().cuda_stream``) or None."""

    def __init__(self, device: int = 0, stream=None):
        h = C.c_void_p()
        rc = lib.spg_create(C.byref(h), device, C.c_void_p(stream) if stream else None)
        if rc != SPG_OK:
            raise SpgError(rc, "spg_create failed")
        self.h = h
        _LIVE["ctx"].add(self)

    def check(self, rc):
        if rc != SPG_OK:
            raise SpgError(rc, lib.spg_last_error(self.h).decode())

    def close(self):
        if self.h:
            lib.spg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Problem:
    def __init__(self, ctx: Context, h):
        self.ctx, self.h = ctx, h
        _LIVE["problem"].add(self)
        r, c = C.c_int32(), C.c_int32()
        ctx.check(lib.spg_problem_shape(h, C.byref(r), C.byref(c), None))
        self.rows, self.cols = r.value, c.value
        d = np.zeros(self.rows * self.cols, np.int32)
        ctx.check(lib.spg_problem_shape(h, None, None, _ptr(d, C.c_int32)))
        self.d = d

    def close(self):
        if self.h:
            lib.spg_problem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def spg_problem_ising(ctx: Context, inst) -> Problem:
    ei = np.ascontiguousarray(inst.ei, np.int32)
    ej = np.ascontiguousarray(inst.ej, np.int32)
    J = np.ascontiguousarray(inst.J, np.float64)
    h = np.ascontiguousarray(inst.h, np.float64)
    cos = np.ascontiguousarray(inst.cluster_of_spin, np.int32)
    cr = np.ascontiguousarray(inst.cluster_row, np.int32)
    cc = np.ascontiguousarray(inst.cluster_col, np.int32)
    out = C.c_void_p()
    ctx.check(lib.spg_problem_ising(ctx.h, inst.n_spins, len(ei), _ptr(ei, C.c_int32), _ptr(ej, C.c_int32),
                                    _ptr(J, C.c_double), _ptr(h, C.c_double), _ptr(cos, C.c_int32),
                                    inst.grid_rows, inst.grid_cols, _ptr(cr, C.c_int32), _ptr(cc, C.c_int32),
                                    inst.energy_shift, inst.node_type, C.byref(out)))
    return Problem(ctx, out)


def spg_problem_potts(ctx: Context, inst) -> Problem:
    d = np.ascontiguousarray(inst.d, np.int32)
    le = np.ascontiguousarray(inst.local_E, np.int64)
    em = np.ascontiguousarray(inst.em, np.int32)
    en = np.ascontiguousarray(inst.en, np.int32)
    pe = np.ascontiguousarray(inst.pair_E, np.int64)
    out = C.c_void_p()
    ctx.check(lib.spg_problem_potts(ctx.h, inst.grid_rows, inst.grid_cols, _ptr(d, C.c_int32), _ptr(le, C.c_int64),
                                    len(em), _ptr(em, C.c_int32), _ptr(en, C.c_int32), _ptr(pe, C.c_int64),
                                    inst.energy_shift, inst.node_type, C.byref(out)))
    return Problem(ctx, out)


class Result:
    def __init__(self, ctx, h):
        self.ctx, self.h = ctx, h
        _LIVE["result"].add(self)

    def get(self):
        """(states [n, N] uint16, energies int64 [n], log_probs [n])"""
        n, N = C.c_int32(), C.c_int32()
        self.ctx.check(lib.spg_result_get(self.h, C.byref(n), C.byref(N), None, None, None, None))
        st = np.zeros((n.value, N.value), np.uint16)
        E = np.zeros(n.value, np.int64)
        lp = np.zeros(n.value, np.float64)
        self.ctx.check(lib.spg_result_get(self.h, None, None, _ptr(st, C.c_uint16), _ptr(E, C.c_int64), None,
                                          _ptr(lp, C.c_double)))
        return st, E, lp

    def info(self) -> dict:
        inf = spg_info()
        self.ctx.check(lib.spg_result_info(self.h, C.byref(inf)))
        return {k: getattr(inf, k) for k, _ in spg_info._fields_}

    def close(self):
        if self.h:
            lib.spg_result_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def spg_solve(ctx: Context, prob: Problem, prm: spg_params) -> Result:
    out = C.c_void_p()
    ctx.check(lib.spg_solve(ctx.h, prob.h, C.byref(prm), C.byref(out)))
    return Result(ctx, out)


def spg_solve_batch(ctx: Context, probs, prms) -> list:
    """Concurrent solves of independent problems (one params per problem)."""
    n = len(probs)
    ph = (C.c_void_p * n)(*[p.h for p in probs])
    pa = (spg_params * n)(*prms)
    out = (C.c_void_p * n)()
    ctx.check(lib.spg_solve_batch(ctx.h, n, ph, pa, out))
    return [Result(ctx, C.c_void_p(out[i])) for i in range(n)]


def spg_debug_marginals(ctx: Context, prob: Problem, prm: spg_params, site: int, prefixes) -> np.ndarray:
    pre = np.ascontiguousarray(np.asarray(prefixes, dtype=np.uint16).reshape(len(prefixes), site))
    d = int(prob.d[site])
    out = np.zeros((len(prefixes), d), np.float64)
    ctx.check(lib.spg_debug_marginals(ctx.h, prob.h, C.byref(prm), site, len(prefixes),
                                      _ptr(pre, C.c_uint16) if site > 0 else None, _ptr(out, C.c_double)))
    return out


def spg_log_partition(ctx: Context, prob: Problem, prm: spg_params) -> float:
    v = C.c_double()
    ctx.check(lib.spg_log_partition(ctx.h, prob.h, C.byref(prm), C.byref(v)))
    return v.value


def spg_profile(ctx: Context, enable: bool) -> None:
    ctx.check(lib.spg_profile(ctx.h, int(bool(enable))))


def spg_profile_report(ctx: Context) -> dict:
    """{kernel: (launches, total_ms, algorithmic_flops)} since profiling was enabled."""
    import json
    buf = C.create_string_buffer(1 << 16)
    ctx.check(lib.spg_profile_report(ctx.h, buf, len(buf)))
    return {k: tuple(v) for k, v in json.loads(buf.value.decode()).items()}


def spg_truncate(ctx: Context, M, keep: int, iters: int = 6):
    """M: torch.float64 CUDA tensor (m x n, contiguous).  Returns device
    tensors (V [n, keep], US [m, keep], sigma [keep])."""
    import torch
    m, n = M.shape
    V = torch.empty((n, keep), dtype=torch.float64, device=M.device)
    US = torch.empty((m, keep), dtype=torch.float64, device=M.device)
    sig = torch.empty(keep, dtype=torch.float64, device=M.device)
    torch.cuda.synchronize(M.device)
    ctx.check(lib.spg_truncate(ctx.h, C.c_void_p(M.data_ptr()), m, n, keep, iters, C.c_void_p(V.data_ptr()),
                               C.c_void_p(US.data_ptr()), C.c_void_p(sig.data_ptr())))
    return V, US, sig


def spg_tc_product(ctx: Context, M, Bt, trans: bool):
    """Tensor-core product step of the FP32 truncation.  M: torch.float32
    CUDA tensor [m, n]; Bt: [s, n] (trans False) or [s, m] (trans True).
    Returns out [s, m] = (M Bt^T)^T or [s, n] = (M^T Bt^T)^T."""
    import torch
    m, n = M.shape
    s = Bt.shape[0]
    out = torch.empty((s, n if trans else m), dtype=torch.float32, device=M.device)
    torch.cuda.synchronize(M.device)
    ctx.check(lib.spg_tc_product(ctx.h, C.c_void_p(M.data_ptr()), m, n, C.c_void_p(Bt.data_ptr()), s,
                                 1 if trans else 0, C.c_void_p(out.data_ptr())))
    return out


def spg_truncate_static(M, keep: int, iters: int = 6, stream=None):
    """spg_truncate without any device allocation inside the library (the
    scratch is a fixed array in the library image; m, n <= 256, keep <= 32).
    Outputs are allocated here by torch, on the caller's side."""
    import torch
    m, n = M.shape
    V = torch.empty((n, keep), dtype=torch.float64, device=M.device)
    US = torch.empty((m, keep), dtype=torch.float64, device=M.device)
    sig = torch.empty(keep, dtype=torch.float64, device=M.device)
    torch.cuda.synchronize(M.device)
    rc = lib.spg_truncate_static(C.c_void_p(M.data_ptr()), m, n, keep, iters, C.c_void_p(V.data_ptr()),
                                 C.c_void_p(US.data_ptr()), C.c_void_p(sig.data_ptr()),
                                 C.c_void_p(stream) if stream else None)
    if rc != SPG_OK:
        raise SpgError(rc, "spg_truncate_static failed")
    return V, US, sig
