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
SPG_TUNE_OFF = 0
SPG_TUNE_ON = 1
SPG_TUNE_FORCE = 2

_ERRNAMES = {v: k for k, v in dict(SPG_EINVAL=-1, SPG_EINEXACT=-2, SPG_ENOMEM=-3, SPG_ECUDA=-4,
                                   SPG_ETIMEOUT=-5, SPG_ENUMERIC=-6, SPG_EUNSUPPORTED=-7).items()}


class spg_params(C.Structure):
    _fields_ = [("beta", C.c_double), ("chi", C.c_int32), ("num_sweeps", C.c_int32),
                ("beam", C.c_int32), ("precision", C.c_int32), ("cut_off_prob", C.c_double),
                ("svd_iters", C.c_int32), ("warm_start", C.c_int32), ("seed", C.c_uint64),
                ("merge", C.c_int32), ("fp64_rows", C.c_int32), ("check_fp64", C.c_int32),
                ("droplet_hamming", C.c_int32), ("droplet_energy", C.c_double), ("group_max", C.c_int32),
                ("reserved", C.c_int32)]


class spg_info(C.Structure):
    _fields_ = [("n_states", C.c_int32), ("near_ties", C.c_int32), ("degenerate_cuts", C.c_int32),
                ("error_flags", C.c_int32), ("ms_boundary", C.c_double), ("ms_search", C.c_double),
                ("candidates", C.c_double), ("boundary_lognorm", C.c_double),
                ("kernel_launches", C.c_int64), ("jacobi_sweeps_max", C.c_int32), ("fp64_rows", C.c_int32),
                ("precision_used", C.c_int32), ("droplet_overflow", C.c_int32), ("max_logmarg_err", C.c_double),
                ("group_size", C.c_int32), ("reserved", C.c_int32)]


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
        "spg_problem_update_ising": (C.c_int, [P, pD, pD]),
        "spg_problem_shape": (C.c_int, [P, pI32, pI32, pI32]),
        "spg_solve": (C.c_int, [P, P, C.POINTER(spg_params), C.POINTER(P)]),
        "spg_solve_batch": (C.c_int, [P, I32, C.POINTER(P), C.POINTER(spg_params), C.POINTER(P)]),
        "spg_solve_group": (C.c_int, [P, I32, C.POINTER(P), C.POINTER(spg_params), C.POINTER(P)]),
        "spg_result_get": (C.c_int, [P, pI32, pI32, pU16, pI64, pD, pD, pD]),
        "spg_result_info": (C.c_int, [P, C.POINTER(spg_info)]),
        "spg_result_droplets": (C.c_int, [P, pI32, pI64, pU16]),
        "spg_result_destroy": (None, [P]),
        "spg_debug_marginals": (C.c_int, [P, P, C.POINTER(spg_params), I32, I32, pU16, pD]),
        "spg_log_partition": (C.c_int, [P, P, C.POINTER(spg_params), pD]),
        "spg_truncate": (C.c_int, [P, P, I32, I32, I32, I32, P, P, P]),
        "spg_truncate_static": (C.c_int, [P, I32, I32, I32, I32, P, P, P, P]),
        "spg_tc_product": (C.c_int, [P, P, I32, I32, P, I32, I32, P]),
        "spg_warm_features": (C.c_int, [P, I32, C.POINTER(C.c_float)]),
        "spg_boundary_export": (C.c_int, [P, P, C.POINTER(spg_params), I32, I32, P, pI32]),
        "spg_mlp_create": (C.c_int, [P, I32, I32, I32, C.c_uint64, C.POINTER(P)]),
        "spg_mlp_destroy": (None, [P]),
        "spg_mlp_num_params": (C.c_int64, [P]),
        "spg_mlp_params": (C.c_int, [P, C.POINTER(C.c_float), C.POINTER(C.c_float)]),
        "spg_mlp_forward": (C.c_int, [P, P, I32, P, I32]),
        "spg_mlp_loss_grad": (C.c_int, [P, P, P, I32, pD, C.POINTER(C.c_float)]),
        "spg_mlp_train": (C.c_int, [P, P, P, C.c_int64, I32, I32, D, C.c_uint64, pD]),
        "spg_set_warm_start": (C.c_int, [P, P]),
        "spg_sweep_trace": (C.c_int, [P, P, C.POINTER(spg_params), I32, I32, I32, pD]),
        "spg_peak_probe_stream": (C.c_int, [P, I32, pD]),
        "spg_check_bounded_wait": (C.c_int, [P, C.c_int64]),
        "spg_solve_lattice8": (C.c_int, [P, P, C.POINTER(spg_params), C.POINTER(P), pI32, pI64]),
        "spg_inject_alloc_failure": (C.c_int, [I32]),
        "spg_profile": (C.c_int, [P, C.c_int]),
        "spg_profile_report": (C.c_int, [P, C.c_char_p, C.c_size_t]),
        "spg_potts_hamiltonian": (C.c_int, [I32, I32, pI32, pI32, pD, pD, pI32, I32, I32, pI32, pI32, I32, I32,
                                            C.POINTER(P)]),
        "spg_hamiltonian_size": (C.c_int, [P, pI32, pI32]),
        "spg_hamiltonian_local": (C.c_int, [P, I32, pI64, pI64]),
        "spg_hamiltonian_edge": (C.c_int, [P, I32, pI32, pI32, pI32, pI32, pI64, pI32, pI32]),
        "spg_hamiltonian_classes": (C.c_int, [P, I32, I32, pI32, pI32, pI32]),
        "spg_hamiltonian_class_weights": (C.c_int, [P, I32, D, pD]),
        "spg_hamiltonian_site_tensor": (C.c_int, [P, I32, D, pI32, pD]),
        "spg_hamiltonian_destroy": (None, [P]),
        "spg_diversity": (C.c_int, [I32, I32, pI32, pI64, C.c_int64, D, pI32, pI32]),
        "spg_autotune_set": (C.c_int, [I32, pI32]),
        "spg_autotune_clear": (C.c_int, []),
        "spg_autotune_report": (C.c_int, [pI32, C.c_char_p, C.c_size_t]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


# Handles still open at interpreter exit are released results -> problems ->
# contexts, before the CUDA runtime is torn down.
_LIVE = {"result": weakref.WeakSet(), "problem": weakref.WeakSet(), "mlp": weakref.WeakSet(),
         "ctx": weakref.WeakSet()}


@atexit.register
def _close_all():
    for kind in ("result", "problem", "mlp", "ctx"):
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


def _stream_handle(stream):
    """cudaStream_t of a torch.cuda.Stream, a raw handle (int) or None."""
    if stream is None:
        return None
    handle = getattr(stream, "cuda_stream", stream)
    return C.c_void_p(int(handle)) if handle else None


def _device_tensor(t, dtype, name, ndim=2, device=None):
    """Reject, before any launch, a tensor the C ABI would misread: the
    library reads plain row-major device arrays of one dtype."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name}: expected a torch tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name}: expected dtype {dtype}, got {t.dtype}")
    if not t.is_cuda:
        raise ValueError(f"{name}: expected a CUDA tensor")
    if t.dim() != ndim or not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous {ndim}-D tensor")
    if device is not None and t.device.index != device:
        raise ValueError(f"{name}: tensor on cuda:{t.device.index}, the context runs on cuda:{device}")
    return t


class Context:
    """spg_create / spg_destroy.  ``stream``: a torch.cuda.Stream, a
    cudaStream_t as an int (e.g. ``torch.cuda.current_stream().cuda_stream``)
    or None (the library creates its own)."""

    def __init__(self, device: int = 0, stream=None):
        h = C.c_void_p()
        rc = lib.spg_create(C.byref(h), device, _stream_handle(stream))
        if rc != SPG_OK:
            raise SpgError(rc, "spg_create failed")
        self.h = h
        self.device = device
        _LIVE["ctx"].add(self)

    def check(self, rc):
        if rc != SPG_OK:
            raise SpgError(rc, lib.spg_last_error(self.h).decode())

    def close(self):
        if self.h:
            # handles made through this context go first: the garbage
            # collector may finalise a cycle (a failed test's frame, say) in
            # any order, and a handle released after its context would read
            # freed memory
            for kind in ("result", "problem", "mlp"):
                for obj in list(_LIVE[kind]):
                    if getattr(obj, "ctx", None) is self:
                        try:
                            obj.close()
                        except Exception:
                            pass
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


class Hamiltonian:
    """The clustered Hamiltonian of an Ising instance, built by the library
    on the host (spg_potts_hamiltonian; no device).  E_loc: int64 [d_s] per
    site; edges: {(m, n): (R int64 [Dm, Dn], Pm int32 [d_m], Pn int32
    [d_n])}; classes(s, which) and class_weights(s, beta) as in
    include/spg.h."""

    L, U, R, D, G = 0, 1, 2, 3, 4

    def __init__(self, h):
        self.h = h
        ns, ne = C.c_int32(), C.c_int32()
        lib.spg_hamiltonian_size(h, C.byref(ns), C.byref(ne))
        self.E_loc = []
        for s in range(ns.value):
            n = C.c_int64()
            lib.spg_hamiltonian_local(h, s, C.byref(n), None)
            E = np.empty(n.value, np.int64)
            lib.spg_hamiltonian_local(h, s, None, _ptr(E, C.c_int64))
            self.E_loc.append(E)
        self.edges = {}
        for k in range(ne.value):
            m, n, Dm, Dn = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
            lib.spg_hamiltonian_edge(h, k, C.byref(m), C.byref(n), C.byref(Dm), C.byref(Dn), None, None, None)
            R = np.empty((Dm.value, Dn.value), np.int64)
            Pm = np.empty(len(self.E_loc[m.value]), np.int32)
            Pn = np.empty(len(self.E_loc[n.value]), np.int32)
            lib.spg_hamiltonian_edge(h, k, None, None, None, None, _ptr(R, C.c_int64), _ptr(Pm, C.c_int32),
                                     _ptr(Pn, C.c_int32))
            self.edges[(m.value, n.value)] = (R, Pm, Pn)

    def classes(self, site: int, which: int):
        """(P int32 [d_site], reps int32 [n_classes]) of joint projection
        `which` (Hamiltonian.L, U, R, D, G)."""
        nc = C.c_int32()
        rc = lib.spg_hamiltonian_classes(self.h, site, which, C.byref(nc), None, None)
        if rc != 0:
            raise SpgError(rc, "spg_hamiltonian_classes")
        P = np.empty(len(self.E_loc[site]), np.int32)
        reps = np.empty(nc.value, np.int32)
        lib.spg_hamiltonian_classes(self.h, site, which, None, _ptr(P, C.c_int32), _ptr(reps, C.c_int32))
        return P, reps

    def class_weights(self, site: int, beta: float):
        """C [NL, NU, NR, ND] (float64): the summed state weights per class
        tuple."""
        dims = [len(self.classes(site, w)[1]) for w in (self.L, self.U, self.R, self.D)]
        Cw = np.empty(dims, np.float64)
        rc = lib.spg_hamiltonian_class_weights(self.h, site, float(beta), _ptr(Cw, C.c_double))
        if rc != 0:
            raise SpgError(rc, "spg_hamiltonian_class_weights")
        return Cw

    def site_tensor(self, site: int, beta: float):
        """W [DL, DR, DU, ND] (float64): the site's PEPS tensor."""
        dims = np.zeros(4, np.int32)
        rc = lib.spg_hamiltonian_site_tensor(self.h, site, float(beta), _ptr(dims, C.c_int32), None)
        if rc != 0:
            raise SpgError(rc, "spg_hamiltonian_site_tensor")
        W = np.empty(tuple(int(v) for v in dims), np.float64)
        lib.spg_hamiltonian_site_tensor(self.h, site, float(beta), _ptr(dims, C.c_int32), _ptr(W, C.c_double))
        return W

    def close(self):
        if self.h:
            lib.spg_hamiltonian_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def spg_potts_hamiltonian(inst) -> Hamiltonian:
    """spg_potts_hamiltonian of an Ising instance (host only)."""
    ei = np.ascontiguousarray(inst.ei, np.int32)
    ej = np.ascontiguousarray(inst.ej, np.int32)
    J = np.ascontiguousarray(inst.J, np.float64)
    h = np.ascontiguousarray(inst.h, np.float64)
    cos = np.ascontiguousarray(inst.cluster_of_spin, np.int32)
    cr = np.ascontiguousarray(inst.cluster_row, np.int32)
    cc = np.ascontiguousarray(inst.cluster_col, np.int32)
    H = C.c_void_p()
    rc = lib.spg_potts_hamiltonian(inst.n_spins, len(ei), _ptr(ei, C.c_int32), _ptr(ej, C.c_int32),
                                   _ptr(J, C.c_double), _ptr(h, C.c_double), _ptr(cos, C.c_int32), inst.grid_rows,
                                   inst.grid_cols, _ptr(cr, C.c_int32), _ptr(cc, C.c_int32), inst.energy_shift,
                                   inst.node_type, C.byref(H))
    if rc != 0:
        raise SpgError(rc, "spg_potts_hamiltonian refused the instance")
    return Hamiltonian(H)


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
        self.ctx.check(lib.spg_result_get(self.h, C.byref(n), C.byref(N), None, None, None, None, None))
        st = np.zeros((n.value, N.value), np.uint16)
        E = np.zeros(n.value, np.int64)
        lp = np.zeros(n.value, np.float64)
        self.ctx.check(lib.spg_result_get(self.h, None, None, _ptr(st, C.c_uint16), _ptr(E, C.c_int64), None,
                                          _ptr(lp, C.c_double), None))
        return st, E, lp

    def droplets(self):
        """(energies int64 [n], states [n, N]) of the best state's droplets."""
        n = C.c_int32()
        self.ctx.check(lib.spg_result_droplets(self.h, C.byref(n), None, None))
        _, N = self.shape()
        E = np.zeros(n.value, np.int64)
        st = np.zeros((n.value, N), np.uint16)
        self.ctx.check(lib.spg_result_droplets(self.h, None, _ptr(E, C.c_int64), _ptr(st, C.c_uint16)))
        return E, st

    def shape(self):
        n, N = C.c_int32(), C.c_int32()
        self.ctx.check(lib.spg_result_get(self.h, C.byref(n), C.byref(N), None, None, None, None, None))
        return n.value, N.value

    def max_logmarg_err(self) -> float:
        """Log-marginal error of the result against plain FP64 (params
        check_fp64; NaN when unchecked, 0 in the FP64 mode)."""
        v = C.c_double()
        self.ctx.check(lib.spg_result_get(self.h, None, None, None, None, None, None, C.byref(v)))
        return v.value

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


def spg_solve_group(ctx: Context, probs, prm: spg_params) -> list:
    """Problems of one structure solved in lockstep (one launch sequence)."""
    n = len(probs)
    ph = (C.c_void_p * n)(*[p.h for p in probs])
    out = (C.c_void_p * n)()
    ctx.check(lib.spg_solve_group(ctx.h, n, ph, C.byref(prm), out))
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


def spg_diversity(solutions, energies, e_best: int, a_r: float = 0.01):
    """(count, indices in counting order) of spg_diversity: solutions [n, N]
    (spins or Potts states), energies [n] int64."""
    X = np.ascontiguousarray(np.asarray(solutions).reshape(len(energies), -1), np.int32)
    E = np.ascontiguousarray(energies, np.int64)
    n, N = X.shape
    cnt = C.c_int32()
    chosen = np.empty(max(n, 1), np.int32)
    rc = lib.spg_diversity(n, N, _ptr(X, C.c_int32), _ptr(E, C.c_int64), int(e_best), float(a_r), C.byref(cnt),
                           _ptr(chosen, C.c_int32))
    if rc != 0:
        raise SpgError(rc, "spg_diversity: bad arguments")
    return cnt.value, [int(v) for v in chosen[:cnt.value]]


def spg_autotune_set(mode: int) -> int:
    """Sets the process-wide autotuner mode (SPG_TUNE_OFF, SPG_TUNE_ON or
    SPG_TUNE_FORCE + k); returns the previous mode."""
    prev = C.c_int32(0)
    rc = lib.spg_autotune_set(int(mode), C.byref(prev))
    if rc != 0:
        raise SpgError(rc, f"autotuner mode {mode} out of range")
    return prev.value


def spg_autotune_clear() -> None:
    """Forgets every timed shape."""
    rc = lib.spg_autotune_clear()
    if rc != 0:
        raise SpgError(rc, "a shape is being timed")


def spg_autotune_report() -> list:
    """[(kernel, device, group, shape tuple, chosen variant, [best us per
    variant, -1: could not run])] of every timed shape."""
    n = C.c_int32(0)
    buf = C.create_string_buffer(1 << 20)
    lib.spg_autotune_report(C.byref(n), buf, len(buf))
    out = []
    for line in buf.value.decode().splitlines():
        head, tail = line.split(" -> ")
        f = head.split()
        choice, times = tail.split(" us")
        out.append((f[0], int(f[2]), int(f[4]), tuple(int(x) for x in f[6:]), int(choice),
                    [float(t) for t in times.split()]))
    return out


def spg_truncate(ctx: Context, M, keep: int, iters: int = 6):
    """M: torch.float64 CUDA tensor (m x n, contiguous).  Returns device
    tensors (V [n, keep], US [m, keep], sigma [keep])."""
    import torch
    _device_tensor(M, torch.float64, "M", device=ctx.device)
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
    _device_tensor(M, torch.float32, "M", device=ctx.device)
    _device_tensor(Bt, torch.float32, "Bt", device=ctx.device)
    m, n = M.shape
    s = Bt.shape[0]
    if Bt.shape[1] != (m if trans else n):
        raise ValueError("Bt: second dimension must be m (trans) or n")
    out = torch.empty((s, n if trans else m), dtype=torch.float32, device=M.device)
    torch.cuda.synchronize(M.device)
    ctx.check(lib.spg_tc_product(ctx.h, C.c_void_p(M.data_ptr()), m, n, C.c_void_p(Bt.data_ptr()), s,
                                 1 if trans else 0, C.c_void_p(out.data_ptr())))
    return out


def spg_truncate_static(M, keep: int, iters: int = 6, stream=None):
    """spg_truncate without any device allocation inside the library (the
    scratch is a fixed array in the library image; m, n <= 256, keep <= 32).
    Outputs are allocated here by torch, on the caller's side.  M: contiguous
    torch.float64 CUDA tensor; the call runs on M's device, on ``stream`` (a
    torch.cuda.Stream or a raw handle; default: torch's current stream of
    that device, so it is ordered after the caller's work on it)."""
    import torch
    _device_tensor(M, torch.float64, "M")
    m, n = M.shape
    with torch.cuda.device(M.device):
        if stream is None:
            stream = torch.cuda.current_stream(M.device)
        V = torch.empty((n, keep), dtype=torch.float64, device=M.device)
        US = torch.empty((m, keep), dtype=torch.float64, device=M.device)
        sig = torch.empty(keep, dtype=torch.float64, device=M.device)
        rc = lib.spg_truncate_static(C.c_void_p(M.data_ptr()), m, n, keep, iters, C.c_void_p(V.data_ptr()),
                                     C.c_void_p(US.data_ptr()), C.c_void_p(sig.data_ptr()),
                                     _stream_handle(stream))
    if rc != SPG_OK:
        raise SpgError(rc, "spg_truncate_static failed")
    return V, US, sig


# ---------------------------------------------------------------- warm start
SPG_WS_FEATURES = 800
SPG_WS_PER_CLUSTER = 52


def spg_warm_features(prob: Problem, row: int) -> np.ndarray:
    """Network inputs of the sites of boundary row `row`: [cols, 800] float32."""
    out = np.zeros((prob.cols, SPG_WS_FEATURES), np.float32)
    rc = lib.spg_warm_features(prob.h, row, _ptr(out, C.c_float))
    if rc != SPG_OK:
        raise SpgError(rc, "spg_warm_features failed")
    return out


def spg_boundary_export(ctx: Context, prob: Problem, prm: spg_params, row: int, fix_signs: bool = True):
    """(sites, dims): the boundary MPS B_row as a device tensor [cols, 16,
    chi, chi] (float64 in SPG_FP64, float32 in SPG_MIXED) and the sites'
    dims [cols, 3] = (p, chi_l, chi_r); row 0: every row 1 .. rows-1,
    [rows-1, cols, 16, chi, chi] and [rows-1, cols, 3]."""
    import torch
    chi = prm.chi
    dtype = torch.float64 if prm.precision == SPG_FP64 else torch.float32
    lead = (prob.rows - 1, prob.cols) if row == 0 else (prob.cols,)
    with torch.cuda.device(ctx.device):
        out = torch.empty(lead + (16, chi, chi), dtype=dtype, device=f"cuda:{ctx.device}")
        torch.cuda.synchronize()
        dims = np.zeros(lead + (3,), np.int32)
        ctx.check(lib.spg_boundary_export(ctx.h, prob.h, C.byref(prm), row, int(bool(fix_signs)),
                                          C.c_void_p(out.data_ptr()), _ptr(dims, C.c_int32)))
    return out, dims


class Mlp:
    """spg_mlp_*: the warm-start network (parameters and Adam state on the
    context's device).  Inputs and targets are contiguous float32 CUDA
    tensors."""

    def __init__(self, ctx: Context, n_in: int, n_hidden: int, n_out: int, seed: int = 0):
        h = C.c_void_p()
        ctx.check(lib.spg_mlp_create(ctx.h, n_in, n_hidden, n_out, seed, C.byref(h)))
        self.ctx, self.h = ctx, h
        self.n_in, self.n_hidden, self.n_out = n_in, n_hidden, n_out
        _LIVE["mlp"].add(self)

    def num_params(self) -> int:
        return int(lib.spg_mlp_num_params(self.h))

    def params(self) -> np.ndarray:
        out = np.zeros(self.num_params(), np.float32)
        self.ctx.check(lib.spg_mlp_params(self.h, _ptr(out, C.c_float), None))
        return out

    def set_params(self, flat) -> None:
        flat = np.ascontiguousarray(flat, np.float32)
        if flat.size != self.num_params():
            raise ValueError("parameter count mismatch")
        self.ctx.check(lib.spg_mlp_params(self.h, None, _ptr(flat, C.c_float)))

    def forward(self, X, bf16: bool = False):
        import torch
        _device_tensor(X, torch.float32, "X", device=self.ctx.device)
        if X.shape[1] != self.n_in:
            raise ValueError("X: wrong number of inputs")
        Y = torch.empty((X.shape[0], self.n_out), dtype=torch.float32, device=X.device)
        torch.cuda.synchronize(X.device)
        self.ctx.check(lib.spg_mlp_forward(self.h, C.c_void_p(X.data_ptr()), X.shape[0], C.c_void_p(Y.data_ptr()),
                                           int(bool(bf16))))
        return Y

    def loss_grad(self, X, T):
        """(loss, flat gradient) over all rows of X, T."""
        import torch
        _device_tensor(X, torch.float32, "X", device=self.ctx.device)
        _device_tensor(T, torch.float32, "T", device=self.ctx.device)
        g = np.zeros(self.num_params(), np.float32)
        loss = C.c_double()
        torch.cuda.synchronize(X.device)
        self.ctx.check(lib.spg_mlp_loss_grad(self.h, C.c_void_p(X.data_ptr()), C.c_void_p(T.data_ptr()), X.shape[0],
                                             C.byref(loss), _ptr(g, C.c_float)))
        return loss.value, g

    def train(self, X, T, batch: int, steps: int, lr: float, seed: int = 0) -> float:
        import torch
        _device_tensor(X, torch.float32, "X", device=self.ctx.device)
        _device_tensor(T, torch.float32, "T", device=self.ctx.device)
        loss = C.c_double()
        torch.cuda.synchronize(X.device)
        self.ctx.check(lib.spg_mlp_train(self.h, C.c_void_p(X.data_ptr()), C.c_void_p(T.data_ptr()), X.shape[0],
                                         batch, steps, lr, seed, C.byref(loss)))
        return loss.value

    def split(self, flat) -> dict:
        """The flat layout as {W1, b1, W2, b2, W3, b3} views."""
        I, H, O = self.n_in, self.n_hidden, self.n_out
        out, o = {}, 0
        for k, shape in (("W1", (H, I)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (O, H)), ("b3", (O,))):
            n = int(np.prod(shape))
            out[k] = flat[o:o + n].reshape(shape)
            o += n
        return out

    def close(self):
        if self.h:
            lib.spg_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def spg_set_warm_start(ctx: Context, mlp) -> None:
    ctx.check(lib.spg_set_warm_start(ctx.h, mlp.h if mlp is not None else None))
    ctx._warm = mlp  # keep it alive while attached


def spg_sweep_trace(ctx: Context, prob: Problem, prm: spg_params, row: int, init: int, n_sweeps: int) -> np.ndarray:
    """log <phi_k | W psi> after each of n_sweeps sweeps of row `row`
    started from the zipper (init 0) or the attached network (init 1);
    init 2: both, [2, n_sweeps] (zipper first)."""
    out = np.zeros((2, n_sweeps) if init == 2 else n_sweeps, np.float64)
    ctx.check(lib.spg_sweep_trace(ctx.h, prob.h, C.byref(prm), row, init, n_sweeps, _ptr(out, C.c_double)))
    return out


def spg_peak_probe(kind: str, stream=None) -> float:
    """Measured FMA throughput of the current device in TFLOP/s ("fp32" or
    "fp64")."""
    v = C.c_double()
    rc = lib.spg_peak_probe_stream(_stream_handle(stream), {"fp32": 0, "fp64": 1}[kind], C.byref(v))
    if rc != SPG_OK:
        raise SpgError(rc, "spg_peak_probe failed")
    return v.value


def spg_check_bounded_wait(ctx: Context, polls: int) -> int:
    """Return code of the bounded-wait failure path (SPG_ETIMEOUT expected)."""
    return int(lib.spg_check_bounded_wait(ctx.h, polls))


def spg_inject_alloc_failure(after: int) -> None:
    """Test hook: the (after+1)-th device allocation from now fails (-1: off)."""
    lib.spg_inject_alloc_failure(after)


def spg_solve_lattice8(ctx: Context, prob: Problem, prm: spg_params):
    """(result, best_k, best energy of every lattice): the 8 lattice
    transformations solved as one batch, best of 8, states on the original
    sites."""
    out = C.c_void_p()
    k = C.c_int32()
    per = np.zeros(8, np.int64)
    ctx.check(lib.spg_solve_lattice8(ctx.h, prob.h, C.byref(prm), C.byref(out), C.byref(k), _ptr(per, C.c_int64)))
    return Result(ctx, out), k.value, per


def spg_problem_update_ising(prob: Problem, J, h=None) -> None:
    """New couplings (and fields) of the same structure, written in place."""
    J = np.ascontiguousarray(J, np.float64)
    h = None if h is None else np.ascontiguousarray(h, np.float64)
    prob.ctx.check(lib.spg_problem_update_ising(prob.h, _ptr(J, C.c_double), _ptr(h, C.c_double)))
