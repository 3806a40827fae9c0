"""GB300-native SPAI preconditioning, cheap parameter update and block GMRES.

Thin ctypes binding over ``libspai_gb300.so``, whose C ABI is declared in
``include/spai_gb300.h``.  Every function here has the name of the C entry point it
wraps and only marshals arguments: device memory comes from the caller (typically torch
tensors, passed by ``data_ptr()``), every step of the computation runs in the library's
CUDA kernels, and there is no CPU fallback -- if the library has not been built, the
first call raises.

Method: arXiv 1809.06574 -- SPAI (Sec. 2.2), its update (Sec. 2.3 Table 1, Sec. 2.4),
and right-preconditioned block Krylov solves (Sec. 2.1, Sec. 2.2 footnote).
"""

from __future__ import annotations

import ctypes as C
import os

__all__ = [
    "SpaiError", "spai_csr", "spai_solve_opts", "spai_solve_info", "csr", "lib",
    "spai_ctx_create", "spai_ctx_destroy", "spai_last_error", "spai_ctx_sync",
    "spai_ctx_mem_in_use", "spai_ctx_set_wait_limit", "spai_ctx_inject_stall", "spai_launch_count", "spai_ctx_profile", "spai_ctx_profile_count", "spai_measure_fp64_rate",
    "spai_measure_fp32_rate",
    "spai_ctx_profile_entry", "spai_affine_create", "spai_affine_pattern",
    "spai_assemble", "spai_affine_export", "spai_affine_destroy", "spai_build", "spai_update", "spai_pc_info",
    "spai_pc_export", "spai_pc_destroy", "spai_build_batch", "block_solve_batch", "spai_spmm", "spai_pc_apply", "spai_spmm_fp32", "spai_pc_apply_fp32", "block_solve", "block_solve_gcro",
    "spai_recycle_create", "spai_recycle_info", "spai_recycle_export", "spai_recycle_clear", "spai_recycle_destroy",
    "spai_shifted_coefficients", "spai_assemble_shifted", "spai_server_add_shifted_system", "PATTERN_A", "PATTERN_A2", "UPDATE_FIRST", "UPDATE_CHAINED", "UPDATE_DIAGONAL", "PREC_FP32", "PREC_BF16",
    "LIB_PATH", "spai_ctx_trim", "spai_solve_workspace_size", "spai_pc_mem_size",
    "spai_server_opts", "spai_request", "spai_result", "spai_server_stats", "spai_server_create",
    "spai_server_add_system", "spai_server_submit", "spai_server_wait", "spai_server_clock",
    "spai_server_stats_get", "spai_server_last_error", "spai_server_destroy",
    "ROUTE_BUILD", "ROUTE_UPDATE", "ROUTE_REUSE", "SOLVE_FP64", "SOLVE_MIXED",
]

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libspai_gb300.so")

SPAI_OK, SPAI_EINVAL, SPAI_ENOMEM, SPAI_ECUDA, SPAI_ESINGULAR, SPAI_ENOTCONV, SPAI_ETIMEOUT = range(7)
STATUS_NAMES = {0: "SPAI_OK", 1: "SPAI_EINVAL", 2: "SPAI_ENOMEM", 3: "SPAI_ECUDA",
                4: "SPAI_ESINGULAR", 5: "SPAI_ENOTCONV", 6: "SPAI_ETIMEOUT"}
PATTERN_A, PATTERN_A2 = 0, 1
UPDATE_FIRST, UPDATE_CHAINED = 1, 2
UPDATE_DIAGONAL = 4  # OR into an approach: diagonal Q_l
PREC_FP32 = 0x100  # OR into a pattern kind or an update approach: FP32 least squares and factor
PREC_BF16 = 0x200  # the same least squares, factor stored in BF16
LS_NORMAL = 0x400  # OR into a pattern kind or an update approach: column problems by their normal equations


class SpaiError(RuntimeError):
    def __init__(self, status, message, result=None):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
        self.message = message
        self.result = result


class spai_csr(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int32), ("rowptr", C.c_void_p),
                ("colind", C.c_void_p), ("val", C.c_void_p)]


class spai_solve_opts(C.Structure):
    _fields_ = [("restart", C.c_int32), ("max_cycles", C.c_int32), ("tol", C.c_double),
                ("orth", C.c_int32), ("precision", C.c_int32)]


ORTH_AUTO, ORTH_FP64, ORTH_TENSOR = 0, 1, 2
SOLVE_FP64, SOLVE_MIXED = 0, 1  # operator products in FP64, or in FP32 with FP64 refinement


class spai_solve_info(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("cycles", C.c_int32), ("converged", C.c_int32),
                ("worst_column", C.c_int32), ("max_rel_residual", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class spai_server_opts(C.Structure):
    _fields_ = [("slots", C.c_int32), ("pattern_kind", C.c_int32), ("reuse", C.c_int32),
                ("restart", C.c_int32), ("max_cycles", C.c_int32), ("orth", C.c_int32),
                ("radius", C.c_double), ("tol", C.c_double), ("mem_budget", C.c_size_t),
                ("precision", C.c_int32), ("reserved", C.c_int32)]


class spai_request(C.Structure):
    _fields_ = [("system", C.c_int32), ("nrhs", C.c_int32), ("p", C.c_double), ("s", C.c_double),
                ("coef", C.c_void_p), ("B", C.c_void_p), ("X", C.c_void_p), ("t_arrival", C.c_double)]


class spai_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("route", C.c_int32), ("slot", C.c_int32),
                ("iterations", C.c_int32), ("base_p", C.c_double), ("max_rel_residual", C.c_double),
                ("t_arrival", C.c_double), ("t_start", C.c_double), ("t_done", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class spai_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("builds", C.c_int64), ("updates", C.c_int64), ("reuses", C.c_int64),
                ("evictions", C.c_int64), ("waits_for_memory", C.c_int64),
                ("mem_in_use", C.c_size_t), ("mem_peak", C.c_size_t),
                ("cached_builds", C.c_int32), ("reserved", C.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


ROUTE_BUILD, ROUTE_UPDATE, ROUTE_REUSE = 0, 1, 2


class spai_adaptive_opts(C.Structure):
    _fields_ = [("eps", C.c_double), ("max_steps", C.c_int32), ("max_new", C.c_int32),
                ("max_rows", C.c_int32), ("reserved", C.c_int32)]

_lib = None


def lib():
    """Load the library (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, dbl, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_size_t
    P = C.POINTER
    sig = {
        "spai_ctx_create": (i32, [P(vp), vp, sz]),
        "spai_ctx_destroy": (i32, [vp]),
        "spai_last_error": (C.c_char_p, [vp]),
        "spai_ctx_sync": (i32, [vp]),
        "spai_ctx_mem_in_use": (sz, [vp]),
        "spai_ctx_set_wait_limit": (i32, [vp, dbl]),
        "spai_ctx_inject_stall": (i32, [vp, i32]),
        "spai_launch_count": (i64, []),
        "spai_measure_fp64_rate": (i32, [vp, P(dbl)]),
        "spai_measure_fp32_rate": (i32, [vp, P(dbl)]),
        "spai_ctx_profile": (i32, [vp, i32]),
        "spai_ctx_profile_count": (i32, [vp]),
        "spai_ctx_profile_entry": (i32, [vp, i32, P(C.c_char_p), P(i64), P(dbl), P(dbl), P(dbl)]),
        "spai_affine_create": (i32, [vp, i32, P(spai_csr), P(vp)]),
        "spai_affine_pattern": (i32, [vp, P(i32), P(i32), P(vp), P(vp)]),
        "spai_assemble": (i32, [vp, vp, P(dbl), vp]),
        "spai_shifted_coefficients": (i32, [i32, P(dbl), dbl, dbl, dbl, P(dbl)]),
        "spai_assemble_shifted": (i32, [vp, vp, dbl, i32, P(dbl), dbl, dbl, vp]),
        "spai_affine_export": (i32, [vp, vp, vp, vp]),
        "spai_affine_destroy": (i32, [vp]),
        "spai_build": (i32, [vp, P(spai_csr), i32, P(vp)]),
        "spai_update": (i32, [vp, vp, P(spai_csr), i32, P(vp)]),
        "spai_pc_info": (i32, [vp, P(i32), P(i32), P(i64), P(i32)]),
        "spai_pc_export": (i32, [vp, vp, vp, vp, vp, vp, vp, vp]),
        "spai_pc_destroy": (i32, [vp]),
        "spai_spmm": (i32, [vp, P(spai_csr), i32, vp, i64, vp, i64]),
        "spai_pc_apply": (i32, [vp, vp, i32, vp, i64, vp, i64]),
        "spai_pc_apply_noalloc": (i32, [vp, vp, i32, vp, i64, vp, i64]),
        "spai_spmm_fp32": (i32, [vp, P(spai_csr), i32, vp, i64, vp, i64]),
        "spai_pc_apply_fp32": (i32, [vp, vp, i32, vp, i64, vp, i64]),
        "spai_block_gram": (i32, [vp, i32, i32, i32, vp, vp, vp, i32]),
        "spai_block_update": (i32, [vp, i32, i32, i32, vp, vp, vp, dbl, i32]),
        "block_solve": (i32, [vp, P(spai_csr), vp, i32, vp, i64, vp, i64, P(spai_solve_opts),
                              P(spai_solve_info), P(dbl)]),
        "spai_ctx_trim": (i32, [vp]),
        "spai_build_batch": (i32, [vp, i32, P(spai_csr), P(i32), P(vp)]),
        "block_solve_batch": (i32, [vp, i32, P(spai_csr), P(vp), i32, P(vp), P(vp), P(spai_solve_opts),
                                    P(spai_solve_info)]),
        "spai_solve_workspace_size": (sz, [i32, i32, i32]),
        "spai_pc_mem_size": (sz, [vp, i32]),
        "spai_server_create": (i32, [P(spai_server_opts), P(vp)]),
        "spai_server_add_system": (i32, [vp, i32, P(spai_csr), P(i32)]),
        "spai_server_add_shifted_system": (i32, [vp, P(spai_csr), dbl, dbl, P(i32)]),
        "spai_server_submit": (i32, [vp, P(spai_request), P(i64)]),
        "spai_server_wait": (i32, [vp, i64, P(spai_result)]),
        "spai_server_clock": (dbl, [vp]),
        "spai_server_stats_get": (i32, [vp, P(spai_server_stats)]),
        "spai_server_last_error": (C.c_char_p, [vp]),
        "spai_server_destroy": (i32, [vp]),
        "spai_build_adaptive": (i32, [vp, P(spai_csr), P(spai_adaptive_opts), i32, P(vp)]),
        "spai_column_variants": (i32, [i32, i32, i32, P(i32), i32]),
        "spai_recycle_create": (i32, [vp, i32, i32, i32, P(vp)]),
        "spai_recycle_info": (i32, [vp, P(i32)]),
        "spai_recycle_export": (i32, [vp, vp, vp, i64]),
        "spai_recycle_clear": (i32, [vp]),
        "spai_recycle_destroy": (i32, [vp]),
        "block_solve_gcro": (i32, [vp, P(spai_csr), vp, i32, vp, i64, vp, i64, P(spai_solve_opts), vp,
                                   P(spai_solve_info), P(dbl)]),
        "spai_column_variant_get": (i32, [i32, i32, i32]),
        "spai_column_variant_set": (i32, [i32, i32, i32, i32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)!r}")


def csr(n, rowptr, colind, val, nnz=None):
    """spai_csr from arrays (torch tensors or numpy arrays) or raw integer pointers.

    The returned struct keeps references to the arrays so they outlive the call.
    """
    if nnz is None:
        nnz = int(colind.shape[0]) if hasattr(colind, "shape") else 0
    s = spai_csr(int(n), int(nnz), _ptr(rowptr), _ptr(colind), _ptr(val))
    s._keep = (rowptr, colind, val)
    return s


def _check(ctx, st, allow=()):
    if st != SPAI_OK and st not in allow:
        raise SpaiError(st, spai_last_error(ctx) if ctx else "")
    return st


# ------------------------------------------------------------------ context
def spai_ctx_create(stream=None, mem_budget=0):
    out = C.c_void_p()
    st = lib().spai_ctx_create(C.byref(out), _ptr(stream) if stream is not None else None,
                               int(mem_budget))
    if st != SPAI_OK:
        raise SpaiError(st, "spai_ctx_create failed")
    return out


def spai_ctx_destroy(ctx):
    return _check(None, lib().spai_ctx_destroy(ctx))


def spai_last_error(ctx):
    r = lib().spai_last_error(ctx)
    return r.decode() if r else ""


def spai_ctx_sync(ctx):
    return _check(ctx, lib().spai_ctx_sync(ctx))


def spai_ctx_set_wait_limit(ctx, seconds):
    return _check(ctx, lib().spai_ctx_set_wait_limit(ctx, float(seconds)))


def spai_ctx_inject_stall(ctx, count=1):
    return _check(ctx, lib().spai_ctx_inject_stall(ctx, int(count)))


def spai_ctx_mem_in_use(ctx):
    return int(lib().spai_ctx_mem_in_use(ctx))


def spai_launch_count():
    return int(lib().spai_launch_count())


def spai_measure_fp64_rate(ctx):
    r = C.c_double()
    _check(ctx, lib().spai_measure_fp64_rate(ctx, C.byref(r)))
    return r.value


def spai_measure_fp32_rate(ctx):
    r = C.c_double()
    _check(ctx, lib().spai_measure_fp32_rate(ctx, C.byref(r)))
    return r.value


def spai_ctx_profile(ctx, enable):
    return _check(ctx, lib().spai_ctx_profile(ctx, int(bool(enable))))


def spai_ctx_profile_count(ctx):
    return int(lib().spai_ctx_profile_count(ctx))


def spai_ctx_profile_entry(ctx, i):
    name = C.c_char_p()
    launches = C.c_int64()
    ms, fl, by = C.c_double(), C.c_double(), C.c_double()
    _check(ctx, lib().spai_ctx_profile_entry(ctx, int(i), C.byref(name), C.byref(launches),
                                             C.byref(ms), C.byref(fl), C.byref(by)))
    return {"name": name.value.decode(), "launches": launches.value, "ms": ms.value,
            "flops": fl.value, "bytes": by.value}


# ------------------------------------------------------------------ affine assembly
def _params(p):
    ps = [float(x) for x in p] if hasattr(p, "__len__") else [float(p)]
    return len(ps), (C.c_double * max(len(ps), 1))(*ps)


def spai_shifted_coefficients(p, s, alpha, beta):
    """Coefficients of (M, K_0, K_1, ...) in A(p, s) (computed by the library).  p: one
    parameter or a sequence.  Returns a list of len(p) + 2 floats."""
    k, pa = _params(p)
    out = (C.c_double * (k + 2))()
    st = lib().spai_shifted_coefficients(k, pa, float(s), float(alpha), float(beta), out)
    if st != SPAI_OK:
        raise SpaiError(st, "spai_shifted_coefficients: bad parameters")
    return list(out)


def spai_assemble_shifted(ctx, aff, s, p, alpha, beta, val_out):
    """val_out = A(p, s) of the handle's terms (M, K_0, K_1, ...); p one value or a sequence."""
    k, pa = _params(p)
    return _check(ctx, lib().spai_assemble_shifted(ctx, aff, float(s), k, pa, float(alpha), float(beta),
                                                   _ptr(val_out)))


def spai_affine_create(ctx, terms):
    """terms: list of spai_csr (host or device arrays)."""
    arr = (spai_csr * len(terms))(*terms)
    out = C.c_void_p()
    _check(ctx, lib().spai_affine_create(ctx, len(terms), arr, C.byref(out)))
    return out


def spai_affine_pattern(aff):
    n, nnz = C.c_int32(), C.c_int32()
    rp, ci = C.c_void_p(), C.c_void_p()
    _check(None, lib().spai_affine_pattern(aff, C.byref(n), C.byref(nnz), C.byref(rp), C.byref(ci)))
    return n.value, nnz.value, rp.value, ci.value


def spai_assemble(ctx, aff, coef, val_out):
    cf = (C.c_double * len(coef))(*[float(c) for c in coef])
    return _check(ctx, lib().spai_assemble(ctx, aff, cf, _ptr(val_out)))


def spai_affine_export(ctx, aff, rowptr, colind):
    """Copy the union pattern into rowptr / colind (host numpy or device tensors)."""
    return _check(ctx, lib().spai_affine_export(ctx, aff, _ptr(rowptr), _ptr(colind)))


def spai_affine_destroy(aff):
    return _check(None, lib().spai_affine_destroy(aff))


# ------------------------------------------------------------------ preconditioner
def spai_build(ctx, A, pattern_kind=PATTERN_A, allow_singular=False):
    """Returns (pc, status).  SPAI_ESINGULAR raises unless allow_singular."""
    out = C.c_void_p()
    st = lib().spai_build(ctx, C.byref(A), int(pattern_kind), C.byref(out))
    if st == SPAI_ESINGULAR and not allow_singular:
        msg = spai_last_error(ctx)
        if out:
            lib().spai_pc_destroy(out)
        raise SpaiError(st, msg)
    _check(ctx, st, allow=(SPAI_ESINGULAR,))
    return out, st


def spai_build_batch(ctx, As, pattern_kinds, allow_singular=False):
    """SPAI of many systems at once: As list of spai_csr (device), pattern_kinds list of ints.
    Returns (list of handles, status)."""
    m = len(As)
    arr = (spai_csr * m)(*As)
    kinds = (C.c_int32 * m)(*[int(k) for k in pattern_kinds])
    out = (C.c_void_p * m)()
    st = lib().spai_build_batch(ctx, m, arr, kinds, out)
    pcs = [C.c_void_p(out[i]) if out[i] else None for i in range(m)]
    if st == SPAI_ESINGULAR and not allow_singular:
        msg = spai_last_error(ctx)
        for pc in pcs:
            if pc:
                lib().spai_pc_destroy(pc)
        raise SpaiError(st, msg)
    _check(ctx, st, allow=(SPAI_ESINGULAR,))
    return pcs, st


def spai_update(ctx, base, A_new, approach=UPDATE_FIRST, allow_singular=False):
    out = C.c_void_p()
    st = lib().spai_update(ctx, base, C.byref(A_new), int(approach), C.byref(out))
    if st == SPAI_ESINGULAR and not allow_singular:
        msg = spai_last_error(ctx)
        if out:
            lib().spai_pc_destroy(out)
        raise SpaiError(st, msg)
    _check(ctx, st, allow=(SPAI_ESINGULAR,))
    return out, st


def spai_pc_info(pc):
    n, nnz, depth = C.c_int32(), C.c_int32(), C.c_int32()
    nI = C.c_int64()
    _check(None, lib().spai_pc_info(pc, C.byref(n), C.byref(nnz), C.byref(nI), C.byref(depth)))
    return {"n": n.value, "nnz": nnz.value, "nI": nI.value, "depth": depth.value}


def spai_pc_export(ctx, pc, Jptr=None, Jind=None, val=None, Iptr=None, Ilist=None,
                   col_status=None):
    return _check(ctx, lib().spai_pc_export(ctx, pc, _ptr(Jptr), _ptr(Jind), _ptr(val), _ptr(Iptr),
                                            _ptr(Ilist), _ptr(col_status)))


def spai_pc_destroy(pc):
    return _check(None, lib().spai_pc_destroy(pc))


# ------------------------------------------------------------------ products and solve
def spai_spmm(ctx, A, s, X, ldx, Y, ldy):
    return _check(ctx, lib().spai_spmm(ctx, C.byref(A), int(s), _ptr(X), int(ldx), _ptr(Y), int(ldy)))


def spai_pc_apply(ctx, pc, s, X, ldx, Y, ldy):
    return _check(ctx, lib().spai_pc_apply(ctx, pc, int(s), _ptr(X), int(ldx), _ptr(Y), int(ldy)))


def spai_spmm_fp32(ctx, A, s, X, ldx, Y, ldy):
    """Y = A X with the FP32 operator of the mixed-precision solve (FP32 products and sums)."""
    return _check(ctx, lib().spai_spmm_fp32(ctx, C.byref(A), int(s), _ptr(X), int(ldx), _ptr(Y), int(ldy)))


def spai_pc_apply_fp32(ctx, pc, s, X, ldx, Y, ldy):
    """Y = P X with the FP32 operator of the mixed-precision solve."""
    return _check(ctx, lib().spai_pc_apply_fp32(ctx, pc, int(s), _ptr(X), int(ldx), _ptr(Y), int(ldy)))


def spai_pc_apply_noalloc(ctx, pc, s, X, ldx, Y, ldy):
    """Y = P X without allocating device memory (fixed 64 MiB staging array in the library).

    For callers that must not allocate where they apply the preconditioner, e.g. an outside
    solver loop that must not stall the device, or a process whose device memory is held
    by another allocator.  n * s <= 2,097,152; X and Y on the device.  The first call on a
    device caches the array's address (do it before any stream capture); overlapping
    calls share the array and race.
    """
    return _check(ctx, lib().spai_pc_apply_noalloc(ctx, pc, int(s), _ptr(X), int(ldx), _ptr(Y),
                                                   int(ldy)))


def spai_block_gram(ctx, s, n, nblk, V, W, H, method=ORTH_FP64):
    """H_i = V_i^T W for nblk row-major n x s blocks (device); method ORTH_FP64 / ORTH_TENSOR."""
    return _check(ctx, lib().spai_block_gram(ctx, int(s), int(n), int(nblk), _ptr(V), _ptr(W),
                                             _ptr(H), int(method)))


def spai_block_update(ctx, s, n, nblk, V, H, W, sign=-1.0, method=ORTH_FP64):
    """W := W + sign * sum_i V_i H_i in place (device, row-major blocks)."""
    return _check(ctx, lib().spai_block_update(ctx, int(s), int(n), int(nblk), _ptr(V), _ptr(H), _ptr(W),
                                               float(sign), int(method)))


def block_solve(ctx, A, P, s, B, ldb, X, ldx, restart, tol, max_cycles, allow_notconv=False,
                orth=ORTH_AUTO, precision=SOLVE_FP64):
    """Solve A X = B (column-major n x s; host or device).  Returns (status, info, rel)."""
    opts = spai_solve_opts(int(restart), int(max_cycles), float(tol), int(orth), int(precision))
    info = spai_solve_info()
    rel = (C.c_double * int(s))()
    st = lib().block_solve(ctx, C.byref(A), P, int(s), _ptr(B), int(ldb), _ptr(X), int(ldx),
                           C.byref(opts), C.byref(info), rel)
    result = (st, info.as_dict(), list(rel))
    if st == SPAI_ENOTCONV and not allow_notconv:
        raise SpaiError(st, spai_last_error(ctx), result)
    _check(ctx, st, allow=(SPAI_ENOTCONV,))
    return result


def spai_recycle_create(ctx, n, s, kmax):
    """Recycle space of block GCRO: up to kmax columns (a multiple of s) for n unknowns."""
    out = C.c_void_p()
    _check(ctx, lib().spai_recycle_create(ctx, int(n), int(s), int(kmax), C.byref(out)))
    return out


def spai_recycle_info(rc):
    k = C.c_int32()
    _check(None, lib().spai_recycle_info(rc, C.byref(k)))
    return k.value


def spai_recycle_export(ctx, rc, U, ldu):
    return _check(ctx, lib().spai_recycle_export(ctx, rc, _ptr(U), int(ldu)))


def spai_recycle_clear(rc):
    return _check(None, lib().spai_recycle_clear(rc))


def spai_recycle_destroy(rc):
    return _check(None, lib().spai_recycle_destroy(rc))


def block_solve_gcro(ctx, A, P, s, B, ldb, X, ldx, restart, tol, max_cycles, rc, allow_notconv=False,
                     orth=ORTH_AUTO, precision=SOLVE_FP64):
    """Block GCRO with the recycle space rc (see block_solve).  Returns (status, info, rel)."""
    opts = spai_solve_opts(int(restart), int(max_cycles), float(tol), int(orth), int(precision))
    info = spai_solve_info()
    rel = (C.c_double * int(s))()
    st = lib().block_solve_gcro(ctx, C.byref(A), P, int(s), _ptr(B), int(ldb), _ptr(X), int(ldx), C.byref(opts),
                                rc, C.byref(info), rel)
    result = (st, info.as_dict(), list(rel))
    if st == SPAI_ENOTCONV and not allow_notconv:
        raise SpaiError(st, spai_last_error(ctx), result)
    _check(ctx, st, allow=(SPAI_ENOTCONV,))
    return result


def spai_build_adaptive(ctx, A, eps=1e-4, max_steps=5, max_new=5, max_rows=128, flags=0, allow_singular=False):
    """Adaptive SPAI (pattern grown per column, then the column least squares on it).
    Returns (handle, status)."""
    o = spai_adaptive_opts(float(eps), int(max_steps), int(max_new), int(max_rows), 0)
    out = C.c_void_p()
    st = lib().spai_build_adaptive(ctx, C.byref(A), C.byref(o), int(flags), C.byref(out))
    if st == SPAI_ESINGULAR and not allow_singular:
        msg = spai_last_error(ctx)
        if out:
            lib().spai_pc_destroy(out)
        raise SpaiError(st, msg)
    _check(ctx, st, allow=(SPAI_ESINGULAR,))
    return out, st


def spai_column_variants(low_precision, maxI, maxJ):
    """Codes of the column-kernel variants that fit the tile shape (default first)."""
    buf = (C.c_int32 * 32)()
    k = lib().spai_column_variants(int(bool(low_precision)), int(maxI), int(maxJ), buf, 32)
    return [int(buf[i]) for i in range(min(k, 32))]


def spai_column_variant_get(low_precision, maxI, maxJ):
    return int(lib().spai_column_variant_get(int(bool(low_precision)), int(maxI), int(maxJ)))


def spai_column_variant_set(low_precision, maxI, maxJ, code):
    """Pin (code != 0) or clear (code 0) the column-kernel variant of a tile shape."""
    return _check(None, lib().spai_column_variant_set(int(bool(low_precision)), int(maxI), int(maxJ), int(code)))


def spai_ctx_trim(ctx):
    return _check(ctx, lib().spai_ctx_trim(ctx))


def spai_solve_workspace_size(n, s, restart):
    return int(lib().spai_solve_workspace_size(int(n), int(s), int(restart)))


def spai_pc_mem_size(pc, with_analysis=True):
    return int(lib().spai_pc_mem_size(pc, int(bool(with_analysis))))


# ------------------------------------------------------------------ serving
def _server_check(srv, st):
    if st != SPAI_OK:
        raise SpaiError(st, spai_server_last_error(srv) if srv else "")
    return st


def spai_server_create(slots=4, pattern_kind=PATTERN_A, reuse=True, restart=30, max_cycles=50,
                       orth=ORTH_AUTO, radius=0.05, tol=1e-8, mem_budget=0, precision=SOLVE_FP64):
    o = spai_server_opts(int(slots), int(pattern_kind), int(bool(reuse)), int(restart), int(max_cycles),
                         int(orth), float(radius), float(tol), int(mem_budget), int(precision), 0)
    out = C.c_void_p()
    st = lib().spai_server_create(C.byref(o), C.byref(out))
    if st != SPAI_OK:
        raise SpaiError(st, "spai_server_create failed")
    return out


def spai_server_add_system(srv, terms):
    """terms: list of spai_csr (host or device arrays).  Returns the system id."""
    arr = (spai_csr * len(terms))(*terms)
    sid = C.c_int32()
    _server_check(srv, lib().spai_server_add_system(srv, len(terms), arr, C.byref(sid)))
    return sid.value


def spai_server_add_shifted_system(srv, terms, alpha, beta):
    """terms: (M, K_0, K_1) as spai_csr; requests may then pass coef=None (A(p, s) formed by
    the server with damping D = alpha M + beta K(p)).  Returns the system id."""
    arr = (spai_csr * len(terms))(*terms)
    if len(terms) != 3:
        raise SpaiError(SPAI_EINVAL, "a shifted system has the three terms (M, K_0, K_1)")
    sid = C.c_int32()
    _server_check(srv, lib().spai_server_add_shifted_system(srv, arr, float(alpha), float(beta), C.byref(sid)))
    return sid.value


def spai_server_submit(srv, system, nrhs, p, s, coef, B, X=None, t_arrival=-1.0):
    """Queue one solve; B / X host or device, n x nrhs column-major (leading dimension n).
    coef=None for a shifted system (the server forms A(p, s)).  Returns the ticket.  B (and
    X) must stay alive until the request completes."""
    cf = None if coef is None else (C.c_double * len(coef))(*[float(c) for c in coef])
    r = spai_request(int(system), int(nrhs), float(p), float(s), C.cast(cf, C.c_void_p) if cf is not None else None,
                     _ptr(B), _ptr(X), float(t_arrival))
    t = C.c_int64()
    _server_check(srv, lib().spai_server_submit(srv, C.byref(r), C.byref(t)))
    return t.value


def spai_server_wait(srv, ticket):
    """Block until the request completes; returns its result as a dict."""
    res = spai_result()
    _server_check(srv, lib().spai_server_wait(srv, int(ticket), C.byref(res)))
    return res.as_dict()


def spai_server_clock(srv):
    return float(lib().spai_server_clock(srv))


def spai_server_stats_get(srv):
    out = spai_server_stats()
    _server_check(srv, lib().spai_server_stats_get(srv, C.byref(out)))
    return out.as_dict()


def spai_server_last_error(srv):
    r = lib().spai_server_last_error(srv)
    return r.decode() if r else ""


def spai_server_destroy(srv):
    return _server_check(None, lib().spai_server_destroy(srv))


def block_solve_batch(ctx, As, Ps, s, Bs, Xs, restart, tol, max_cycles, allow_notconv=False):
    """Solve the systems As[i] X_i = Bs[i] (device, column-major n_i x s) at once in lockstep.
    Ps: list of handles or None.  Xs hold the initial guesses and receive the solutions.
    Returns (status, list of info dicts)."""
    m = len(As)
    arr = (spai_csr * m)(*As)
    pcs = (C.c_void_p * m)(*[p.value if hasattr(p, "value") else p for p in Ps]) if Ps is not None else None
    bp = (C.c_void_p * m)(*[_ptr(b) for b in Bs])
    xp = (C.c_void_p * m)(*[_ptr(x) for x in Xs])
    opts = spai_solve_opts(int(restart), int(max_cycles), float(tol), 0, 0)
    infos = (spai_solve_info * m)()
    st = lib().block_solve_batch(ctx, m, arr, pcs, int(s), bp, xp, C.byref(opts), infos)
    result = (st, [infos[i].as_dict() for i in range(m)])
    if st == SPAI_ENOTCONV and not allow_notconv:
        raise SpaiError(st, spai_last_error(ctx), result)
    _check(ctx, st, allow=(SPAI_ENOTCONV,))
    return result
