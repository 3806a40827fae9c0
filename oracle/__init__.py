"""Plain FP64 CPU oracle of the SPAI / SPAI-update / right-preconditioned block GMRES path.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package; the product library never does.
It shares no code with the CUDA path (separate C file, separate numpy code); both only
consume the seeded inputs of the ``synth`` module.

What it computes, with the passage of arXiv 1809.06574 it writes out:

* ``coefficients`` / ``assemble`` -- A(p, s) = s^2 M + s D + K(p) with Rayleigh damping
  D = 0.05 M + 0.01 K(p) and K(p) = K0 + p K1, written as the affine combination of
  Sec. 1.1 (Eqs. (4)-(9)) on the union of the terms' patterns.
* ``pattern`` / ``index_sets`` -- the fixed column patterns J_k (pattern of A or of A^2)
  and row sets I_k of the column least-squares problems of Sec. 2.2.
* ``spai_build`` -- min_P ||I - A P||_F, column by column (Sec. 2.2), by Householder QR.
* ``spai_update`` -- min_Q ||A(1) - A(l) Q||_F (Table 1 first approach, Sec. 2.4),
  P_l = Q_l P_1 kept factored; ``spai_update_chained`` is Table 1's second approach;
  ``spai_update_diagonal`` takes Q_l diagonal (the same least squares on J_k = {k}).
* ``spai_adaptive_pattern`` / ``spai_build_adaptive`` -- SPAI on a pattern grown column
  by column (the adaptive pattern of the MSPAI code the paper runs, Sec. 3: tolerance
  1e-4): least squares on J_k, residual, candidate columns that meet the residual's rows,
  their one-dimensional improvement, the best below the mean added, until the residual
  norm is below the tolerance or a step limit is reached.
* ``block_gmres`` -- the right-preconditioned (Sec. 2.2 footnote) block Krylov solve
  of Sec. 2.1: block GMRES(m) over span{R0, AP R0, (AP)^2 R0, ...}.
* ``block_gcro`` -- block GCRO (the solver of the paper's experiments, Sec. 3) with a
  recycled outer space carried along the sequence of systems (Sec. 1.3): the minimal-
  residual iterate over span(U) first, then cycles over span([U, V]) with V the block
  Krylov space of the operator projected against C = AP U.
* ``lu_solve`` -- dense LU with partial pivoting for tiny reference solves.

Pinned by the ``-m "not gpu"`` tests in ``tests/test_oracle_*.py`` against closed forms
(full pattern -> A^{-1}, diagonal A -> 1/a_ii, diagonal pattern -> a_kk/||A(:,k)||^2,
unchanged parameter -> Q = I, scaled A -> Q = I/c, the Appendix I example), brute-force
least squares on dense matrices, SciPy's GMRES for one right-hand side and a dense
solve.  Parity is pinned for every function listed above.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        i32, i64, dbl = C.c_int32, C.c_int64, C.c_double
        P = C.c_void_p
        L.oracle_union_pattern.restype = i64
        L.oracle_union_pattern.argtypes = [i32, i32, P, P, P, P, P]
        L.oracle_assemble_values.restype = None
        L.oracle_assemble_values.argtypes = [i32, i32, P, P, P, P, P, P, P, P]
        L.oracle_csr_to_csc.restype = None
        L.oracle_csr_to_csc.argtypes = [i32, P, P, P, P, P, P]
        L.oracle_pattern_a2.restype = i64
        L.oracle_pattern_a2.argtypes = [i32, P, P, P, P]
        L.oracle_index_sets.restype = i64
        L.oracle_index_sets.argtypes = [i32, P, P, P, P, P, P]
        L.oracle_spai_columns.restype = i64
        L.oracle_spai_columns.argtypes = [i32, P, P, P, P, P, P, P, i32, P, P, P, i32, i32, P, P]
        L.oracle_spmm_csr.restype = None
        L.oracle_spmm_csr.argtypes = [i32, P, P, P, i32, P, i64, P, i64]
        L.oracle_spmm_csc.restype = None
        L.oracle_spmm_csc.argtypes = [i32, P, P, P, i32, P, i64, P, i64]
        L.oracle_dense_lu_solve.restype = i32
        L.oracle_dense_lu_solve.argtypes = [i32, P, i64, i32, P, i64]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------------------
# assembly (Sec. 1.1)
# --------------------------------------------------------------------------------------

def coefficients(p: float, s: float):
    """Coefficients of (M, K0, K1) in A(p, s) = s^2 M + s D(p) + K(p).

    D(p) = 0.05 M + 0.01 K(p) (Rayleigh damping, the alpha M + beta K form of Sec. 3),
    K(p) = K0 + p K1.  Collecting terms: (s^2 + 0.05 s) M + (1 + 0.01 s) K0
    + (1 + 0.01 s) p K1.
    """
    return [s * s + 0.05 * s, 1.0 + 0.01 * s, (1.0 + 0.01 * s) * p]


def _concat_terms(terms, n):
    T = len(terms)
    rp = np.concatenate([_i32(t[0]) for t in terms])
    assert rp.size == T * (n + 1)
    ci = np.concatenate([_i32(t[1]) for t in terms])
    va = np.concatenate([_f64(t[2]) for t in terms])
    off = np.zeros(T, dtype=np.int64)
    acc = 0
    for t in range(T):
        off[t] = acc
        acc += len(terms[t][1])
    return T, rp, ci, va, off


def union_pattern(terms, n):
    T, rp, ci, _va, off = _concat_terms(terms, n)
    L = lib()
    nnz = L.oracle_union_pattern(n, T, _p(rp), _p(ci), _p(off), None, None)
    rowptr = np.zeros(n + 1, np.int32)
    colind = np.zeros(max(nnz, 1), np.int32)
    L.oracle_union_pattern(n, T, _p(rp), _p(ci), _p(off), _p(rowptr), _p(colind))
    return rowptr, colind[:nnz]


def assemble(terms, coef, n):
    """CSR of sum_t coef[t] * terms[t] on the union pattern (structural zeros kept)."""
    T, rp, ci, va, off = _concat_terms(terms, n)
    rowptr, colind = union_pattern(terms, n)
    val = np.zeros(max(len(colind), 1))
    cf = _f64(coef)
    assert cf.size == T
    lib().oracle_assemble_values(n, T, _p(rp), _p(ci), _p(va), _p(off), _p(cf), _p(rowptr),
                                 _p(colind), _p(val))
    return rowptr, colind, val[:len(colind)]


# --------------------------------------------------------------------------------------
# patterns and index sets (Sec. 2.2)
# --------------------------------------------------------------------------------------

def csr_to_csc(A, n):
    rowptr, colind, val = _i32(A[0]), _i32(A[1]), _f64(A[2])
    nnz = len(colind)
    colptr = np.zeros(n + 1, np.int32)
    rowind = np.zeros(max(nnz, 1), np.int32)
    cval = np.zeros(max(nnz, 1))
    lib().oracle_csr_to_csc(n, _p(rowptr), _p(colind), _p(val), _p(colptr), _p(rowind), _p(cval))
    return colptr, rowind[:nnz], cval[:nnz]


PATTERN_A = 0
PATTERN_A2 = 1


def pattern(A, n, kind=PATTERN_A):
    """Column patterns J_k of P: pattern of A (columns of A) or structural pattern of A^2."""
    colptr, rowind, _ = csr_to_csc(A, n)
    if kind == PATTERN_A:
        return colptr, rowind
    L = lib()
    tot = L.oracle_pattern_a2(n, _p(colptr), _p(rowind), None, None)
    Jptr = np.zeros(n + 1, np.int32)
    Jind = np.zeros(max(tot, 1), np.int32)
    L.oracle_pattern_a2(n, _p(colptr), _p(rowind), _p(Jptr), _p(Jind))
    return Jptr, Jind[:tot]


def index_sets(A, n, Jptr, Jind):
    colptr, rowind, _ = csr_to_csc(A, n)
    Jptr, Jind = _i32(Jptr), _i32(Jind)
    L = lib()
    tot = L.oracle_index_sets(n, _p(colptr), _p(rowind), _p(Jptr), _p(Jind), None, None)
    Iptr = np.zeros(n + 1, np.int32)
    Ilist = np.zeros(max(tot, 1), np.int32)
    L.oracle_index_sets(n, _p(colptr), _p(rowind), _p(Jptr), _p(Jind), _p(Iptr), _p(Ilist))
    return Iptr, Ilist[:tot]


# --------------------------------------------------------------------------------------
# SPAI build and update (Sec. 2.2, Sec. 2.3 Table 1, Sec. 2.4)
# --------------------------------------------------------------------------------------

class Precond:
    """Column-wise result on pattern J: column k has rows Jind[Jptr[k]:Jptr[k+1]], values val."""

    def __init__(self, n, Jptr, Jind, Iptr, Ilist, val, status, base=None, A_csc=None):
        self.n, self.Jptr, self.Jind, self.Iptr, self.Ilist = n, Jptr, Jind, Iptr, Ilist
        self.val, self.status, self.base, self.A_csc = val, status, base, A_csc

    def dense(self):
        D = np.zeros((self.n, self.n))
        for k in range(self.n):
            sl = slice(self.Jptr[k], self.Jptr[k + 1])
            D[self.Jind[sl], k] = self.val[sl]
        return D

    def apply_own(self, X):
        """Y = (this factor) X, X of shape (n, s)."""
        X = np.asfortranarray(X, dtype=np.float64)
        n, s = X.shape
        Y = np.zeros((n, s), order="F")
        lib().oracle_spmm_csc(n, _p(self.Jptr), _p(self.Jind), _p(self.val), s, _p(X), n, _p(Y), n)
        return Y

    def apply(self, X):
        """P_l X with P_l = Q_l P_base (factored apply, Sec. 2.4: P_l = Q_l P_1)."""
        if self.base is None:
            return self.apply_own(X)
        return self.apply_own(self.base.apply(X))

    def dense_product(self):
        """Explicit P_l = Q_l P_base (test-only)."""
        if self.base is None:
            return self.dense()
        return self.dense() @ self.base.dense_product()


def _columns(A_csc, n, Jptr, Jind, Iptr, Ilist, mode, R_csc=None, k0=0, k1=None):
    colptr, rowind, cval = A_csc
    k1 = n if k1 is None else k1
    val = np.zeros(max(len(Jind), 1))
    status = np.zeros(max(k1 - k0, 1), np.int32)
    if R_csc is None:
        R_csc = (colptr, rowind, cval)
    lib().oracle_spai_columns(n, _p(colptr), _p(rowind), _p(cval), _p(Jptr), _p(Jind), _p(Iptr),
                              _p(Ilist), mode, _p(R_csc[0]), _p(R_csc[1]), _p(R_csc[2]), k0, k1,
                              _p(val), _p(status))
    return val[:len(Jind)], status[:k1 - k0]


def spai_build(A, n, kind=PATTERN_A, k0=0, k1=None, sets=None):
    """SPAI of A (Sec. 2.2): column k = argmin over supp in J_k of ||e_k - A m||_2.

    Columns k0 <= k < k1 only, if given (the others stay 0).  ``sets`` = (Jptr, Jind,
    Iptr, Ilist) as returned by ``pattern`` and ``index_sets`` for this A and kind, to
    reuse them across calls on the same matrix."""
    A_csc = csr_to_csc(A, n)
    if sets is None:
        Jptr, Jind = pattern(A, n, kind)
        Iptr, Ilist = index_sets(A, n, Jptr, Jind)
    else:
        Jptr, Jind, Iptr, Ilist = (_i32(a) for a in sets)
    val, status = _columns(A_csc, n, Jptr, Jind, Iptr, Ilist, 0, None, k0, k1)
    return Precond(n, Jptr, Jind, Iptr, Ilist, val, status, None, A_csc)


# --------------------------------------------------------------------------------------
# adaptive pattern (MSPAI, Sec. 3; the least squares of Sec. 2.2 on a growing J_k)
# --------------------------------------------------------------------------------------

ADAPTIVE_KEY_BITS = 30   # improvements compare at 2^-30 of ||r||^2 (ties: lower column index)
ADAPTIVE_MAX_COLS = 32   # 1 + max_steps * max_new must not exceed this
ADAPTIVE_MAX_ROWS = 128  # largest accepted max_rows option (|I_k| above max_rows stops the growth)


def _adaptive_key(x, rr):
    """Quantised improvement: floor(x / ||r||^2 * 2^30), clamped to [0, 2^30]."""
    q = np.floor((x / rr) * float(1 << ADAPTIVE_KEY_BITS))
    return int(min(max(q, 0.0), float(1 << ADAPTIVE_KEY_BITS)))


def spai_adaptive_pattern(A, n, eps=1e-4, max_steps=5, max_new=5, max_rows=ADAPTIVE_MAX_ROWS, k0=0, k1=None,
                          trace=None):
    """Column patterns J_k of the adaptive SPAI, one column at a time (plain loops; small n).

    For column k, starting from J_k = {k}:
      1. I_k = {k} and the rows of the columns in J_k; m = argmin ||e_k - A(:, J_k) m||_2
         (the column least squares of Sec. 2.2, solved here by numpy's Householder QR);
      2. r = e_k - sum_c A(:, J_c) m_c (column by column); stop if ||r||_2 <= eps, after
         max_steps additions, or if the least squares is rank deficient;
      3. candidates: the columns j not in J_k with a nonzero in a row of I_k (the rows where
         r can be nonzero); for each, the squared residual after the best one-column
         correction, rho_j = ||r||^2 - (r . A(:,j))^2 / ||A(:,j)||^2;
      4. add the at most max_new candidates of smallest rho_j among those with rho_j not
         above the candidates' mean (compared as floor(rho / ||r||^2 * 2^30); ties by the
         lower column index); the step is undone and the growth stops if |I_k| would
         exceed max_rows.  The options bound the pattern: |J_k| <= 1 + max_steps * max_new
         <= 32, |I_k| <= max_rows <= 128; every candidate of a step is scored, however many
         there are.  A zero column of A offers no improvement (rho_j = ||r||^2).
    Returns (Jptr, Jind) for columns k0 <= k < k1 (others J_k = {k}).  ``trace``, a list,
    receives (k, step, J, I, rr, candidates, rho, chosen) per step for the tests."""
    if 1 + max_steps * max_new > ADAPTIVE_MAX_COLS or max_rows > ADAPTIVE_MAX_ROWS:
        raise ValueError("pattern limits exceed the supported sizes")
    k1 = n if k1 is None else k1
    rowptr, colind, val = _i32(A[0]), _i32(A[1]), _f64(A[2])
    colptr, rowind, cval = csr_to_csc(A, n)
    colnorm2 = np.zeros(n)
    for j in range(n):
        acc = 0.0
        for q in range(colptr[j], colptr[j + 1]):
            acc = acc + cval[q] * cval[q]
        colnorm2[j] = acc
    pats = []
    for k in range(n):
        if not (k0 <= k < k1):
            pats.append([k])
            continue
        J = [k]

        def rows_of(cols):
            out = {k}
            for j in cols:
                out.update(int(x) for x in rowind[colptr[j]:colptr[j + 1]])
            return sorted(out)

        I = rows_of(J)
        for step in range(max_steps + 1 if len(I) <= max_rows else 0):
            pos = {row: i for i, row in enumerate(I)}
            Ah = np.zeros((len(I), len(J)))
            for c, j in enumerate(J):
                for q in range(colptr[j], colptr[j + 1]):
                    Ah[pos[int(rowind[q])], c] = cval[q]
            rhs = np.zeros(len(I))
            rhs[pos[k]] = 1.0
            if len(I) < len(J):
                break
            Q, R = np.linalg.qr(Ah)
            d = np.abs(np.diag(R))
            if d.max() == 0.0 or d.min() <= 1e-14 * d.max():
                break
            m = np.linalg.solve(R, Q.T @ rhs)
            r = rhs.copy()
            for c, j in enumerate(J):
                for q in range(colptr[j], colptr[j + 1]):
                    i = pos[int(rowind[q])]
                    r[i] = r[i] - cval[q] * m[c]
            rr = 0.0
            for x in r:
                rr = rr + x * x
            if np.sqrt(rr) <= eps or step == max_steps:
                break
            inJ = set(J)
            cand = sorted({int(j) for row in I for j in colind[rowptr[row]:rowptr[row + 1]]} - inJ)
            if not cand:
                break
            rho = []
            for j in cand:
                dot = 0.0
                for q in range(colptr[j], colptr[j + 1]):
                    i = pos.get(int(rowind[q]))
                    if i is not None:
                        dot = dot + r[i] * cval[q]
                rho.append(rr if colnorm2[j] == 0.0 else rr - dot * dot / colnorm2[j])
            mean = 0.0
            for x in rho:
                mean = mean + x
            mean = mean / len(rho)
            kmean = _adaptive_key(mean, rr)
            keyed = sorted((_adaptive_key(x, rr), j) for x, j in zip(rho, cand) if _adaptive_key(x, rr) <= kmean)
            chosen = [j for _, j in keyed[:max_new]]
            if trace is not None:
                trace.append((k, step, list(J), list(I), rr, cand, rho, chosen))
            newJ = sorted(J + chosen)
            newI = rows_of(newJ)
            if len(newI) > max_rows:
                break
            J, I = newJ, newI
        pats.append(J)
    Jptr = np.zeros(n + 1, np.int32)
    Jptr[1:] = np.cumsum([len(x) for x in pats])
    Jind = np.array([j for x in pats for j in x], np.int32)
    return Jptr, Jind


def spai_build_adaptive(A, n, eps=1e-4, max_steps=5, max_new=5, max_rows=ADAPTIVE_MAX_ROWS, k0=0, k1=None):
    """Adaptive SPAI: the pattern of ``spai_adaptive_pattern``, then the column least
    squares of ``spai_build`` on it (Householder QR, Sec. 2.2)."""
    Jptr, Jind = spai_adaptive_pattern(A, n, eps, max_steps, max_new, max_rows, k0, k1)
    Iptr, Ilist = index_sets(A, n, Jptr, Jind)
    return spai_build(A, n, PATTERN_A, k0, k1, sets=(Jptr, Jind, Iptr, Ilist))


def spai_update(base: Precond, A_new, n, k0=0, k1=None):
    """Update of the first approach (Table 1, Sec. 2.4).

    Column k of Q_l = argmin over supp in J_k of ||a1_k - A(l) q||_2, where a1_k is column
    k of the base matrix A(1); the preconditioner of A(l) is P_l = Q_l P_1, applied
    factored.  Q_l takes P_1's pattern (the paper does not state one).
    """
    root = base
    while root.base is not None:
        root = root.base
    A_csc = csr_to_csc(A_new, n)
    val, status = _columns(A_csc, n, root.Jptr, root.Jind, root.Iptr, root.Ilist, 1, root.A_csc,
                           k0, k1)
    return Precond(n, root.Jptr, root.Jind, root.Iptr, root.Ilist, val, status, root, A_csc)


def spai_update_chained(prev: Precond, A_new, n):
    """Second approach of Table 1: min ||A(i-1) - A(i) Q_i||_F and P_i = Q_i P_{i-1}."""
    A_csc = csr_to_csc(A_new, n)
    val, status = _columns(A_csc, n, prev.Jptr, prev.Jind, prev.Iptr, prev.Ilist, 1, prev.A_csc)
    return Precond(n, prev.Jptr, prev.Jind, prev.Iptr, prev.Ilist, val, status, prev, A_csc)


def spai_update_diagonal(base: Precond, A_new, n):
    """Update with a diagonal Q_l (Table 1 first approach; Q_l's pattern is not stated in
    Sec. 2.4, this is the diagonal reading): column k of Q_l is argmin over supp in {k} of
    ||a1_k - A(l) q||_2, the same column least squares as ``spai_update`` on the pattern
    J_k = {k}, whose rows are I_k = rows(A(l)(:,k)).  P_l = Q_l P_1, applied factored."""
    root = base
    while root.base is not None:
        root = root.base
    Jptr = np.arange(n + 1, dtype=np.int32)
    Jind = np.arange(n, dtype=np.int32)
    Iptr, Ilist = index_sets(A_new, n, Jptr, Jind)
    A_csc = csr_to_csc(A_new, n)
    val, status = _columns(A_csc, n, Jptr, Jind, Iptr, Ilist, 1, root.A_csc)
    return Precond(n, Jptr, Jind, Iptr, Ilist, val, status, root, A_csc)


def spmm(A, X, n):
    """Y = A X for CSR A and dense X (n, s)."""
    X = np.asfortranarray(X, dtype=np.float64)
    s = X.shape[1]
    Y = np.zeros((n, s), order="F")
    lib().oracle_spmm_csr(n, _p(_i32(A[0])), _p(_i32(A[1])), _p(_f64(A[2])), s, _p(X), n, _p(Y), n)
    return Y


def lu_solve(D, B):
    """Dense LU with partial pivoting: returns D^{-1} B (D and B are copied)."""
    D = np.array(D, dtype=np.float64, order="F")
    B = np.array(B, dtype=np.float64, order="F", ndmin=2)
    if B.shape[0] != D.shape[0]:
        B = B.T.copy(order="F")
    n, nrhs = B.shape
    rc = lib().oracle_dense_lu_solve(n, _p(D), n, nrhs, _p(B), n)
    if rc != 0:
        raise np.linalg.LinAlgError("singular matrix")
    return B


# --------------------------------------------------------------------------------------
# right-preconditioned block GMRES(m) (Sec. 2.1; right preconditioning: Sec. 2.2 footnote)
# --------------------------------------------------------------------------------------

DEFLATE_REL = 1e-12


def _block_qr(W, ref):
    """Orthonormal basis of range(W): W = Q R with R upper triangular (Householder QR).

    Columns are taken in order.  A column whose new direction is negligible -- its
    diagonal |R_kk| in the QR of [kept columns before it, itself] is <= 1e-12 * ref_k
    (ref = the column's norm before orthogonalisation) -- is deflated: it gets no basis
    vector (Q[:, k] = 0, row k of R = 0) and is represented by its coefficients on the
    kept vectors before it, so it adds nothing to the Krylov space.
    """
    n, s = W.shape
    kept = []
    for k in range(s):
        _, Rt = np.linalg.qr(W[:, kept + [k]], mode="reduced")
        if abs(Rt[-1, -1]) > DEFLATE_REL * ref[k]:
            kept.append(k)
    Q = np.zeros((n, s))
    R = np.zeros((s, s))
    if kept:
        Qk, Rk = np.linalg.qr(W[:, kept], mode="reduced")
        Q[:, kept] = Qk
        for a, ka in enumerate(kept):
            for b, kb in enumerate(kept):
                R[ka, kb] = Rk[a, b]
        for k in range(s):
            if k in kept:
                continue
            for a, ka in enumerate(kept):
                if ka < k:
                    R[ka, k] = Qk[:, a] @ W[:, k]
    return Q, R


class GmresInfo(dict):
    pass


def block_gmres(apply_A, apply_P, B, restart, tol, max_cycles, X0=None, history=False):
    """Solve A X = B by right-preconditioned block GMRES(restart): A P X~ = B, X = P X~.

    Each cycle builds an orthonormal basis V_0..V_j of the block Krylov space
    span{R0, (AP) R0, ..., (AP)^j R0} (R0 = B - A X0) by block Arnoldi with two passes of
    block classical Gram-Schmidt, and takes the iterate minimising every column's
    residual over that space: Y = argmin ||E_1 S_0 - Hbar_j Y|| (solved directly by
    least squares), X = X0 + P [V_0..V_j] Y.  The cycle stops early once every column's
    least-squares residual is <= tol * ||b_i||; after each cycle the true residual
    B - A X is formed, and the solve stops when every column has ||b_i - A x_i|| <=
    tol * ||b_i||.  ``apply_P`` may be None (no preconditioner).
    """
    B = np.asarray(B, dtype=np.float64)
    n, s = B.shape
    m = int(restart)
    if apply_P is None:
        def apply_P(X):
            return X
    X = np.zeros((n, s)) if X0 is None else np.array(X0, dtype=np.float64)
    bnorm = np.linalg.norm(B, axis=0)
    thresh = tol * bnorm
    R = B - apply_A(X)
    iters, cycles = 0, 0
    est_hist = []
    while True:
        rn = np.linalg.norm(R, axis=0)
        if np.all(rn <= thresh) or cycles >= max_cycles:
            break
        cycles += 1
        V0, S0 = _block_qr(R, rn)
        Vs = [V0]
        H = np.zeros(((m + 1) * s, m * s))
        G0 = np.zeros(((m + 1) * s, s))
        G0[:s] = S0
        Y = None
        for j in range(m):
            Z = apply_P(Vs[j])
            W = apply_A(Z)
            wn = np.linalg.norm(W, axis=0)
            Vc = np.hstack(Vs)
            H1 = Vc.T @ W
            W = W - Vc @ H1
            H2 = Vc.T @ W
            W = W - Vc @ H2
            H[:(j + 1) * s, j * s:(j + 1) * s] = H1 + H2
            Vn, Rn = _block_qr(W, wn)
            H[(j + 1) * s:(j + 2) * s, j * s:(j + 1) * s] = Rn
            Vs.append(Vn)
            Hb = H[:(j + 2) * s, :(j + 1) * s]
            Gb = G0[:(j + 2) * s]
            Y = np.linalg.lstsq(Hb, Gb, rcond=None)[0]
            est = np.linalg.norm(Gb - Hb @ Y, axis=0)
            est_hist.append(est)
            iters += 1
            if np.all(est <= thresh):
                break
        U = np.hstack(Vs[:Y.shape[0] // s]) @ Y
        X = X + apply_P(U)
        R = B - apply_A(X)
    rn = np.linalg.norm(R, axis=0)
    rel = np.where(bnorm > 0, rn / np.where(bnorm > 0, bnorm, 1.0), rn)
    info = GmresInfo(iterations=iters, cycles=cycles, converged=bool(np.all(rn <= thresh)),
                     rel_residual=rel)
    if history:
        info["estimates"] = est_hist
    return X, info


def block_gcro(apply_A, apply_P, B, restart, tol, max_cycles, U=None, kmax=0, history=False):
    """Right-preconditioned block GCRO with a recycled outer space (the GCRO solver the paper
    runs, Sec. 3, in block form; its outer space carried along the sequence of systems of
    Sec. 1.3).  With the operator AP = A P and a recycled space U (n x k, in the
    preconditioned space; None: none):

      1. C T = AP U, the thin QR of the image with the deflation rule of ``_block_qr`` (a
         column that AP U leaves dependent gets C[:, i] = 0 and U[:, i] = 0), U <- U T^{-1},
         so that AP U = C, C^T C = I;
      2. X~ = U C^T B, R = B - C C^T B: the minimal-residual iterate over span(U);
      3. cycles of block Arnoldi of (I - C C^T) AP from R, with two passes of block
         classical Gram-Schmidt against [C, V_0..V_j]: AP V_j = C B_j + V_{0..j+1} Hbar_j.
         With Gbar = [[I_k, B], [0, Hbar]], AP [U, V_{0..j}] = [C, V_{0..j+1}] Gbar, and the
         iterate minimises every column's residual over X~ + span([U, V_{0..j}]):
         y = argmin ||[0; E_1 S_0] - Gbar y|| (solved directly by least squares),
         X~ += [U, V] y.  Early stop and true residuals as ``block_gmres``;
      4. X = P X~.

    Returns (X, info, U_next): U_next = the last kmax columns of [U, X~], the recycled space
    of the next system (None when kmax = 0).  With U None this is ``block_gmres``.
    """
    B = np.asarray(B, dtype=np.float64)
    n, s = B.shape
    m = int(restart)
    if apply_P is None:
        def apply_P(X):
            return X

    def apply_AP(X):
        return apply_A(apply_P(X))

    bnorm = np.linalg.norm(B, axis=0)
    thresh = tol * bnorm
    Xh = np.zeros((n, s))
    if U is not None and U.shape[1] > 0:
        U = np.asarray(U, dtype=np.float64)
        k = U.shape[1]
        CU = apply_AP(U)
        C, T = _block_qr(CU, np.linalg.norm(CU, axis=0))
        kept = [i for i in range(k) if np.any(C[:, i] != 0.0)]
        Un = np.zeros((n, k))
        if kept:
            Un[:, kept] = U[:, kept] @ np.linalg.inv(T[np.ix_(kept, kept)])
        U = Un
        coef = C.T @ B
        Xh = U @ coef
        R = B - C @ coef
    else:
        k = 0
        U = np.zeros((n, 0))
        C = np.zeros((n, 0))
        R = B.copy()
    iters, cycles = 0, 0
    est_hist = []
    while True:
        rn = np.linalg.norm(R, axis=0)
        if np.all(rn <= thresh) or cycles >= max_cycles:
            break
        cycles += 1
        V0, S0 = _block_qr(R, rn)
        Vs = [V0]
        Gbar = np.zeros((k + (m + 1) * s, k + m * s))
        Gbar[:k, :k] = np.eye(k)
        rhs = np.zeros((k + (m + 1) * s, s))
        rhs[k:k + s] = S0
        y = None
        for j in range(m):
            W = apply_AP(Vs[j])
            wn = np.linalg.norm(W, axis=0)
            Bas = np.hstack([C] + Vs)
            H1 = Bas.T @ W
            W = W - Bas @ H1
            H2 = Bas.T @ W
            W = W - Bas @ H2
            Gbar[:k + (j + 1) * s, k + j * s:k + (j + 1) * s] = H1 + H2
            Vn, Rn = _block_qr(W, wn)
            Gbar[k + (j + 1) * s:k + (j + 2) * s, k + j * s:k + (j + 1) * s] = Rn
            Vs.append(Vn)
            Gb = Gbar[:k + (j + 2) * s, :k + (j + 1) * s]
            rb = rhs[:k + (j + 2) * s]
            y = np.linalg.lstsq(Gb, rb, rcond=None)[0]
            est = np.linalg.norm(rb - Gb @ y, axis=0)
            est_hist.append(est)
            iters += 1
            if np.all(est <= thresh):
                break
        Xh = Xh + np.hstack([U] + Vs[:(y.shape[0] - k) // s]) @ y
        R = B - apply_AP(Xh)
    X = apply_P(Xh)
    rn = np.linalg.norm(B - apply_A(X), axis=0)
    rel = np.where(bnorm > 0, rn / np.where(bnorm > 0, bnorm, 1.0), rn)
    info = GmresInfo(iterations=iters, cycles=cycles, converged=bool(np.all(rn <= thresh)),
                     rel_residual=rel)
    if history:
        info["estimates"] = est_hist
    U_next = None
    if kmax:
        U_next = np.hstack([U, Xh])[:, -int(kmax):]
    return X, info, U_next


def csr_apply(A, n):
    """Closure X -> A X for the oracle's solve (CSR sparse times dense)."""
    def f(X):
        return np.asarray(spmm(A, X, n))
    return f
