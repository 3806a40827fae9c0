"""Pins of the oracle's SPAI build and update (CPU only).

Closed forms: full pattern -> A^{-1}; diagonal A -> 1/a_ii; diagonal pattern ->
a_kk/||A(:,k)||^2; unchanged parameter -> Q = I; A(l) = c A(1) -> Q = I/c; the Appendix I
example, whose inverse has the pattern of A, so SPAI and the update reproduce
A^{-1} exactly.  Brute force: dense least squares over all n rows (LAPACK lstsq) on
tiny random sparse matrices; normal-equation orthogonality; feasibility bounds.
"""

import json
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _csr(D, keep=None):
    return synth.dense_to_csr(D, keep)


def test_full_pattern_gives_inverse():
    rng = np.random.default_rng(0)
    n = 17
    D = rng.standard_normal((n, n)) + n * np.eye(n)
    A = _csr(D, np.ones((n, n), dtype=bool))
    P = oracle.spai_build(A, n)
    assert not P.status.any()
    Ainv = oracle.lu_solve(D, np.eye(n))
    assert np.max(np.abs(P.dense() - Ainv)) <= 1e-12 * np.max(np.abs(Ainv))
    assert np.max(np.abs(P.dense() - np.linalg.inv(D))) <= 1e-12 * np.max(np.abs(Ainv))


def test_diagonal_matrix_gives_reciprocal():
    d = np.array([3.0, -0.5, 7.25, 1e-3, 2.0])
    A = synth.diag_csr(d)
    P = oracle.spai_build(A, 5)
    assert np.allclose(np.diag(P.dense()), 1.0 / d, rtol=1e-15, atol=0)


def test_diagonal_pattern_closed_form():
    n = 29
    (A, D) = synth.random_sparse(n, 0.15, seed=11)
    Jptr = np.arange(n + 1, dtype=np.int32)
    Jind = np.arange(n, dtype=np.int32)
    Iptr, Ilist = oracle.index_sets(A, n, Jptr, Jind)
    val, st = oracle._columns(oracle.csr_to_csc(A, n), n, Jptr, Jind, Iptr, Ilist, 0)
    ref = np.diag(D) / np.sum(D * D, axis=0)
    assert not st.any()
    assert np.max(np.abs(val - ref) / np.abs(ref)) <= 1e-14


@pytest.mark.parametrize("seed,kind", [(0, oracle.PATTERN_A), (1, oracle.PATTERN_A),
                                       (2, oracle.PATTERN_A2), (3, oracle.PATTERN_A2)])
def test_build_matches_dense_lstsq(seed, kind):
    n = 40
    (A, D) = synth.random_sparse(n, 0.07, seed=seed)
    P = oracle.spai_build(A, n, kind)
    Pd = P.dense()
    for k in range(n):
        J = P.Jind[P.Jptr[k]:P.Jptr[k + 1]]
        e = np.zeros(n)
        e[k] = 1.0
        m = np.linalg.lstsq(D[:, J], e, rcond=None)[0]
        assert np.max(np.abs(Pd[J, k] - m)) <= 1e-12 * max(1.0, np.max(np.abs(m)))
        # zero outside the pattern
        mask = np.ones(n, dtype=bool)
        mask[J] = False
        assert not np.any(Pd[mask, k])


def test_build_normal_equations_and_residual_bound():
    n = 60
    (A, D) = synth.random_sparse(n, 0.05, seed=7)
    P = oracle.spai_build(A, n)
    Pd = P.dense()
    for k in range(n):
        J = P.Jind[P.Jptr[k]:P.Jptr[k + 1]]
        e = np.zeros(n)
        e[k] = 1.0
        r = e - D @ Pd[:, k]
        # orthogonality of the residual to the columns A(:, J_k)
        assert np.max(np.abs(D[:, J].T @ r)) <= 1e-12 * np.linalg.norm(D[:, J])
        # m = 0 is feasible, so the optimum has residual <= ||e_k|| = 1
        assert np.linalg.norm(r) <= 1.0 + 1e-14


def test_update_matches_dense_lstsq_and_bounds():
    n = 45
    (A1, D1) = synth.random_sparse(n, 0.08, seed=21)
    # A(l): same pattern, perturbed values
    rng = np.random.default_rng(4)
    Dl = np.where(D1 != 0, D1 * (1 + 0.1 * rng.standard_normal(D1.shape)), 0.0)
    Al = _csr(Dl, D1 != 0)
    P1 = oracle.spai_build(A1, n)
    Q = oracle.spai_update(P1, Al, n)
    Qd = Q.dense()
    for k in range(n):
        J = Q.Jind[Q.Jptr[k]:Q.Jptr[k + 1]]
        q = np.linalg.lstsq(Dl[:, J], D1[:, k], rcond=None)[0]
        assert np.max(np.abs(Qd[J, k] - q)) <= 1e-12 * max(1.0, np.max(np.abs(q)))
        # q = e_k is feasible (k in J_k)
        r_opt = np.linalg.norm(D1[:, k] - Dl @ Qd[:, k])
        r_ek = np.linalg.norm(D1[:, k] - Dl[:, k])
        assert r_opt <= r_ek * (1 + 1e-13) + 1e-15


def test_update_unchanged_parameter_is_identity():
    w = synth.grid_workload((10, 9), "5pt", seed=2, nrhs=1, params=[0.4])
    n = w.n
    A = oracle.assemble(w.terms, oracle.coefficients(0.4, 1.0), n)
    P1 = oracle.spai_build(A, n)
    Q = oracle.spai_update(P1, A, n)
    assert np.max(np.abs(Q.dense() - np.eye(n))) <= 1e-13
    # so the updated preconditioner is the old one
    X = np.random.default_rng(0).standard_normal((n, 3))
    assert np.max(np.abs(Q.apply(X) - P1.apply(X))) <= 1e-12 * np.max(np.abs(P1.apply(X)))


def test_update_scaled_matrix_gives_scaled_identity():
    w = synth.grid_workload((8, 8), "5pt", seed=2, nrhs=1, params=[0.4])
    n = w.n
    coef = oracle.coefficients(0.4, 1.0)
    A1 = oracle.assemble(w.terms, coef, n)
    c = 2.5
    Al = (A1[0], A1[1], c * A1[2])
    P1 = oracle.spai_build(A1, n)
    Q = oracle.spai_update(P1, Al, n)
    assert np.max(np.abs(Q.dense() - np.eye(n) / c)) <= 1e-13


def _appendix1_from_golden(s, p):
    g = json.load(open(os.path.join(GOLDEN, "appendix1.json")))
    n = g["n"]
    D = np.zeros((n, n))

    def val(x):
        if isinstance(x, str):
            return -p if x.startswith("-") else p
        return float(x)

    for b, name in ((0, "A1"), (2, "A2"), (4, "A3")):
        blk = np.array([[val(x) for x in row] for row in g["blocks"][name]["entries"]])
        D[b:b + 2, b:b + 2] = s * np.eye(2) - blk
    a4 = g["blocks"]["A4"]
    k = np.arange(a4["diagonal_from"], a4["diagonal_to"] + 1, dtype=float)
    D[6 + np.arange(k.size), 6 + np.arange(k.size)] = s - k
    return D


@pytest.mark.parametrize("s,p1,pl", [(0.5, 0.3, 0.45), (2.5, 1.0, 1.7)])
def test_appendix1_spai_and_update_are_exact_inverses(s, p1, pl):
    n = 1006
    D1 = _appendix1_from_golden(s, p1)
    Dl = _appendix1_from_golden(s, pl)
    A1 = synth.appendix1_matrix(s, p1)
    Al = synth.appendix1_matrix(s, pl)
    assert np.array_equal(synth.csr_to_dense(A1, n), D1)
    P1 = oracle.spai_build(A1, n)
    assert not P1.status.any()
    # closed form of the 2x2 block inverse [[a, -b], [b, a]]^{-1} = [[a, b], [-b, a]]/(a^2+b^2)
    a, b = s + 1.0, p1
    blk = np.array([[a, b], [-b, a]]) / (a * a + b * b)
    Pd = P1.dense()
    assert np.max(np.abs(Pd[:2, :2] - blk)) <= 1e-15 * 4
    kk = np.arange(1, 1001, dtype=float)
    assert np.max(np.abs(np.diag(Pd)[6:] * (s - kk) - 1.0)) <= 1e-14
    # the inverse has the pattern of A, so P = A^{-1}
    assert np.max(np.abs(D1 @ Pd - np.eye(n))) <= 1e-13
    # update: Q_l = A(l)^{-1} A(1) is block diagonal too, so Q_l P_1 = A(l)^{-1}
    Q = oracle.spai_update(P1, Al, n)
    assert np.max(np.abs(Dl @ Q.dense_product() - np.eye(n))) <= 1e-13
    # and only the first 2x2 block of Q differs from the identity (Appendix I)
    Qd = Q.dense()
    assert np.max(np.abs(Qd[2:, 2:] - np.eye(n - 2))) <= 1e-15


def test_chained_update_second_approach():
    n = 30
    (A1, D1) = synth.random_sparse(n, 0.1, seed=9)
    rng = np.random.default_rng(1)
    D2 = np.where(D1 != 0, D1 * (1 + 0.05 * rng.standard_normal(D1.shape)), 0.0)
    D3 = np.where(D1 != 0, D2 * (1 + 0.05 * rng.standard_normal(D1.shape)), 0.0)
    A2, A3 = _csr(D2, D1 != 0), _csr(D3, D1 != 0)
    P1 = oracle.spai_build(A1, n)
    Q2 = oracle.spai_update_chained(P1, A2, n)
    Q3 = oracle.spai_update_chained(Q2, A3, n)
    # column k of Q3 solves min ||A2(:,k) - A3 q|| on J_k
    Q3d = Q3.dense()
    for k in range(n):
        J = Q3.Jind[Q3.Jptr[k]:Q3.Jptr[k + 1]]
        q = np.linalg.lstsq(D3[:, J], D2[:, k], rcond=None)[0]
        assert np.max(np.abs(Q3d[J, k] - q)) <= 1e-12 * max(1.0, np.max(np.abs(q)))
    # P3 = Q3 Q2 P1
    assert np.allclose(Q3.dense_product(), Q3.dense() @ Q2.dense() @ P1.dense(), rtol=0, atol=1e-14)


def test_singular_column_reported():
    # two identical columns in A(I_k, J_k) -> rank deficient least-squares problem
    D = np.array([[1.0, 1.0, 0.0], [2.0, 2.0, 0.0], [0.0, 0.0, 3.0]])
    A = _csr(D, D != 0)
    P = oracle.spai_build(A, 3)
    assert P.status[0] == 1 and P.status[1] == 1 and P.status[2] == 0


def test_lu_matches_numpy():
    rng = np.random.default_rng(3)
    D = rng.standard_normal((25, 25))
    B = rng.standard_normal((25, 3))
    assert np.allclose(oracle.lu_solve(D, B), np.linalg.solve(D, B), rtol=1e-10, atol=1e-12)


def test_build_with_precomputed_sets_and_column_range():
    """spai_build(sets=..., k0, k1) reuses the given pattern / index sets and fills only
    the requested columns: identical to the full build there, zero elsewhere."""
    A, _ = synth.random_sparse(60, 0.06, seed=4)
    n = 60
    full = oracle.spai_build(A, n, oracle.PATTERN_A2)
    Jptr, Jind = oracle.pattern(A, n, oracle.PATTERN_A2)
    Iptr, Ilist = oracle.index_sets(A, n, Jptr, Jind)
    part = oracle.spai_build(A, n, oracle.PATTERN_A2, k0=10, k1=25, sets=(Jptr, Jind, Iptr, Ilist))
    sl = slice(Jptr[10], Jptr[25])
    assert np.array_equal(part.val[sl], full.val[sl])
    assert not part.val[:Jptr[10]].any() and not part.val[Jptr[25]:].any()


def test_diagonal_update_closed_form_and_invariants():
    """Diagonal Q_l: the least squares over one unknown has the closed form
    q_kk = <A(l)(:,k), a1_k> / ||A(l)(:,k)||^2 (brute force on dense columns here); an
    unchanged matrix gives Q = I, A(l) = c A(1) gives Q = I / c, and for a diagonal A the
    diagonal update equals the full-pattern update."""
    A1, D1 = synth.random_sparse(40, 0.1, seed=6)
    rng = np.random.default_rng(7)
    D2 = D1 + np.where(D1 != 0, 0.05 * rng.standard_normal(D1.shape), 0.0)
    n = 40
    A2 = _csr(D2, D1 != 0)
    P1 = oracle.spai_build(A1, n)
    Q = oracle.spai_update_diagonal(P1, A2, n)
    want = np.einsum("ik,ik->k", D2, D1) / np.einsum("ik,ik->k", D2, D2)
    assert np.allclose(Q.val, want, rtol=1e-14, atol=0)
    assert np.array_equal(Q.Jptr, np.arange(n + 1)) and np.array_equal(Q.Jind, np.arange(n))
    # factored apply: P_l X = Q_l (P_1 X)
    X = rng.standard_normal((n, 3))
    assert np.allclose(Q.apply(X), want[:, None] * P1.apply(X), rtol=1e-14, atol=1e-15)
    assert np.allclose(oracle.spai_update_diagonal(P1, A1, n).val, 1.0, rtol=1e-14)
    A3 = _csr(2.5 * D1, D1 != 0)
    assert np.allclose(oracle.spai_update_diagonal(P1, A3, n).val, 1 / 2.5, rtol=1e-14)
    d = rng.uniform(1.0, 2.0, n)
    Ad1, Ad2 = synth.diag_csr(d), synth.diag_csr(1.3 * d + 0.1)
    Pd = oracle.spai_build(Ad1, n)
    assert np.allclose(oracle.spai_update_diagonal(Pd, Ad2, n).val, oracle.spai_update(Pd, Ad2, n).val,
                       rtol=1e-15)
