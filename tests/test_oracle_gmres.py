"""Pins of the oracle's right-preconditioned block GMRES (CPU only).

* one right-hand side, one cycle of k steps == SciPy's GMRES on the operator A P
  (right preconditioning: A P x~ = b, x = P x~), a separate implementation;
* a block cycle of j steps == brute-force minimisation of every column's residual over
  the explicitly built block Krylov space span{R0, (AP)R0, ..., (AP)^{j-1}R0};
* n <= m*s: one cycle reaches the dense LU solution;
* least-squares estimates are non-increasing inside a cycle and match the true residual;
* converged solves satisfy ||b_i - A x_i|| <= tol ||b_i|| and agree with a dense solve.
"""

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
import synth


def _system(n=64, seed=0, density=0.06):
    (A, D) = synth.random_sparse(n, density, seed=seed)
    return A, D


def test_single_rhs_one_cycle_equals_scipy_gmres_right_preconditioned():
    n = 64
    A, D = _system(n, 3)
    P = oracle.spai_build(A, n)
    Pd = P.dense()
    b = np.random.default_rng(1).standard_normal((n, 1))
    k = 9
    X, info = oracle.block_gmres(oracle.csr_apply(A, n), P.apply, b, restart=k, tol=0.0,
                                 max_cycles=1)
    assert info["iterations"] == k
    op = spla.LinearOperator((n, n), matvec=lambda v: D @ (Pd @ v), dtype=float)
    xt, _ = spla.gmres(op, b[:, 0], rtol=1e-300, atol=0.0, restart=k, maxiter=1)
    x_ref = Pd @ xt
    assert np.linalg.norm(X[:, 0] - x_ref) <= 1e-9 * np.linalg.norm(x_ref)


@pytest.mark.parametrize("s,j", [(2, 3), (4, 2), (3, 4)])
def test_block_cycle_equals_brute_force_krylov_minimiser(s, j):
    n = 50
    A, D = _system(n, 5)
    P = oracle.spai_build(A, n)
    Pd = P.dense()
    B = np.random.default_rng(2).standard_normal((n, s))
    X, info = oracle.block_gmres(oracle.csr_apply(A, n), P.apply, B, restart=j, tol=0.0,
                                 max_cycles=1)
    # explicit block Krylov space of A P from R0 = B (X0 = 0), orthonormalised for stability
    blocks = [B]
    for _ in range(j - 1):
        blocks.append(D @ (Pd @ blocks[-1]))
    K, _ = np.linalg.qr(np.hstack(blocks))
    C = np.linalg.lstsq(D @ Pd @ K, B, rcond=None)[0]
    X_ref = Pd @ K @ C
    assert np.linalg.norm(X - X_ref) <= 1e-9 * np.linalg.norm(X_ref)


def test_full_space_in_one_cycle_gives_exact_solution():
    n, s, m = 24, 4, 6          # n <= m * s
    A, D = _system(n, 8, density=0.2)
    P = oracle.spai_build(A, n)
    B = np.random.default_rng(3).standard_normal((n, s))
    X, info = oracle.block_gmres(oracle.csr_apply(A, n), P.apply, B, restart=m, tol=1e-12,
                                 max_cycles=1)
    X_ref = oracle.lu_solve(D, B)
    assert info["cycles"] == 1
    assert np.linalg.norm(X - X_ref) <= 1e-10 * np.linalg.norm(X_ref)


def test_estimates_monotone_and_match_true_residual():
    w = synth.grid_workload((20, 20), "5pt", seed=0, nrhs=4, params=[0.2])
    n = w.n
    A = oracle.assemble(w.terms, oracle.coefficients(0.2, 1.0), n)
    P = oracle.spai_build(A, n)
    X, info = oracle.block_gmres(oracle.csr_apply(A, n), P.apply, w.B, restart=15, tol=0.0,
                                 max_cycles=1, history=True)
    est = np.array(info["estimates"])
    assert np.all(np.diff(est, axis=0) <= 1e-12 * est[0])
    true = np.linalg.norm(w.B - oracle.spmm(A, X, n), axis=0)
    assert np.allclose(est[-1], true, rtol=1e-6, atol=1e-12 * np.linalg.norm(w.B, axis=0).max())


@pytest.mark.parametrize("p", [0.1, 0.3, 0.5])
def test_plain_2d_converges_and_matches_dense_solve(p):
    w = synth.plain_2d_32()
    n = w.n
    A = oracle.assemble(w.terms, oracle.coefficients(p, 1.0), n)
    P = oracle.spai_build(A, n)
    X, info = oracle.block_gmres(oracle.csr_apply(A, n), P.apply, w.B, restart=30, tol=1e-8,
                                 max_cycles=50)
    assert info["converged"]
    rel = np.linalg.norm(w.B - oracle.spmm(A, X, n), axis=0) / np.linalg.norm(w.B, axis=0)
    assert np.all(rel <= 1e-8)
    Ad = sp.csr_matrix((A[2], A[1], A[0]), shape=(n, n))
    X_ref = spla.spsolve(Ad.tocsc(), w.B)
    assert np.linalg.norm(X - X_ref) <= 1e-6 * np.linalg.norm(X_ref)


def test_update_preconditioner_in_solve():
    w = synth.plain_2d_32()
    n = w.n
    A1 = oracle.assemble(w.terms, oracle.coefficients(0.1, 1.0), n)
    Al = oracle.assemble(w.terms, oracle.coefficients(0.5, 1.0), n)
    P1 = oracle.spai_build(A1, n)
    Q = oracle.spai_update(P1, Al, n)
    X, info = oracle.block_gmres(oracle.csr_apply(Al, n), Q.apply, w.B, restart=30, tol=1e-8,
                                 max_cycles=50)
    assert info["converged"]
    X0, info0 = oracle.block_gmres(oracle.csr_apply(Al, n), None, w.B, restart=30, tol=1e-8,
                                   max_cycles=50)
    assert info0["converged"]
    # the update preconditioner is a real preconditioner: fewer iterations than none
    assert info["iterations"] < info0["iterations"]


def test_zero_rhs_column_and_restarts():
    n = 40
    A, D = _system(n, 12)
    B = np.random.default_rng(0).standard_normal((n, 3))
    B[:, 1] = 0.0
    X, info = oracle.block_gmres(oracle.csr_apply(A, n), None, B, restart=3, tol=1e-10,
                                 max_cycles=200)
    assert info["converged"] and info["cycles"] > 1
    assert np.all(X[:, 1] == 0.0)
    assert np.allclose(X, np.linalg.solve(D, B), rtol=0, atol=1e-8 * np.abs(X).max())


def test_paper_quoted_savings_from_printed_tables():
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))
    block = 1 - g["table3_block_gcro_total_seconds"] / g["table3_gcro_total_seconds"]
    upd = 1 - sum(g["table4_update_minutes"]) / sum(g["table4_spai_minutes"])
    both = 1 - sum(g["table5_block_gcro_update_minutes"]) / sum(g["table5_block_gcro_spai_minutes"])
    assert abs(block - g["quoted_block_saving"]) < 0.01
    assert abs(upd - g["quoted_update_saving"]) < 0.02
    assert abs(both - g["quoted_block_plus_update_saving"]) < 0.02


@pytest.mark.parametrize("scale", [1.0, 1e-6, 1e-11, 1e-13])
def test_cgs2_coefficients_give_the_deflation_scale(scale):
    """The deflation scale of the new block's QR is each column's norm before the two block
    CGS passes (``wn`` in the oracle's Arnoldi step).  Against a basis whose columns are
    orthonormal or zero (deflated), W0 = V (H1 + H2) + W2 with W2 orthogonal to V, so
    ||W0(:, c)||^2 = ||(H1 + H2)(:, c)||^2 + ||W2(:, c)||^2: the GPU's first Cholesky-QR pass
    forms the scale this way from quantities it already has.  Checked on blocks from fully
    independent down to numerically dependent (scale = the size of the part outside V),
    and the deflation decision of ``_block_qr``'s threshold is the same with either scale."""
    rng = np.random.default_rng(7)
    n, s, nb = 500, 8, 6
    V, _ = np.linalg.qr(rng.standard_normal((n, nb * s)))
    V[:, [5, 19, 40]] = 0.0  # deflated basis columns
    W0 = V @ rng.standard_normal((nb * s, s)) + scale * rng.standard_normal((n, s))
    W0[:, 2] *= 1e3  # columns of different sizes
    wn2 = np.sum(W0 * W0, axis=0)
    H1 = V.T @ W0
    W1 = W0 - V @ H1
    H2 = V.T @ W1
    W2 = W1 - V @ H2
    est = np.sum((H1 + H2) ** 2, axis=0) + np.sum(W2 * W2, axis=0)
    assert np.max(np.abs(est - wn2) / wn2) <= 1e-13
    # the deflation threshold (|R_kk| <= 1e-12 * scale) decides the same with either scale
    _, R = np.linalg.qr(W2)
    d = np.abs(np.diag(R))
    assert np.array_equal(d <= oracle.DEFLATE_REL * np.sqrt(wn2), d <= oracle.DEFLATE_REL * np.sqrt(est))
