"""Pins of the oracle's block GCRO with a recycled outer space (the paper's solver, Sec. 3,
in block form; the outer space carried along a sequence of systems, Sec. 1.3).

Checked against what the method's definition fixes, independently of the oracle's code:
without a recycled space it is block GMRES (the same iterates); a recycled space that holds
the solution gives it with no Arnoldi step; every cycle's iterate is the brute-force
minimiser of the residual over X~0 + span([U, K_j]), K_j the block Krylov space of the
operator projected against C = AP U, built here from explicit powers; converged solutions
match a dense solve; and a recycled space from a neighbouring system saves iterations."""

import numpy as np
import pytest

import oracle
import synth


def _system(side=7, p=0.3, s=4, seed=3):
    w = synth.grid_workload((side, side, side), "7pt", seed=seed, nrhs=s, params=[p, p + 0.05, p + 0.1])
    n = w.n
    As = [oracle.assemble(w.terms, oracle.coefficients(q, 1.0), n) for q in w.params]
    return w, n, As


def _dense(A, n):
    return synth.csr_to_dense(A, n)


def test_without_recycled_space_it_is_block_gmres():
    w, n, As = _system()
    P = oracle.spai_build(As[0], n)
    Xg, ig = oracle.block_gmres(oracle.csr_apply(As[0], n), P.apply, w.B, 8, 1e-10, 10)
    Xc, ic, _ = oracle.block_gcro(oracle.csr_apply(As[0], n), P.apply, w.B, 8, 1e-10, 10)
    assert ic["iterations"] == ig["iterations"] and ic["cycles"] == ig["cycles"]
    assert np.max(np.abs(Xc - Xg)) <= 1e-13 * np.max(np.abs(Xg))


def test_a_recycled_space_holding_the_solution_needs_no_arnoldi_step():
    w, n, As = _system()
    P = oracle.spai_build(As[0], n)
    D = _dense(As[0], n)
    Pd = P.dense()
    Xt = np.linalg.solve(D @ Pd, w.B)  # the preconditioned-space solution
    rng = np.random.default_rng(0)
    U = np.hstack([rng.standard_normal((n, 3)), Xt, rng.standard_normal((n, 2))])
    X, info, _ = oracle.block_gcro(oracle.csr_apply(As[0], n), P.apply, w.B, 8, 1e-10, 10, U=U)
    assert info["iterations"] == 0 and info["converged"]
    assert np.max(np.abs(X - np.linalg.solve(D, w.B))) <= 1e-9 * np.max(np.abs(X))


@pytest.mark.parametrize("steps", [1, 2, 4])
def test_each_iterate_is_the_brute_force_minimiser(steps):
    """One cycle of `steps` block Arnoldi steps: X~ minimises ||B - AP X~|| over
    X~0 + span([U, R0, Ap R0, ..., Ap^(steps-1) R0]) with Ap = (I - C C^T) AP (the iterate
    and the minimiser are computed here from explicit matrices)."""
    w, n, As = _system(side=6, s=3)
    P = oracle.spai_build(As[0], n)
    D = _dense(As[0], n) @ P.dense()  # AP
    rng = np.random.default_rng(5)
    U0 = rng.standard_normal((n, 6))
    B = w.B
    X, info, _ = oracle.block_gcro(lambda Y: np.asarray(_dense(As[0], n) @ Y), P.apply, B, steps, 0.0, 1, U=U0)
    assert info["iterations"] == steps and info["cycles"] == 1
    # the same space, explicitly
    C, _ = np.linalg.qr(D @ U0)
    X0t = U0 @ np.linalg.lstsq(D @ U0, B, rcond=None)[0]
    R0 = B - D @ X0t
    Ap = D - C @ (C.T @ D)
    K = [R0]
    for _ in range(steps - 1):
        K.append(Ap @ K[-1])
    S = np.hstack([U0] + K)
    Y = np.linalg.lstsq(D @ S, R0, rcond=None)[0]
    Xt = X0t + S @ Y
    Xref = P.dense() @ Xt
    assert np.linalg.norm(X - Xref) <= 1e-8 * np.linalg.norm(Xref)
    r_gcro = np.linalg.norm(B - _dense(As[0], n) @ X)
    r_ref = np.linalg.norm(B - D @ Xt)
    assert r_gcro <= r_ref * (1 + 1e-9) + 1e-13


def test_converged_solution_matches_a_dense_solve_and_recycling_saves_iterations():
    w, n, As = _system(side=8, s=4)
    D = [_dense(A, n) for A in As]
    P1 = oracle.spai_build(As[0], n)
    X1, i1, U = oracle.block_gcro(oracle.csr_apply(As[0], n), P1.apply, w.B, 30, 1e-10, 20, kmax=8)
    assert i1["converged"] and U.shape == (n, 4)  # this solve's X~ only
    assert np.linalg.norm(X1 - np.linalg.solve(D[0], w.B)) <= 1e-8 * np.linalg.norm(X1)
    # the next system of the sequence: the update of P_1 (Table 1), the recycled space
    Q2 = oracle.spai_update(P1, As[1], n)
    X2, i2, U2 = oracle.block_gcro(oracle.csr_apply(As[1], n), Q2.apply, w.B, 30, 1e-10, 20, U=U, kmax=8)
    X2g, i2g = oracle.block_gmres(oracle.csr_apply(As[1], n), Q2.apply, w.B, 30, 1e-10, 20)
    assert i2["converged"]
    assert np.linalg.norm(X2 - np.linalg.solve(D[1], w.B)) <= 1e-8 * np.linalg.norm(X2)
    assert i2["iterations"] < i2g["iterations"]
    # the recycled space keeps the newest kmax columns: the last block is this solve's X~
    assert U2.shape == (n, 8)
    Xt2 = np.linalg.solve(D[1] @ Q2.dense_product(), w.B)
    assert np.linalg.norm(U2[:, -4:] - Xt2) <= 1e-8 * np.linalg.norm(Xt2)


def test_dependent_recycled_columns_are_dropped():
    """A recycled space with repeated columns: the thin QR of its image deflates the copies
    (zero columns), and the solve is unchanged."""
    w, n, As = _system(side=6, s=2)
    P = oracle.spai_build(As[0], n)
    rng = np.random.default_rng(2)
    U = rng.standard_normal((n, 4))
    Ud = np.hstack([U, U[:, :2]])
    Xa, ia, _ = oracle.block_gcro(oracle.csr_apply(As[0], n), P.apply, w.B, 10, 1e-10, 10, U=U)
    Xb, ib, _ = oracle.block_gcro(oracle.csr_apply(As[0], n), P.apply, w.B, 10, 1e-10, 10, U=Ud)
    assert ia["iterations"] == ib["iterations"]
    assert np.linalg.norm(Xa - Xb) <= 1e-9 * np.linalg.norm(Xa)
