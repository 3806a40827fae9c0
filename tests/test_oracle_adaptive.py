"""Pins of the oracle's adaptive SPAI pattern (the MSPAI-style pattern growth the paper's
experiments use, Sec. 3; the column least squares of Sec. 2.2 on each J_k).

Checked against what the definition fixes, independently of the oracle's own code:
closed forms (no growth: a_kk / ||A(:,k)||^2; diagonal A: 1 / a_kk and no growth), a
brute-force re-derivation of every traced step (dense least squares over all n rows,
every column of A as a candidate, the one-dimensional improvement by a dense lstsq), the
exact inverse when the pattern may grow to every column, and the monotone residual."""

import numpy as np
import pytest

import oracle
import synth


def _dense(A, n):
    rp, ci, va = A
    D = np.zeros((n, n))
    for i in range(n):
        D[i, ci[rp[i]:rp[i + 1]]] = va[rp[i]:rp[i + 1]]
    return D


def _random(n, density, seed):
    A, _ = synth.random_sparse(n, density, seed=seed)
    return A


def test_no_growth_is_the_diagonal_closed_form():
    n = 60
    A = _random(n, 0.08, 3)
    P = oracle.spai_build_adaptive(A, n, max_steps=0)
    D = _dense(A, n)
    assert np.array_equal(np.diff(P.Jptr), np.ones(n, np.int32))
    assert np.array_equal(P.Jind, np.arange(n))
    ref = np.diag(D) / np.sum(D * D, axis=0)
    assert np.max(np.abs(P.val - ref)) <= 1e-14 * np.max(np.abs(ref))


def test_diagonal_matrix_needs_no_growth():
    n = 40
    d = np.linspace(0.5, 3.0, n)
    A = (np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), d)
    P = oracle.spai_build_adaptive(A, n, eps=1e-12)
    assert np.array_equal(P.Jind, np.arange(n))
    assert np.max(np.abs(P.val - 1.0 / d)) <= 1e-15


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_every_step_against_brute_force(seed):
    """Each traced step re-derived with dense algebra over all n rows: the residual
    norm, the candidate set (every column of A outside J_k with a nonzero in a row of
    I_k), each improvement rho_j = min_alpha ||r - alpha A(:,j)||^2, and the choice."""
    n = 45
    A = _random(n, 0.07, seed)
    D = _dense(A, n)
    trace = []
    oracle.spai_adaptive_pattern(A, n, eps=1e-6, max_steps=3, max_new=3, trace=trace)
    assert len(trace) > n  # most columns take at least one step
    for (k, step, J, I, rr, cand, rho, chosen) in trace:
        e = np.zeros(n)
        e[k] = 1.0
        m = np.linalg.lstsq(D[:, J], e, rcond=None)[0]
        r = e - D[:, J] @ m
        assert abs(r @ r - rr) <= 1e-10 * max(rr, 1e-300)
        # I_k: {k} and the rows of the columns in J_k
        assert I == sorted({k} | set(np.nonzero(D[:, J].any(axis=1))[0].tolist()))
        want = sorted(j for j in range(n) if j not in J and D[I, j].any())
        assert cand == want
        for j, x in zip(cand, rho):
            a = D[:, j]
            alpha = np.linalg.lstsq(a[:, None], r, rcond=None)[0][0]
            bf = np.sum((r - alpha * a) ** 2)
            assert abs(x - bf) <= 1e-10 * rr
        keys = [oracle._adaptive_key(x, rr) for x in rho]
        kmean = oracle._adaptive_key(sum(rho) / len(rho), rr)
        pick = [j for _, j in sorted((q, j) for q, j in zip(keys, cand) if q <= kmean)][:3]
        assert chosen == pick


def test_full_growth_gives_the_inverse():
    """A dense 8 x 8 matrix: every column is a candidate, so with enough steps and no
    tolerance J_k grows to all columns and P = A^{-1} (unique least squares)."""
    rng = np.random.default_rng(4)
    n = 8
    D = rng.standard_normal((n, n)) + 4 * np.eye(n)
    rp = np.arange(0, n * n + 1, n, dtype=np.int32)
    ci = np.tile(np.arange(n, dtype=np.int32), n)
    A = (rp, ci, D.reshape(-1))
    P = oracle.spai_build_adaptive(A, n, eps=0.0, max_steps=7, max_new=1)
    assert np.array_equal(np.diff(P.Jptr), np.full(n, n))
    assert np.max(np.abs(D @ P.dense() - np.eye(n))) <= 1e-12


def test_residual_never_grows_and_stops_for_a_reason():
    w = synth.grid_workload((11, 11), "5pt", seed=5, nrhs=4, params=[0.4])
    n = w.n
    A = oracle.assemble(w.terms, oracle.coefficients(0.4, 1.0), n)
    trace = []
    eps = 1e-3
    Jptr, Jind = oracle.spai_adaptive_pattern(A, n, eps=eps, max_steps=4, max_new=4, trace=trace)
    last = {}
    for (k, step, J, I, rr, cand, rho, chosen) in trace:
        if k in last:
            assert rr <= last[k] * (1 + 1e-12)
        last[k] = rr
        assert len(I) <= oracle.ADAPTIVE_MAX_ROWS
    P = oracle.spai_build(A, n, oracle.PATTERN_A, sets=(Jptr, Jind) + oracle.index_sets(A, n, Jptr, Jind))
    D = _dense(A, n)
    R = np.eye(n) - D @ P.dense()
    col = np.linalg.norm(R, axis=0)
    full = 1 + 4 * 4
    for k in range(n):
        # a column that stopped before its step limit met the tolerance (the 5-point grid
        # always has candidates and stays far below the row cap here)
        if Jptr[k + 1] - Jptr[k] < full and not any(t[0] == k and t[1] == 3 for t in trace):
            assert col[k] <= eps * (1 + 1e-9), k


def test_row_limit_undoes_the_step_that_would_exceed_it():
    """With a tight row limit the growth stops at the last step that kept |I_k| within it:
    every final pattern's row set fits, and adding the chosen columns of the next traced
    step would not have (checked against the dense pattern)."""
    w = synth.grid3d_7pt(side=6, nparams=2, seed=5)
    n = w.n
    A = oracle.assemble(w.terms, oracle.coefficients(0.5, 2.0), n)
    D = _dense(A, n)
    limit = 30
    trace = []
    Jptr, Jind = oracle.spai_adaptive_pattern(A, n, eps=1e-10, max_steps=6, max_new=5, max_rows=limit, trace=trace)
    last = {}
    for t in trace:
        last[t[0]] = t
    stopped = 0
    for k in range(n):
        J = Jind[Jptr[k]:Jptr[k + 1]].tolist()
        rows = {k} | set(np.nonzero(D[:, J].any(axis=1))[0].tolist())
        assert len(rows) <= limit
        t = last.get(k)
        if t is not None and t[2] == J and t[7]:  # the last traced step chose columns but J did not grow
            grown = {k} | set(np.nonzero(D[:, sorted(J + t[7])].any(axis=1))[0].tolist())
            assert len(grown) > limit
            stopped += 1
    assert stopped > 0  # the limit binds for some columns in this case


def test_every_candidate_is_scored_however_many():
    """A bordered matrix (row 0 full): column 0's first row set holds row 0, so every other
    column (1,199 of them, more than any fixed buffer of 1,024) is a candidate.  The rule of
    the adaptive pattern has no cap on candidates: all of them are scored, the choice is the
    brute-force one over all of them, and the pattern grows."""
    n = 1200
    A, D = synth.bordered_sparse(n, 0.002, seed=7)
    trace = []
    Jptr, Jind = oracle.spai_adaptive_pattern(A, n, eps=1e-10, max_steps=2, max_new=3, k0=0, k1=1, trace=trace)
    first = [t for t in trace if t[0] == 0 and t[1] == 0]
    assert first
    (k, step, J, I, rr, cand, rho, chosen) = first[0]
    assert cand == [j for j in range(1, n)]  # all of them
    e = np.zeros(n)
    e[0] = 1.0
    m = np.linalg.lstsq(D[:, J], e, rcond=None)[0]
    r = e - D[:, J] @ m
    assert abs(r @ r - rr) <= 1e-10 * rr
    cn = np.sum(D * D, axis=0)
    bf = r @ r - (r @ D) ** 2 / cn  # one-column improvement of every column at once
    assert np.max(np.abs(np.array(rho) - bf[1:])) <= 1e-10 * rr
    keys = [oracle._adaptive_key(x, rr) for x in rho]
    kmean = oracle._adaptive_key(sum(rho) / len(rho), rr)
    assert chosen == [j for _, j in sorted((q, j) for q, j in zip(keys, cand) if q <= kmean)][:3]
    assert len(chosen) == 3 and Jptr[1] - Jptr[0] > 1
