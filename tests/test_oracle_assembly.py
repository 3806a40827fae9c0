"""Pins of the oracle's assembly, transposition, patterns and index sets (CPU only).

Each check compares the oracle with something other than itself: dense brute force,
the paper's unexpanded formula for A(p, s), or the closed-form stencil sizes.
"""

import numpy as np
import pytest

import oracle
import synth


def _dense(csr, n):
    return synth.csr_to_dense(csr, n)


def _pattern_dense(csr, n):
    P = np.zeros((n, n), dtype=bool)
    rp, ci, _ = csr
    for i in range(n):
        P[i, ci[rp[i]:rp[i + 1]]] = True
    return P


def test_union_assembly_matches_dense_sum_bit_exact():
    w = synth.grid_workload((7, 5), "5pt", seed=3, nrhs=2, params=[0.3])
    n = w.n
    coef = oracle.coefficients(0.37, 1.3)
    A = oracle.assemble(w.terms, coef, n)
    # dense sum in the same order (numpy rounds each product and each sum separately)
    D = np.zeros((n, n))
    for c, t in zip(coef, w.terms):
        D = D + c * _dense(t, n)
    pat = np.zeros((n, n), dtype=bool)
    for t in w.terms:
        pat |= _pattern_dense(t, n)
    assert np.array_equal(_pattern_dense(A, n), pat)
    assert np.array_equal(_dense(A, n)[pat], D[pat])


def test_union_keeps_structural_zeros():
    # two terms that cancel exactly on one entry: the entry stays in the pattern
    n = 3
    T0 = synth.dense_to_csr(np.array([[1.0, 2.0, 0], [0, 1.0, 0], [0, 0, 1.0]]))
    T1 = synth.dense_to_csr(np.array([[0, -2.0, 0], [0, 0, 0], [5.0, 0, 0]]))
    A = oracle.assemble([T0, T1], [1.0, 1.0], n)
    assert list(A[0]) == [0, 2, 3, 5]
    assert list(A[1]) == [0, 1, 1, 0, 2]
    assert A[2][1] == 0.0


@pytest.mark.parametrize("p,s", [(0.1, 1.0), (0.73, 0.5), (1.0, 2.0)])
def test_coefficients_match_unexpanded_formula(p, s):
    # A(p, s) = s^2 M + s D + K,  D = 0.05 M + 0.01 K,  K = K0 + p K1 (Sec. 1.1 / Sec. 3)
    w = synth.grid_workload((4, 3, 2), "7pt", seed=1, nrhs=1, params=[p])
    n = w.n
    M, K0, K1 = (_dense(t, n) for t in w.terms)
    K = K0 + p * K1
    D = 0.05 * M + 0.01 * K
    ref = s * s * M + s * D + K
    A = _dense(oracle.assemble(w.terms, oracle.coefficients(p, s), n), n)
    assert np.max(np.abs(A - ref)) <= 1e-14 * np.max(np.abs(ref))


def test_csr_to_csc_is_transpose():
    (A, D) = synth.random_sparse(23, 0.2, seed=5)
    n = 23
    cp, ri, cv = oracle.csr_to_csc(A, n)
    T = np.zeros((n, n))
    for k in range(n):
        assert np.all(np.diff(ri[cp[k]:cp[k + 1]]) > 0)
        T[ri[cp[k]:cp[k + 1]], k] = cv[cp[k]:cp[k + 1]]
    assert np.array_equal(T, D)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_patterns_and_index_sets_brute_force(seed):
    n = 31
    (A, D) = synth.random_sparse(n, 0.08, seed=seed)
    S = D != 0
    for kind in (oracle.PATTERN_A, oracle.PATTERN_A2):
        Jptr, Jind = oracle.pattern(A, n, kind)
        Sj = S if kind == oracle.PATTERN_A else (S.astype(int) @ S.astype(int)) > 0
        Iptr, Ilist = oracle.index_sets(A, n, Jptr, Jind)
        for k in range(n):
            J = Jind[Jptr[k]:Jptr[k + 1]]
            assert list(J) == list(np.nonzero(Sj[:, k])[0])
            I = Ilist[Iptr[k]:Iptr[k + 1]]
            ref = np.nonzero(S[:, J].any(axis=1))[0]
            assert list(I) == list(ref)


@pytest.mark.parametrize("dims,kind,kindp,nJ,nI", [
    ((9, 9), "5pt", oracle.PATTERN_A, 5, 13),
    ((7, 7, 7), "7pt", oracle.PATTERN_A, 7, 25),
    ((9, 9), "5pt", oracle.PATTERN_A2, 13, 25),
    ((6, 6, 6), "27pt", oracle.PATTERN_A, 27, 125),
])
def test_interior_sizes_closed_form(dims, kind, kindp, nJ, nI):
    # interior column of a radius-1 stencil: |J| = stencil size; |I| = points within
    # radius 2 (l1-ball for 5/7-point, l_inf box 5^3 for 27-point)
    w = synth.grid_workload(dims, kind, seed=0, nrhs=1, params=[0.5])
    n = w.n
    A = oracle.assemble(w.terms, oracle.coefficients(0.5, 1.0), n)
    Jptr, Jind = oracle.pattern(A, n, kindp)
    Iptr, Ilist = oracle.index_sets(A, n, Jptr, Jind)
    c = tuple(d // 2 for d in dims)
    k = c[0] + dims[0] * (c[1] + (dims[1] * c[2] if len(dims) == 3 else 0))
    assert Jptr[k + 1] - Jptr[k] == nJ
    assert Iptr[k + 1] - Iptr[k] == nI


def test_stencil_nnz_counts():
    # nnz of the 2D 32^2 5-point and 3D 64^3 7-point grids
    r, c, v = synth.stencil_csr((32, 32), "5pt", 4.0, -1.0)
    assert len(c) == 4992
    r, c, v = synth.stencil_csr((16, 16, 16), "7pt", 6.0, -1.0)
    assert len(c) == 7 * 16 ** 3 - 6 * 16 ** 2
    r, c, v = synth.stencil_csr((5, 5, 5), "27pt", 26.0, -1.0)
    assert len(c) == (3 * 5 - 2) ** 3
