"""GPU parity of assembly, index sets, SPAI build / update and the sparse products.

Everything is called through the C ABI (ctypes binding) and compared with the oracle:
bit-exact for patterns, index sets and the assembled values (both sides add the terms in
the same order with separately rounded products and sums); within 1e-10 of the largest
entry of each column for SPAI and update factors; 1e-13 relative for the products.
"""

import numpy as np
import pytest

import oracle
import synth
from gpu_util import column_rel_err, context, dev_csr, export

pytestmark = pytest.mark.gpu

TOL_FACTOR = 1e-10


def _sg():
    import paper_1809_06574_gb300 as sg
    return sg


def _assemble_dev(ctx, terms, n, coefs, host_terms=True):
    import torch
    sg = _sg()
    if host_terms:
        cs = [sg.csr(n, t[0], t[1], t[2]) for t in terms]
    else:
        cs = [dev_csr(t, n) for t in terms]
    aff = sg.spai_affine_create(ctx, cs)
    _, nnz, _, _ = sg.spai_affine_pattern(aff)
    outs = []
    for c in coefs:
        v = torch.empty(max(nnz, 1), dtype=torch.float64, device="cuda:0")
        sg.spai_assemble(ctx, aff, c, v)
        outs.append(v)
    rowptr = np.zeros(n + 1, np.int32)
    colind = np.zeros(max(nnz, 1), np.int32)
    sg.spai_affine_export(ctx, aff, rowptr, colind)
    sg.spai_ctx_sync(ctx)
    return aff, nnz, rowptr, colind[:nnz], outs


# ----------------------------------------------------------------------------- assembly
@pytest.mark.parametrize("case", ["2d-32", "3d-10-7pt", "3d-6-27pt", "random"])
@pytest.mark.parametrize("host_terms", [True, False])
def test_assembly_bit_exact(case, host_terms):
    if case == "2d-32":
        w = synth.plain_2d_32()
        terms = w.terms
    elif case == "3d-10-7pt":
        w = synth.grid3d_7pt(side=10, nparams=2)
        terms = w.terms
    elif case == "3d-6-27pt":
        w = synth.grid3d_27pt(side=6, nparams=2)
        terms = w.terms
    else:
        n0 = 97
        terms = [synth.random_sparse(n0, d, seed=s)[0] for s, d in ((1, 0.05), (2, 0.02), (3, 0.1))]

        class W:
            n = n0
        w = W()
    n = w.n
    coefs = [[1.3, -0.7, 2.25], [0.1, 1.0, 1e-3]]
    with context() as ctx:
        aff, nnz, rpn, cin, outs = _assemble_dev(ctx, terms, n, coefs, host_terms)
        for c, v in zip(coefs, outs):
            ref = oracle.assemble(terms, c, n)
            assert np.array_equal(rpn, ref[0])
            assert np.array_equal(cin, ref[1])
            assert np.array_equal(v.cpu().numpy()[:nnz], ref[2])
        _sg().spai_affine_destroy(aff)


@pytest.mark.parametrize("case", ["2d-32", "3d-10-7pt", "3d-6-27pt"])
def test_assemble_shifted_bit_exact(case):
    """A(p, s) = s^2 M + s D(p) + K(p), D = alpha M + beta K(p) (Sec. 1.1, Sec. 3), formed
    entirely by the library (coefficients and assembly), equals the oracle's assembly of
    the same system bit for bit, for several shifts and parameters."""
    import torch
    sg = _sg()
    w = {"2d-32": synth.plain_2d_32, "3d-10-7pt": lambda: synth.grid3d_7pt(side=10, nparams=2),
         "3d-6-27pt": lambda: synth.grid3d_27pt(side=6, nparams=2)}[case]()
    n = w.n
    with context() as ctx:
        aff = sg.spai_affine_create(ctx, [dev_csr(t, n) for t in w.terms])
        _, nnz, _, _ = sg.spai_affine_pattern(aff)
        for p, s in ((0.1, 1.0), (0.73, 0.5), (1.9, 2.0), (0.0, 0.0)):
            v = torch.empty(max(nnz, 1), dtype=torch.float64, device="cuda:0")
            sg.spai_assemble_shifted(ctx, aff, s, p, w.alpha, w.beta, v)
            sg.spai_ctx_sync(ctx)
            ref = oracle.assemble(w.terms, oracle.coefficients(p, s), n)
            assert np.array_equal(v.cpu().numpy()[:nnz], ref[2]), (p, s)
        with pytest.raises(sg.SpaiError):  # (M, K_0, K_1) needs exactly one parameter
            sg.spai_assemble_shifted(ctx, aff, 1.0, [0.1, 0.2], w.alpha, w.beta, v)
        sg.spai_affine_destroy(aff)


# ----------------------------------------------------------------------------- build
def _build_cases():
    cases = []
    for seed, kind in ((0, oracle.PATTERN_A), (1, oracle.PATTERN_A2)):
        A, _ = synth.random_sparse(150, 0.03, seed=seed)
        cases.append((f"random150-{kind}", A, 150, kind))
    w = synth.plain_2d_32()
    A = oracle.assemble(w.terms, oracle.coefficients(0.1, 1.0), w.n)
    cases.append(("2d-32-A", A, w.n, oracle.PATTERN_A))
    cases.append(("2d-32-A2", A, w.n, oracle.PATTERN_A2))
    w = synth.grid3d_7pt(side=16, nparams=2)
    A = oracle.assemble(w.terms, oracle.coefficients(0.5, 2.0), w.n)
    cases.append(("3d-16-7pt", A, w.n, oracle.PATTERN_A))
    w = synth.grid3d_27pt(side=7, nparams=2)
    A = oracle.assemble(w.terms, oracle.coefficients(0.5, 1.0), w.n)
    cases.append(("3d-7-27pt", A, w.n, oracle.PATTERN_A))
    cases.append(("appendix1", synth.appendix1_matrix(0.5, 0.3), 1006, oracle.PATTERN_A))
    cases.append(("n1", synth.diag_csr([2.5]), 1, oracle.PATTERN_A))
    cases.append(("diag", synth.diag_csr(np.linspace(1, 3, 77)), 77, oracle.PATTERN_A2))
    return cases


@pytest.mark.parametrize("name,A,n,kind", _build_cases(), ids=[c[0] for c in _build_cases()])
def test_build_parity(name, A, n, kind):
    sg = _sg()
    ref = oracle.spai_build(A, n, kind)
    with context() as ctx:
        Ad = dev_csr(A, n)
        pc, st = sg.spai_build(ctx, Ad, kind)
        got = export(ctx, pc)
        sg.spai_pc_destroy(pc)
    assert st == 0
    assert np.array_equal(got["Jptr"], ref.Jptr) and np.array_equal(got["Jind"], ref.Jind)
    assert np.array_equal(got["Iptr"], ref.Iptr) and np.array_equal(got["Ilist"], ref.Ilist)
    assert np.array_equal(got["status"], ref.status)
    assert column_rel_err(ref.Jptr, got["val"], ref.val) <= TOL_FACTOR


@pytest.mark.parametrize("approach", [1, 2])
def test_update_parity(approach):
    sg = _sg()
    w = synth.grid3d_7pt(side=12, nparams=3)
    n = w.n
    As = [oracle.assemble(w.terms, oracle.coefficients(p, 1.0), n) for p in (0.1, 0.4, 0.9)]
    P1 = oracle.spai_build(As[0], n)
    if approach == 1:
        Q2 = oracle.spai_update(P1, As[1], n)
        Q3 = oracle.spai_update(P1, As[2], n)
    else:
        Q2 = oracle.spai_update_chained(P1, As[1], n)
        Q3 = oracle.spai_update_chained(Q2, As[2], n)
    with context() as ctx:
        Ad = [dev_csr(A, n) for A in As]
        pc1, _ = sg.spai_build(ctx, Ad[0])
        pc2, _ = sg.spai_update(ctx, pc1, Ad[1], approach)
        pc3, _ = sg.spai_update(ctx, pc2, Ad[2], approach)
        g2, g3 = export(ctx, pc2), export(ctx, pc3)
        assert g2["depth"] == 1 and g3["depth"] == (1 if approach == 1 else 2)
        # factored apply Q3 (...) P1 X against the oracle's chain
        import torch
        X = np.asfortranarray(np.random.default_rng(0).standard_normal((n, 4)))
        Xd = torch.as_tensor(X.T.copy(), device="cuda:0")  # (4, n) row-major == column-major n x 4
        Yd = torch.empty_like(Xd)
        sg.spai_pc_apply(ctx, pc3, 4, Xd, n, Yd, n)
        sg.spai_ctx_sync(ctx)
        Y = Yd.cpu().numpy().T
        for h in (pc3, pc2, pc1):
            sg.spai_pc_destroy(h)
    assert column_rel_err(Q2.Jptr, g2["val"], Q2.val) <= TOL_FACTOR
    assert column_rel_err(Q3.Jptr, g3["val"], Q3.val) <= TOL_FACTOR
    Yref = Q3.apply(X)
    assert np.max(np.abs(Y - Yref)) <= 1e-12 * np.max(np.abs(Yref))


def test_update_unchanged_parameter_is_identity_on_gpu():
    sg = _sg()
    w = synth.plain_2d_32()
    n = w.n
    A = oracle.assemble(w.terms, oracle.coefficients(0.3, 1.0), n)
    with context() as ctx:
        Ad = dev_csr(A, n)
        pc1, _ = sg.spai_build(ctx, Ad)
        pc2, _ = sg.spai_update(ctx, pc1, Ad)
        g = export(ctx, pc2)
        sg.spai_pc_destroy(pc2)
        sg.spai_pc_destroy(pc1)
    eye = np.zeros_like(g["val"])
    for k in range(n):
        seg = g["Jind"][g["Jptr"][k]:g["Jptr"][k + 1]]
        eye[g["Jptr"][k] + np.nonzero(seg == k)[0]] = 1.0
    assert np.max(np.abs(g["val"] - eye)) <= 1e-13


def test_singular_columns_reported():
    sg = _sg()
    D = np.array([[1.0, 1.0, 0.0], [2.0, 2.0, 0.0], [0.0, 0.0, 3.0]])
    A = synth.dense_to_csr(D, D != 0)
    ref = oracle.spai_build(A, 3)
    with context() as ctx:
        pc, st = sg.spai_build(ctx, dev_csr(A, 3), allow_singular=True)
        g = export(ctx, pc)
        sg.spai_pc_destroy(pc)
        with pytest.raises(sg.SpaiError) as ei:
            sg.spai_build(ctx, dev_csr(A, 3))
        assert "column 0" in str(ei.value)
    assert st == sg.SPAI_ESINGULAR
    assert np.array_equal(g["status"], ref.status)


@pytest.mark.parametrize("bad", ["unsorted", "range", "rowptr"])
def test_malformed_csr_rejected(bad):
    sg = _sg()
    rp = np.array([0, 2, 3, 5], np.int32)
    ci = np.array([0, 1, 1, 0, 2], np.int32)
    va = np.ones(5)
    if bad == "unsorted":
        ci = np.array([1, 0, 1, 0, 2], np.int32)
    elif bad == "range":
        ci = np.array([0, 3, 1, 0, 2], np.int32)
    else:
        rp = np.array([0, 3, 2, 5], np.int32)
    with context() as ctx:
        with pytest.raises(sg.SpaiError) as ei:
            sg.spai_build(ctx, dev_csr((rp, ci, va), 3))
        assert ei.value.status == sg.SPAI_EINVAL
        with pytest.raises(sg.SpaiError):
            sg.spai_affine_create(ctx, [sg.csr(3, rp, ci, va)])


def test_update_rejects_other_pattern():
    sg = _sg()
    A, _ = synth.random_sparse(40, 0.1, seed=1)
    B, _ = synth.random_sparse(40, 0.1, seed=2)
    with context() as ctx:
        pc, _ = sg.spai_build(ctx, dev_csr(A, 40))
        with pytest.raises(sg.SpaiError) as ei:
            sg.spai_update(ctx, pc, dev_csr(B, 40))
        assert ei.value.status == sg.SPAI_EINVAL
        sg.spai_pc_destroy(pc)


@pytest.mark.parametrize("s", [1, 2, 4, 8, 16])
def test_spmm_parity(s):
    import torch
    sg = _sg()
    A, D = synth.random_sparse(333, 0.02, seed=4)
    n = 333
    X = np.random.default_rng(s).standard_normal((n, s))
    ld = n + 5
    Xh = np.zeros((s, ld))
    Xh[:, :n] = X.T
    with context() as ctx:
        Xd = torch.as_tensor(Xh, device="cuda:0")
        Yd = torch.zeros((s, ld), dtype=torch.float64, device="cuda:0")
        sg.spai_spmm(ctx, dev_csr(A, n), s, Xd, ld, Yd, ld)
        sg.spai_ctx_sync(ctx)
        Y = Yd.cpu().numpy()[:, :n].T
    Yref = oracle.spmm(A, X, n)
    assert np.max(np.abs(Y - Yref)) <= 1e-13 * np.max(np.abs(Yref))


def test_memory_budget_refusal():
    sg = _sg()
    w = synth.plain_2d_32()
    A = oracle.assemble(w.terms, oracle.coefficients(0.1, 1.0), w.n)
    with context(mem_budget=4096) as ctx:
        with pytest.raises(sg.SpaiError) as ei:
            sg.spai_build(ctx, dev_csr(A, w.n))
        assert ei.value.status == sg.SPAI_ENOMEM
        assert sg.spai_ctx_mem_in_use(ctx) == 0


@pytest.mark.parametrize("prec", [0, 0x100, 0x200])
def test_diagonal_update_against_oracle(prec):
    """SPAI_UPDATE_DIAGONAL: q_kk of the one-unknown column least squares, bit-exact
    pattern and row sets, values within the FP64 bar (FP32 / BF16 bars otherwise), and
    the factored apply Q_l (P_1 X) against the oracle's."""
    import torch
    sg = _sg()
    w = synth.grid3d_7pt(side=11, nparams=3, seed=2)
    n = w.n
    A1 = oracle.assemble(w.terms, oracle.coefficients(0.2, 1.0), n)
    A2 = oracle.assemble(w.terms, oracle.coefficients(0.7, 1.0), n)
    P1 = oracle.spai_build(A1, n)
    Q = oracle.spai_update_diagonal(P1, A2, n)
    X = np.random.default_rng(1).standard_normal((n, 8))
    with context() as ctx:
        pc1, _ = sg.spai_build(ctx, dev_csr(A1, n), sg.PATTERN_A | prec)
        q, st = sg.spai_update(ctx, pc1, dev_csr(A2, n), sg.UPDATE_FIRST | sg.UPDATE_DIAGONAL | prec)
        g = export(ctx, q)
        Xd = torch.as_tensor(np.ascontiguousarray(X.T), device="cuda:0")
        Yd = torch.zeros((8, n), dtype=torch.float64, device="cuda:0")
        sg.spai_pc_apply(ctx, q, 8, Xd, n, Yd, n)
        sg.spai_ctx_sync(ctx)
        Y = Yd.cpu().numpy().T
        sg.spai_pc_destroy(q)
        sg.spai_pc_destroy(pc1)
    assert st == 0 and g["nnz"] == n and g["depth"] == 1
    assert np.array_equal(g["Jptr"], Q.Jptr) and np.array_equal(g["Jind"], Q.Jind)
    assert np.array_equal(g["Iptr"], Q.Iptr) and np.array_equal(g["Ilist"], Q.Ilist)
    assert not g["status"].any()
    rel = np.max(np.abs(g["val"] - Q.val) / np.abs(Q.val))
    bar = {0: 1e-14, 0x100: 1e-6, 0x200: 2.0 ** -8 + 1e-6}[prec]
    assert rel <= bar, rel
    Yref = Q.apply(X)
    bar_apply = {0: 1e-12, 0x100: 1e-4, 0x200: 2e-2}[prec]
    assert np.max(np.abs(Y - Yref)) <= bar_apply * np.max(np.abs(Yref))


def test_diagonal_update_solve_converges():
    import torch
    sg = _sg()
    w = synth.grid3d_7pt(side=14, nparams=3, seed=4)
    n = w.n
    A1 = oracle.assemble(w.terms, oracle.coefficients(w.params[0], 1.0), n)
    A2 = oracle.assemble(w.terms, oracle.coefficients(w.params[1], 1.0), n)
    Q = oracle.spai_update_diagonal(oracle.spai_build(A1, n), A2, n)
    Xo, io = oracle.block_gmres(oracle.csr_apply(A2, n), Q.apply, w.B, 30, 1e-8, 50)
    with context() as ctx:
        d2 = dev_csr(A2, n)
        pc1, _ = sg.spai_build(ctx, dev_csr(A1, n))
        q, _ = sg.spai_update(ctx, pc1, d2, sg.UPDATE_FIRST | sg.UPDATE_DIAGONAL)
        X = np.zeros((n, w.B.shape[1]), order="F")
        st, info, rel = sg.block_solve(ctx, d2, q, w.B.shape[1], np.asfortranarray(w.B), n, X, n, 30, 1e-8, 50)
        sg.spai_pc_destroy(q)
        sg.spai_pc_destroy(pc1)
    assert info["converged"] and io["converged"]
    assert np.linalg.norm(X - Xo) <= 1e-6 * np.linalg.norm(Xo)


def test_update_across_shifts():
    """Update over the shift (Sec. 2.4 also reuses a factor across expansion points): the
    base is built at (p1, s1) and updated for (p2, s2) with s2 != s1 -- the same column
    least squares against A(p1, s1)'s columns; entries and the solve against the oracle."""
    import torch
    sg = _sg()
    w = synth.grid3d_7pt(side=12, nparams=3, seed=8)
    n = w.n
    A1 = oracle.assemble(w.terms, oracle.coefficients(0.3, 0.5), n)
    A2 = oracle.assemble(w.terms, oracle.coefficients(0.4, 2.0), n)
    Q = oracle.spai_update(oracle.spai_build(A1, n), A2, n)
    Xo, io = oracle.block_gmres(oracle.csr_apply(A2, n), Q.apply, w.B, 30, 1e-8, 50)
    with context() as ctx:
        d1, d2 = dev_csr(A1, n), dev_csr(A2, n)
        pc1, _ = sg.spai_build(ctx, d1)
        q, _ = sg.spai_update(ctx, pc1, d2)
        g = export(ctx, q)
        X = np.zeros((n, w.B.shape[1]), order="F")
        st, info, rel = sg.block_solve(ctx, d2, q, w.B.shape[1], np.asfortranarray(w.B), n, X, n, 30, 1e-8, 50)
        sg.spai_pc_destroy(q)
        sg.spai_pc_destroy(pc1)
    assert column_rel_err(Q.Jptr, g["val"], Q.val) <= TOL_FACTOR
    assert info["converged"] and io["converged"]
    assert np.linalg.norm(X - Xo) <= 1e-6 * np.linalg.norm(Xo)
