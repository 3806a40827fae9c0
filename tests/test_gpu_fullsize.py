"""Parity at the benchmark's full size (3D 64^3 7-point grid, n = 262,144, 8 RHS), through
the same C ABI calls and launch configuration that bench.py times.

The oracle is fast enough here to compare every index set and every SPAI / update
entry, and to run one full block-GMRES(50) solve.
"""

import numpy as np
import pytest

import oracle
import synth
from gpu_util import column_rel_err_vec, context, export

pytestmark = pytest.mark.gpu


def test_fullsize_sweep_pieces():
    import torch
    import paper_1809_06574_gb300 as sg
    w = synth.grid3d_7pt(side=64, nparams=20)
    n = w.n
    s_shift = 0.5
    p1, p2 = w.params[0], w.params[7]
    with context() as ctx:
        d_terms = [tuple(torch.as_tensor(np.ascontiguousarray(a), device="cuda:0") for a in t)
                   for t in w.terms]
        aff = sg.spai_affine_create(ctx, [sg.csr(n, *t) for t in d_terms])
        _, nnz, rp, ci = sg.spai_affine_pattern(aff)
        assert nnz == 1810432
        v1 = torch.empty(nnz, dtype=torch.float64, device="cuda:0")
        v2 = torch.empty(nnz, dtype=torch.float64, device="cuda:0")
        sg.spai_assemble_shifted(ctx, aff, s_shift, p1, w.alpha, w.beta, v1)
        sg.spai_assemble_shifted(ctx, aff, s_shift, p2, w.alpha, w.beta, v2)
        A1d, A2d = sg.csr(n, rp, ci, v1, nnz), sg.csr(n, rp, ci, v2, nnz)
        pc1, _ = sg.spai_build(ctx, A1d, sg.PATTERN_A)
        pc2, _ = sg.spai_update(ctx, pc1, A2d, sg.UPDATE_FIRST)
        g1, g2 = export(ctx, pc1), export(ctx, pc2)
        X = np.zeros((n, 8), order="F")
        st, info, rel = sg.block_solve(ctx, A2d, pc2, 8, np.asfortranarray(w.B), n, X, n, 50, 1e-8, 50)
        v2h = v2.cpu().numpy()
        sg.spai_pc_destroy(pc2)
        sg.spai_pc_destroy(pc1)
        sg.spai_affine_destroy(aff)
    A1 = oracle.assemble(w.terms, oracle.coefficients(p1, s_shift), n)
    A2 = oracle.assemble(w.terms, oracle.coefficients(p2, s_shift), n)
    assert np.array_equal(v2h, A2[2])
    P1 = oracle.spai_build(A1, n)
    Q2 = oracle.spai_update(P1, A2, n)
    for g, ref in ((g1, P1), (g2, Q2)):
        assert np.array_equal(g["Jptr"], ref.Jptr) and np.array_equal(g["Jind"], ref.Jind)
        assert np.array_equal(g["Iptr"], ref.Iptr) and np.array_equal(g["Ilist"], ref.Ilist)
        assert not g["status"].any()
        assert column_rel_err_vec(ref.Jptr, g["val"], ref.val) <= 1e-10
    assert info["converged"]
    true_rel = np.linalg.norm(w.B - oracle.spmm(A2, X, n), axis=0) / np.linalg.norm(w.B, axis=0)
    assert np.all(true_rel <= 1e-8)
    Xo, io = oracle.block_gmres(oracle.csr_apply(A2, n), Q2.apply, w.B, 50, 1e-8, 50)
    assert np.linalg.norm(X - Xo) <= 1e-6 * np.linalg.norm(Xo)


def _sample_ranges(n, width=1500):
    """Column ranges spanning the grid: the first and last planes (boundary columns) and
    two interior stretches."""
    return [(0, width), (n // 3, n // 3 + width), (n // 2 + 17, n // 2 + 17 + width), (n - width, n)]


def test_fullsize_27pt_128_bf16_build_update_solve():
    """The large workload: 3D 128^3 27-point grid (n = 2,097,152, nnz = 55,742,968), SPAI in
    FP32 stored as BF16, updated for a second parameter, FP64 block GMRES with 16 RHS.

    The oracle runs the whole pattern analysis (every J_k and I_k is compared) and the
    column least squares on sampled column ranges; the FP64 build is compared on the same
    columns at the FP64 bar.  The solve is checked by its true residual, recomputed on the
    host in FP64 (a property that holds at any size)."""
    import torch
    import paper_1809_06574_gb300 as sg
    w = synth.grid3d_27pt(side=128, nparams=50)
    n = w.n
    p1, p2 = w.params[0], w.params[1]
    ranges = _sample_ranges(n)
    with context() as ctx:
        d_terms = [tuple(torch.as_tensor(np.ascontiguousarray(a), device="cuda:0") for a in t)
                   for t in w.terms]
        aff = sg.spai_affine_create(ctx, [sg.csr(n, *t) for t in d_terms])
        _, nnz, rp, ci = sg.spai_affine_pattern(aff)
        assert nnz == 55742968
        v1 = torch.empty(nnz, dtype=torch.float64, device="cuda:0")
        v2 = torch.empty(nnz, dtype=torch.float64, device="cuda:0")
        sg.spai_assemble_shifted(ctx, aff, 1.0, p1, w.alpha, w.beta, v1)
        sg.spai_assemble_shifted(ctx, aff, 1.0, p2, w.alpha, w.beta, v2)
        A1d, A2d = sg.csr(n, rp, ci, v1, nnz), sg.csr(n, rp, ci, v2, nnz)
        pc64, _ = sg.spai_build(ctx, A1d, sg.PATTERN_A)
        g64 = export(ctx, pc64)
        sg.spai_pc_destroy(pc64)
        pc1, _ = sg.spai_build(ctx, A1d, sg.PATTERN_A | sg.PREC_BF16)
        pc2, _ = sg.spai_update(ctx, pc1, A2d, sg.UPDATE_FIRST | sg.PREC_BF16)
        g1 = export(ctx, pc1)
        g2 = export(ctx, pc2)
        X = np.zeros((n, 16), order="F")
        st, info, rel = sg.block_solve(ctx, A2d, pc2, 16, np.asfortranarray(w.B), n, X, n, 30, 1e-8, 50)
        sg.spai_pc_destroy(pc2)
        sg.spai_pc_destroy(pc1)
        sg.spai_affine_destroy(aff)
    A1 = oracle.assemble(w.terms, oracle.coefficients(p1, 1.0), n)
    A2 = oracle.assemble(w.terms, oracle.coefficients(p2, 1.0), n)
    Jptr, Jind = oracle.pattern(A1, n)
    Iptr, Ilist = oracle.index_sets(A1, n, Jptr, Jind)
    for g in (g64, g1, g2):
        assert np.array_equal(g["Jptr"], Jptr) and np.array_equal(g["Jind"], Jind)
        assert np.array_equal(g["Iptr"], Iptr) and np.array_equal(g["Ilist"], Ilist)
        assert not g["status"].any()
    assert int(np.diff(Iptr).max()) == 125 and int(np.diff(Jptr).max()) == 27
    for k0, k1 in ranges:
        P1 = oracle.spai_build(A1, n, k0=k0, k1=k1, sets=(Jptr, Jind, Iptr, Ilist))
        Q2 = oracle.spai_update(P1, A2, n, k0=k0, k1=k1)
        sl = slice(Jptr[k0], Jptr[k1])
        Jp = Jptr[k0:k1 + 1] - Jptr[k0]
        assert column_rel_err_vec(Jp, g64["val"][sl], P1.val[sl]) <= 1e-10
        for g, ref in ((g1, P1), (g2, Q2)):
            err = column_rel_err_vec(Jp, g["val"][sl], ref.val[sl])
            assert err <= 2 * 2.0 ** -8 + 5e-6, (k0, err)
    assert info["converged"]
    true_rel = np.linalg.norm(w.B - oracle.spmm(A2, X, n), axis=0) / np.linalg.norm(w.B, axis=0)
    assert np.all(true_rel <= 1e-8), true_rel


def test_fullsize_batched_256_systems():
    """The many-small-systems workload at full size: 256 2D 5-point systems (sides 48..256,
    6.47 M unknowns), all FP32-factor SPAIs from one spai_build_batch call and all solves
    from one block_solve_batch call, as bench.py runs them.  Every system's true residual is
    recomputed on the host in FP64; three sampled systems (the smallest, the largest, one of
    pattern A^2) are compared with the oracle: index sets bit-exact, factor entries within
    the FP32 bar, solutions within 1e-6 of the oracle's all-FP64 solve."""
    import torch
    import paper_1809_06574_gb300 as sg
    ws = synth.batched_2d(256)
    kinds = [(sg.PATTERN_A if w.extra["pattern"] == "A" else sg.PATTERN_A2) | sg.PREC_FP32 for w in ws]
    As = [oracle.assemble(w.terms, oracle.coefficients(w.params[0], 1.0), w.n) for w in ws]
    sizes = [w.n for w in ws]
    sample = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), next(i for i, w in enumerate(ws)
                                                                       if w.extra["pattern"] == "A2")})
    with context() as ctx:
        from gpu_util import dev_csr
        ds = [dev_csr(A, w.n) for A, w in zip(As, ws)]
        pcs, st = sg.spai_build_batch(ctx, ds, kinds)
        assert st == 0
        got = {i: export(ctx, pcs[i]) for i in sample}
        Bd = [torch.as_tensor(np.ascontiguousarray(w.B.T), device="cuda:0") for w in ws]
        Xd = [torch.zeros((4, w.n), dtype=torch.float64, device="cuda:0") for w in ws]
        st, infos = sg.block_solve_batch(ctx, ds, pcs, 4, Bd, Xd, 30, 1e-8, 100)
        Xs = [x.cpu().numpy().T.copy() for x in Xd]
        for pc in pcs:
            sg.spai_pc_destroy(pc)
    assert st == 0 and all(i["converged"] for i in infos)
    for w, A, X in zip(ws, As, Xs):
        rel = np.linalg.norm(w.B - oracle.spmm(A, X, w.n), axis=0) / np.linalg.norm(w.B, axis=0)
        assert np.all(rel <= 1e-8)
    for i in sample:
        w, A = ws[i], As[i]
        ref = oracle.spai_build(A, w.n, oracle.PATTERN_A if w.extra["pattern"] == "A" else oracle.PATTERN_A2)
        g = got[i]
        for key in ("Jptr", "Jind", "Iptr", "Ilist", "status"):
            assert np.array_equal(g[key], getattr(ref, key)), (i, key)
        assert column_rel_err_vec(ref.Jptr, g["val"], ref.val) <= 5e-6, i
        Xo, io = oracle.block_gmres(oracle.csr_apply(A, w.n), ref.apply, w.B, 30, 1e-8, 100)
        assert io["converged"]
        assert np.linalg.norm(Xs[i] - Xo) <= 1e-6 * np.linalg.norm(Xo), i
