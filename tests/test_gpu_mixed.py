"""Mixed precision (SPAI_PREC_FP32, SPAI_PREC_BF16): FP32 column least squares and FP32
(or BF16-stored) factors, applied with FP64 products and sums, inside the FP64 block GMRES.

Bars (the error against the FP64 oracle, stated per result):
  * patterns, index sets and column status: bit-exact, as in the FP64 path;
  * factor entries: within 1e-4 of the largest oracle entry of their column for every
    case, within 5e-6 for the stencil workloads (FP32 Householder: about kappa(A_k) * 6e-8);
  * solves: every column's true residual <= tol, recomputed here in FP64, and the
    solution within 1e-6 (relative, Frobenius) of the oracle's all-FP64 solution.
The measured errors are printed (pytest -s).
"""

import numpy as np
import pytest

import oracle
import synth
from gpu_util import column_rel_err, context, dev_csr, export

pytestmark = pytest.mark.gpu

TOL32_ANY = 1e-4
TOL32_STENCIL = 5e-6


def _sg():
    import paper_1809_06574_gb300 as sg
    return sg


def _cases():
    cases = []
    A, _ = synth.random_sparse(150, 0.03, seed=0)
    cases.append(("random150-A", A, 150, oracle.PATTERN_A, False))
    A, _ = synth.random_sparse(150, 0.03, seed=1)
    cases.append(("random150-A2", A, 150, oracle.PATTERN_A2, False))
    w = synth.plain_2d_32()
    A = oracle.assemble(w.terms, oracle.coefficients(0.1, 1.0), w.n)
    cases.append(("2d-32-A", A, w.n, oracle.PATTERN_A, True))
    cases.append(("2d-32-A2", A, w.n, oracle.PATTERN_A2, True))
    w = synth.grid3d_7pt(side=16, nparams=2)
    A = oracle.assemble(w.terms, oracle.coefficients(0.5, 2.0), w.n)
    cases.append(("3d-16-7pt", A, w.n, oracle.PATTERN_A, True))
    w = synth.grid3d_27pt(side=7, nparams=2)
    A = oracle.assemble(w.terms, oracle.coefficients(0.5, 1.0), w.n)
    cases.append(("3d-7-27pt", A, w.n, oracle.PATTERN_A, True))
    cases.append(("appendix1", synth.appendix1_matrix(0.5, 0.3), 1006, oracle.PATTERN_A, False))
    return cases


@pytest.mark.parametrize("name,A,n,kind,stencil", _cases(), ids=[c[0] for c in _cases()])
def test_fp32_build_against_fp64_oracle(name, A, n, kind, stencil):
    sg = _sg()
    ref = oracle.spai_build(A, n, kind)
    with context() as ctx:
        pc, st = sg.spai_build(ctx, dev_csr(A, n), kind | sg.PREC_FP32)
        got = export(ctx, pc)
        sg.spai_pc_destroy(pc)
    assert st == 0
    assert np.array_equal(got["Jptr"], ref.Jptr) and np.array_equal(got["Jind"], ref.Jind)
    assert np.array_equal(got["Iptr"], ref.Iptr) and np.array_equal(got["Ilist"], ref.Ilist)
    assert np.array_equal(got["status"], ref.status)
    err = column_rel_err(ref.Jptr, got["val"], ref.val)
    print(f"FP32 build {name}: max column-relative entry error vs FP64 oracle {err:.2e}")
    assert err <= (TOL32_STENCIL if stencil else TOL32_ANY)


def test_fp32_update_against_fp64_oracle():
    sg = _sg()
    w = synth.grid3d_7pt(side=12, nparams=3)
    n = w.n
    As = [oracle.assemble(w.terms, oracle.coefficients(p, 1.0), n) for p in (0.1, 0.6)]
    P1 = oracle.spai_build(As[0], n)
    Q2 = oracle.spai_update(P1, As[1], n)
    with context() as ctx:
        Ad = [dev_csr(A, n) for A in As]
        pc1, _ = sg.spai_build(ctx, Ad[0], sg.PATTERN_A | sg.PREC_FP32)
        pc2, _ = sg.spai_update(ctx, pc1, Ad[1], sg.UPDATE_FIRST | sg.PREC_FP32)
        g2 = export(ctx, pc2)
        sg.spai_pc_destroy(pc2)
        sg.spai_pc_destroy(pc1)
    err = column_rel_err(Q2.Jptr, g2["val"], Q2.val)
    print(f"FP32 update 3d-12-7pt: max column-relative entry error vs FP64 oracle {err:.2e}")
    assert np.array_equal(g2["status"], Q2.status)
    assert err <= TOL32_STENCIL


@pytest.mark.parametrize("s", [1, 8])
def test_fp32_preconditioner_solve_reaches_fp64_tolerance(s):
    import torch
    sg = _sg()
    w = synth.grid3d_7pt(side=16, nparams=3, seed=5)
    n = w.n
    As = [oracle.assemble(w.terms, oracle.coefficients(p, 1.0), n) for p in w.params[:2]]
    B = np.ascontiguousarray(w.B[:, :s])
    P1 = oracle.spai_build(As[0], n)
    Pref = oracle.spai_update(P1, As[1], n)
    Xo, io = oracle.block_gmres(oracle.csr_apply(As[1], n), Pref.apply, B, 30, 1e-8, 50)
    with context() as ctx:
        Ad = [dev_csr(A, n) for A in As]
        its = {}
        for prec in (0, sg.PREC_FP32):
            pc1, _ = sg.spai_build(ctx, Ad[0], sg.PATTERN_A | prec)
            pc2, _ = sg.spai_update(ctx, pc1, Ad[1], sg.UPDATE_FIRST | prec)
            Bd = torch.as_tensor(B.T.copy(), device="cuda:0")
            Xd = torch.zeros((s, n), dtype=torch.float64, device="cuda:0")
            st, info, rel = sg.block_solve(ctx, Ad[1], pc2, s, Bd, n, Xd, n, 30, 1e-8, 50)
            X = Xd.cpu().numpy().T
            sg.spai_pc_destroy(pc2)
            sg.spai_pc_destroy(pc1)
            assert info["converged"]
            R = B - oracle.spmm(As[1], X, n)
            true_rel = np.linalg.norm(R, axis=0) / np.linalg.norm(B, axis=0)
            assert np.all(true_rel <= 1e-8)
            sol = np.linalg.norm(X - Xo) / np.linalg.norm(Xo)
            its[prec] = info["iterations"]
            print(f"solve s={s} {'FP32' if prec else 'FP64'} factors: {info['iterations']} iterations, "
                  f"max true residual {true_rel.max():.2e}, solution error vs FP64 oracle {sol:.2e}")
            assert sol <= 1e-6
        assert its[sg.PREC_FP32] <= its[0] + 1


# --------------------------------------------------------------------------- BF16 factors
# SPAI_PREC_BF16: the same FP32 least squares, each entry rounded to nearest-even BF16 for
# storage.  Bar per entry: |got - ref| <= 2^-8 |ref| (one BF16 rounding, half an ulp of
# 2^-7 relative) + the FP32 bar of its column; every stored value is a BF16 number.
BF16_REL = 2.0 ** -8


def _bf16_exact(v):
    import torch
    t = torch.as_tensor(v, dtype=torch.float64)
    return bool(torch.equal(t.to(torch.bfloat16).to(torch.float64), t))


@pytest.mark.parametrize("name,A,n,kind,stencil", _cases(), ids=[c[0] for c in _cases()])
def test_bf16_build_against_fp64_oracle(name, A, n, kind, stencil):
    sg = _sg()
    ref = oracle.spai_build(A, n, kind)
    with context() as ctx:
        pc, st = sg.spai_build(ctx, dev_csr(A, n), kind | sg.PREC_BF16)
        got = export(ctx, pc)
        mem16 = sg.spai_pc_mem_size(pc, False)
        sg.spai_pc_destroy(pc)
    assert st == 0
    assert np.array_equal(got["Jptr"], ref.Jptr) and np.array_equal(got["Jind"], ref.Jind)
    assert np.array_equal(got["Iptr"], ref.Iptr) and np.array_equal(got["Ilist"], ref.Ilist)
    assert np.array_equal(got["status"], ref.status)
    assert _bf16_exact(got["val"])
    lens = np.diff(ref.Jptr)
    colmax = np.zeros(n)
    np.maximum.at(colmax, np.repeat(np.arange(n), lens), np.abs(ref.val))
    bound = BF16_REL * np.abs(ref.val) + (TOL32_STENCIL if stencil else TOL32_ANY) * np.repeat(colmax, lens)
    excess = np.abs(got["val"] - ref.val) / np.maximum(bound, 1e-300)
    print(f"BF16 build {name}: worst entry error / bound {excess.max():.2f}, "
          f"column-relative {column_rel_err(ref.Jptr, got['val'], ref.val):.2e}")
    assert np.all(excess <= 1.0)
    # 2 bytes per factor entry (plus the matrix values and column status the handle keeps)
    assert mem16 <= 2 * len(ref.val) + 8 * len(A[1]) + 4 * n + 3 * 256


def test_bf16_update_and_solve_reach_fp64_tolerance():
    import torch
    sg = _sg()
    w = synth.grid3d_7pt(side=16, nparams=3, seed=5)
    n, s = w.n, 8
    As = [oracle.assemble(w.terms, oracle.coefficients(p, 1.0), n) for p in w.params[:2]]
    B = np.ascontiguousarray(w.B[:, :s])
    P1 = oracle.spai_build(As[0], n)
    Q2 = oracle.spai_update(P1, As[1], n)
    Xo, io = oracle.block_gmres(oracle.csr_apply(As[1], n), Q2.apply, B, 30, 1e-8, 50)
    with context() as ctx:
        Ad = [dev_csr(A, n) for A in As]
        its = {}
        for prec in (0, sg.PREC_BF16):
            pc1, _ = sg.spai_build(ctx, Ad[0], sg.PATTERN_A | prec)
            pc2, _ = sg.spai_update(ctx, pc1, Ad[1], sg.UPDATE_FIRST | prec)
            if prec:
                g2 = export(ctx, pc2)
                assert _bf16_exact(g2["val"])
                err = column_rel_err(Q2.Jptr, g2["val"], Q2.val)
                print(f"BF16 update 3d-16-7pt: max column-relative entry error {err:.2e}")
                assert err <= 2 * BF16_REL + TOL32_STENCIL
            Bd = torch.as_tensor(B.T.copy(), device="cuda:0")
            Xd = torch.zeros((s, n), dtype=torch.float64, device="cuda:0")
            st, info, rel = sg.block_solve(ctx, Ad[1], pc2, s, Bd, n, Xd, n, 30, 1e-8, 50)
            X = Xd.cpu().numpy().T
            sg.spai_pc_destroy(pc2)
            sg.spai_pc_destroy(pc1)
            assert info["converged"]
            true_rel = np.linalg.norm(B - oracle.spmm(As[1], X, n), axis=0) / np.linalg.norm(B, axis=0)
            assert np.all(true_rel <= 1e-8)
            sol = np.linalg.norm(X - Xo) / np.linalg.norm(Xo)
            its[prec] = info["iterations"]
            print(f"solve s={s} {'BF16' if prec else 'FP64'} factors: {info['iterations']} iterations, "
                  f"max true residual {true_rel.max():.2e}, solution error vs FP64 oracle {sol:.2e}")
            assert sol <= 1e-6
        assert its[sg.PREC_BF16] <= its[0] + 3


def test_fp32_and_bf16_flags_are_exclusive():
    sg = _sg()
    w = synth.plain_2d_32()
    A = oracle.assemble(w.terms, oracle.coefficients(0.1, 1.0), w.n)
    with context() as ctx:
        with pytest.raises(sg.SpaiError) as e:
            sg.spai_build(ctx, dev_csr(A, w.n), sg.PATTERN_A | sg.PREC_FP32 | sg.PREC_BF16)
        assert e.value.status == sg.SPAI_EINVAL


# ----------------------------------------------------------------------------- FP32 operator
U32 = 2.0 ** -24


def _abs_csr(A):
    return (A[0], A[1], np.abs(A[2]))


@pytest.mark.parametrize("case", ["3d-12-7pt", "3d-6-27pt", "random200"])
@pytest.mark.parametrize("s", [1, 2, 4, 8, 16])
def test_spmm_fp32_within_its_rounding_bound(case, s):
    """Y = A X with A's values and X rounded to FP32 and k products summed in FP32 (k the
    row's nonzeros): every entry is within (k + 2) u32 (|A| |X|) of the exact FP64 product
    (two input roundings and k multiply-add roundings, u32 = 2^-24)."""
    import torch
    sg = _sg()
    if case == "3d-12-7pt":
        w = synth.grid3d_7pt(side=12, nparams=2)
        A, n = oracle.assemble(w.terms, oracle.coefficients(0.5, 1.0), w.n), w.n
    elif case == "3d-6-27pt":
        w = synth.grid3d_27pt(side=6, nparams=2)
        A, n = oracle.assemble(w.terms, oracle.coefficients(0.5, 1.0), w.n), w.n
    else:
        n = 200
        A, _ = synth.random_sparse(n, 0.05, seed=3)
    X = np.asfortranarray(np.random.default_rng(s).standard_normal((n, s)))
    ref = oracle.spmm(A, X, n)
    mag = oracle.spmm(_abs_csr(A), np.abs(X), n)
    k = np.diff(A[0]).astype(np.float64)[:, None]
    ld = n + 5
    with context() as ctx:
        Xd = torch.zeros((s, ld), dtype=torch.float64, device="cuda:0")
        Xd[:, :n] = torch.as_tensor(X.T)
        Yd = torch.full((s, ld), 3.0, dtype=torch.float64, device="cuda:0")
        sg.spai_spmm_fp32(ctx, dev_csr(A, n), s, Xd, ld, Yd, ld)
        sg.spai_ctx_sync(ctx)
        Y = Yd.cpu().numpy()
    got = Y[:, :n].T
    assert np.all(Y[:, n:] == 3.0)
    err = np.abs(got - ref)
    bound = 1.001 * (k + 2) * U32 * mag
    assert np.all(err <= bound), float(np.max(err / np.maximum(bound, 1e-300)))
    # it is an FP32 computation: not all entries equal the FP64 product
    assert np.max(err / np.maximum(mag, 1e-300)) > 1e-10


def test_fp32_operator_conversions_are_ieee_exact():
    """The FP32 operator converts its FP64 input to FP32 and its FP32 result to FP64 with
    integer operations on the IEEE 754 layouts: with A = I (one product by 1.0 per row) Y is
    X rounded to FP32 and widened back (plus +0, the sum's start), which must equal numpy's
    IEEE conversions bit for bit -- ties to even, the overflow threshold, the subnormal range
    and zeros included."""
    import torch
    sg = _sg()
    f32 = np.float32
    tiny, big = float(np.finfo(f32).tiny), float(np.finfo(f32).max)
    ulp1 = 2.0 ** -23
    special = [0.0, -0.0, 1.0, -1.0, 1.0 + ulp1 / 2, 1.0 + 1.5 * ulp1, -(1.0 + ulp1 / 2), 3.0 + 2 * ulp1,
               1.0 + ulp1 / 2 + 2.0 ** -40, 1.0 + ulp1 / 2 - 2.0 ** -40, tiny, tiny / 2, tiny / 3, -tiny * 0.75,
               1e-42, 1e-46, big, -big, big * (1 + 2.0 ** -25), big * (1 + 2.0 ** -23), 1e39, -1e300,
               float(np.nextafter(f32(1.0), f32(2.0))), 0.1, -0.1, 2.0 ** -126, 2.0 ** 127, 7e-39]
    rng = np.random.default_rng(17)
    body = np.concatenate([rng.standard_normal(3000) * 10.0 ** rng.integers(-40, 40, 3000),
                           (rng.integers(1, 2 ** 24, 2000) + 0.5) * 2.0 ** rng.integers(-60, 60, 2000)])
    x = np.concatenate([np.array(special), body])
    n = len(x)
    A = (np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.ones(n))
    with np.errstate(over="ignore"):
        want = x.astype(f32).astype(np.float64) + 0.0  # the row sum starts from +0: -0 + +0 = +0
    with context() as ctx:
        Xd = torch.as_tensor(x.reshape(1, n).copy(), device="cuda:0")
        Yd = torch.zeros((1, n), dtype=torch.float64, device="cuda:0")
        sg.spai_spmm_fp32(ctx, dev_csr(A, n), 1, Xd, n, Yd, n)
        sg.spai_ctx_sync(ctx)
        got = Yd.cpu().numpy()[0]
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp64"])
def test_pc_apply_fp32_chain_within_its_rounding_bound(prec):
    """The FP32 apply of a factored update Q_2 (P_1 X) (values as stored, X and the FP32
    intermediate rounded once each, FP32 sums): within (kP + kQ + 4) u32 |Q_2| (|P_1| |X|) of
    the exact product of the stored factors, computed here from their exported values."""
    import torch
    sg = _sg()
    w = synth.grid3d_7pt(side=11, nparams=3)
    n = w.n
    As = [oracle.assemble(w.terms, oracle.coefficients(p, 1.0), n) for p in (0.2, 0.7)]
    flag = {"fp32": sg.PREC_FP32, "bf16": sg.PREC_BF16, "fp64": 0}[prec]
    s = 8
    X = np.asfortranarray(np.random.default_rng(9).standard_normal((n, s)))
    with context() as ctx:
        Ad = [dev_csr(A, n) for A in As]
        p1, _ = sg.spai_build(ctx, Ad[0], sg.PATTERN_A | flag)
        q2, _ = sg.spai_update(ctx, p1, Ad[1], sg.UPDATE_FIRST | flag)
        g1, g2 = export(ctx, p1), export(ctx, q2)
        Xd = torch.as_tensor(np.ascontiguousarray(X.T), device="cuda:0")
        Yd = torch.zeros((s, n), dtype=torch.float64, device="cuda:0")
        sg.spai_pc_apply_fp32(ctx, q2, s, Xd, n, Yd, n)
        sg.spai_ctx_sync(ctx)
        got = Yd.cpu().numpy().T
        sg.spai_pc_destroy(q2)
        sg.spai_pc_destroy(p1)

    def csc_to_csr(g):  # exported column-order factor -> CSR triplet of the same matrix
        cols = np.repeat(np.arange(n), np.diff(g["Jptr"]))
        order = np.lexsort((cols, g["Jind"]))
        rp = np.zeros(n + 1, np.int32)
        np.add.at(rp, g["Jind"] + 1, 1)
        return (np.cumsum(rp).astype(np.int32), cols[order].astype(np.int32), g["val"][order])

    P1, Q2 = csc_to_csr(g1), csc_to_csr(g2)
    ref = oracle.spmm(Q2, oracle.spmm(P1, X, n), n)
    mag = oracle.spmm(_abs_csr(Q2), oracle.spmm(_abs_csr(P1), np.abs(X), n), n)
    kk = float(np.diff(P1[0]).max() + np.diff(Q2[0]).max() + 4)
    err = np.abs(got - ref)
    assert np.all(err <= 1.001 * kk * U32 * mag), float(np.max(err / np.maximum(kk * U32 * mag, 1e-300)))


def _mixed_cases():
    return [("2d-32", 4, 0, 1), ("3d-16-7pt", 8, 1, 1), ("3d-16-7pt", 1, 1, 0), ("3d-14-7pt", 16, 2, 1),
            ("3d-9-27pt", 8, 1, 1)]


@pytest.mark.parametrize("name,s,factor,update", _mixed_cases(),
                         ids=[f"{c[0]}-s{c[1]}-f{c[2]}-u{c[3]}" for c in _mixed_cases()])
def test_mixed_solve_reaches_fp64_tolerance(name, s, factor, update):
    """SPAI_SOLVE_MIXED: the operator A P in FP32 inside each cycle, FP64 basis, Gram-Schmidt,
    least squares and true residual, FP64 refinement across cycles.  Every column's true
    residual (recomputed here in FP64) meets tol 1e-8, and the solution is within 1e-6 of the
    oracle's all-FP64 solve; factors FP64 (0), FP32 (1) or BF16 (2), built or updated."""
    sg = _sg()
    if name == "2d-32":
        w = synth.plain_2d_32()
    elif name == "3d-9-27pt":
        w = synth.grid3d_27pt(side=9, nparams=3, nrhs=s)
    else:
        w = synth.grid3d_7pt(side=int(name.split("-")[1]), nparams=3, nrhs=max(s, 1), seed=5)
    n = w.n
    B = np.asfortranarray(w.B[:, :s])
    As = [oracle.assemble(w.terms, oracle.coefficients(p, 1.0), n) for p in w.params[:2]]
    Af = As[1] if update else As[0]
    P1 = oracle.spai_build(As[0], n)
    Pref = oracle.spai_update(P1, As[1], n) if update else P1
    Xo, io = oracle.block_gmres(oracle.csr_apply(Af, n), Pref.apply, B, 30, 1e-8, 50)
    flag = {0: 0, 1: sg.PREC_FP32, 2: sg.PREC_BF16}[factor]
    with context() as ctx:
        Ad = [dev_csr(A, n) for A in As]
        pc1, _ = sg.spai_build(ctx, Ad[0], sg.PATTERN_A | flag)
        pc = sg.spai_update(ctx, pc1, Ad[1], sg.UPDATE_FIRST | flag)[0] if update else pc1
        res = {}
        for precision in (sg.SOLVE_FP64, sg.SOLVE_MIXED):
            X = np.zeros((n, s), order="F")
            st, info, rel = sg.block_solve(ctx, Ad[1] if update else Ad[0], pc, s, B, n, X, n, 30, 1e-8, 50,
                                           precision=precision)
            res[precision] = (X, info)
        if update:
            sg.spai_pc_destroy(pc)
        sg.spai_pc_destroy(pc1)
    for precision, (X, info) in res.items():
        assert info["converged"]
        true_rel = np.linalg.norm(B - oracle.spmm(Af, X, n), axis=0) / np.linalg.norm(B, axis=0)
        sol = np.linalg.norm(X - Xo) / np.linalg.norm(Xo)
        print(f"{name} s={s} factor={factor} update={update} "
              f"{'mixed' if precision else 'fp64'}: {info['iterations']} iterations in {info['cycles']} cycles "
              f"(oracle {io['iterations']}), max true residual {true_rel.max():.2e}, "
              f"solution error vs FP64 oracle {sol:.2e}")
        assert np.all(true_rel <= 1e-8)
        assert sol <= 1e-6
