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
