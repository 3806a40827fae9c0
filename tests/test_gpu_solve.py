"""GPU parity of right-preconditioned block GMRES (through the C ABI) with the oracle.

Bar: solutions within 1e-6 relative (Frobenius) of the oracle's, and every column's true
residual ||b_i - A x_i|| <= tol ||b_i||, recomputed here in FP64 on the host.
"""

import numpy as np
import pytest

import oracle
import synth
from gpu_util import context, dev_csr

pytestmark = pytest.mark.gpu

SOL_TOL = 1e-6


def _sg():
    import paper_1809_06574_gb300 as sg
    return sg


def _true_rel(A, X, B, n):
    R = B - oracle.spmm(A, X, n)
    return np.linalg.norm(R, axis=0) / np.where(np.linalg.norm(B, axis=0) > 0,
                                                 np.linalg.norm(B, axis=0), 1.0)


def _solve_gpu(ctx, Ad, pc, B, restart, tol, max_cycles, device_buffers=False, X0=None):
    import torch
    sg = _sg()
    n, s = B.shape
    if device_buffers:
        Bd = torch.as_tensor(np.ascontiguousarray(B.T), device="cuda:0")
        Xd = torch.zeros((s, n), dtype=torch.float64, device="cuda:0")
        if X0 is not None:
            Xd.copy_(torch.as_tensor(np.ascontiguousarray(X0.T)))
        st, info, rel = sg.block_solve(ctx, Ad, pc, s, Bd, n, Xd, n, restart, tol, max_cycles)
        return Xd.cpu().numpy().T.copy(), info, rel
    X = np.zeros((n, s), order="F") if X0 is None else np.asfortranarray(X0.copy())
    Bf = np.asfortranarray(B)
    st, info, rel = sg.block_solve(ctx, Ad, pc, s, Bf, n, X, n, restart, tol, max_cycles)
    return X, info, rel


def test_plain_2d_sweep_build_then_updates():
    """2D 32x32: build at p = 0.1, update for p = 0.2..0.5, GMRES(30), tol 1e-8, 4 RHS."""
    sg = _sg()
    w = synth.plain_2d_32()
    n = w.n
    As = [oracle.assemble(w.terms, oracle.coefficients(p, 1.0), n) for p in w.params]
    P1 = oracle.spai_build(As[0], n)
    with context() as ctx:
        Ad = [dev_csr(A, n) for A in As]
        pc1, _ = sg.spai_build(ctx, Ad[0])
        for i, p in enumerate(w.params):
            if i == 0:
                pc, Pref = pc1, P1
            else:
                pc, _ = sg.spai_update(ctx, pc1, Ad[i])
                Pref = oracle.spai_update(P1, As[i], n)
            X, info, rel = _solve_gpu(ctx, Ad[i], pc, w.B, 30, 1e-8, 50)
            Xo, io = oracle.block_gmres(oracle.csr_apply(As[i], n), Pref.apply, w.B, 30, 1e-8, 50)
            assert info["converged"] and io["converged"]
            assert np.all(_true_rel(As[i], X, w.B, n) <= 1e-8)
            assert np.allclose(rel, _true_rel(As[i], X, w.B, n), rtol=1e-6, atol=1e-14)
            assert np.linalg.norm(X - Xo) <= SOL_TOL * np.linalg.norm(Xo)
            assert abs(info["iterations"] - io["iterations"]) <= 1
            if i:
                sg.spai_pc_destroy(pc)
        sg.spai_pc_destroy(pc1)


@pytest.mark.parametrize("s", [1, 2, 8, 16])
def test_block_sizes_and_buffers(s):
    sg = _sg()
    w = synth.grid3d_7pt(side=10, nparams=2, nrhs=s)
    n = w.n
    A = oracle.assemble(w.terms, oracle.coefficients(w.params[0], 0.5), n)
    P = oracle.spai_build(A, n)
    Xo, io = oracle.block_gmres(oracle.csr_apply(A, n), P.apply, w.B, 20, 1e-8, 50)
    with context() as ctx:
        Ad = dev_csr(A, n)
        pc, _ = sg.spai_build(ctx, Ad)
        Xh, info_h, _ = _solve_gpu(ctx, Ad, pc, w.B, 20, 1e-8, 50, device_buffers=False)
        Xd, info_d, _ = _solve_gpu(ctx, Ad, pc, w.B, 20, 1e-8, 50, device_buffers=True)
        sg.spai_pc_destroy(pc)
    assert np.array_equal(Xh, Xd)
    assert info_h == info_d
    assert np.all(_true_rel(A, Xh, w.B, n) <= 1e-8)
    assert np.linalg.norm(Xh - Xo) <= SOL_TOL * np.linalg.norm(Xo)


def test_no_preconditioner_and_restarts():
    sg = _sg()
    w = synth.grid3d_7pt(side=8, nparams=2, nrhs=4)
    n = w.n
    A = oracle.assemble(w.terms, oracle.coefficients(w.params[0], 1.0), n)
    Xo, io = oracle.block_gmres(oracle.csr_apply(A, n), None, w.B, 5, 1e-10, 200)
    with context() as ctx:
        X, info, _ = _solve_gpu(ctx, dev_csr(A, n), None, w.B, 5, 1e-10, 200)
    assert info["cycles"] > 1 and info["converged"]
    assert np.all(_true_rel(A, X, w.B, n) <= 1e-10)
    assert np.linalg.norm(X - Xo) <= SOL_TOL * np.linalg.norm(Xo)


def test_full_space_one_cycle_and_zero_column():
    """n <= m*s: the Krylov space fills up (deflation of the invariant block)."""
    sg = _sg()
    n, s, m = 24, 4, 6
    A, D = synth.random_sparse(n, 0.2, seed=8)
    B = np.random.default_rng(3).standard_normal((n, s))
    B[:, 2] = 0.0
    with context() as ctx:
        Ad = dev_csr(A, n)
        pc, _ = sg.spai_build(ctx, Ad)
        X, info, rel = _solve_gpu(ctx, Ad, pc, B, m, 1e-12, 3)
        sg.spai_pc_destroy(pc)
    X_ref = oracle.lu_solve(D, B)
    assert info["converged"]
    assert np.all(X[:, 2] == 0.0)
    assert np.linalg.norm(X - X_ref) <= 1e-9 * np.linalg.norm(X_ref)


def test_initial_guess_used():
    sg = _sg()
    w = synth.plain_2d_32()
    n = w.n
    A = oracle.assemble(w.terms, oracle.coefficients(0.3, 1.0), n)
    X_exact = oracle.lu_solve(synth.csr_to_dense(A, n), w.B)
    with context() as ctx:
        X, info, _ = _solve_gpu(ctx, dev_csr(A, n), None, w.B, 30, 1e-8, 10, X0=X_exact)
    assert info["cycles"] == 0 and info["iterations"] == 0
    assert np.array_equal(X, X_exact)


def test_not_converged_reported():
    sg = _sg()
    w = synth.grid3d_7pt(side=10, nparams=2, nrhs=2)
    n = w.n
    A = oracle.assemble(w.terms, oracle.coefficients(w.params[0], 0.5), n)
    with context() as ctx:
        with pytest.raises(sg.SpaiError) as ei:
            _solve_gpu(ctx, dev_csr(A, n), None, w.B, 2, 1e-12, 1)
        assert ei.value.status == sg.SPAI_ENOTCONV
        st, info, rel = ei.value.result
        assert info["converged"] == 0 and info["cycles"] == 1 and max(rel) > 1e-12


def test_appendix1_solve_with_updated_preconditioner_is_exact():
    """Appendix I: Q_l P_1 = A(l)^{-1}, so one Krylov step solves the system."""
    sg = _sg()
    n = 1006
    A1 = synth.appendix1_matrix(0.5, 0.3)
    Al = synth.appendix1_matrix(0.5, 0.45)
    B = synth.rhs_block(n, 2, seed=5)
    with context() as ctx:
        A1d, Ald = dev_csr(A1, n), dev_csr(Al, n)
        pc1, _ = sg.spai_build(ctx, A1d)
        pc2, _ = sg.spai_update(ctx, pc1, Ald)
        X, info, rel = _solve_gpu(ctx, Ald, pc2, B, 5, 1e-12, 2)
        sg.spai_pc_destroy(pc2)
        sg.spai_pc_destroy(pc1)
    assert info["converged"] and info["iterations"] == 1
    X_ref = oracle.lu_solve(synth.csr_to_dense(Al, n), B)
    assert np.linalg.norm(X - X_ref) <= 1e-12 * np.linalg.norm(X_ref)
