"""Block Gram product H = V^T W of the orthogonalisation: tensor-core digit method vs FP64.

The digit method (nine 6-bit fixed-point digits, exact FP32 sums on the tensor cores, FP64
recombination) must be as accurate as FP64 arithmetic: both are compared with a sum in
extended precision on the host, per column relative to ||w_b|| ||v_a|| (= ||w_b||).
Solves with either method must give the same iterates up to rounding.
"""

import numpy as np
import pytest

import oracle
import synth
from gpu_util import context, dev_csr

pytestmark = pytest.mark.gpu


def _blocks(n, nblk, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, nblk * 8)))   # orthonormal basis columns
    W = rng.standard_normal((n, 8)) * np.array([1e3, 1.0, 1e-5, 3.0, 1e8, 0.5, 2.0, 0.0])
    W[: n // 3, 6] *= 1e-9                                      # mixed magnitudes in one column
    return Q, W


def _to_dev_blocks(Q, n, nblk):
    import torch
    # block i = rows x 8 row-major: element (r, a) of block i at (i * n + r) * 8 + a
    Vb = np.ascontiguousarray(Q.reshape(n, nblk, 8).transpose(1, 0, 2))
    return torch.as_tensor(Vb, device="cuda:0")


def _ref(Q, W):
    return (Q.astype(np.longdouble).T @ W.astype(np.longdouble)).astype(np.float64)


@pytest.mark.parametrize("n,nblk", [(1000, 1), (30000, 2), (4999, 4), (20000, 17), (12345, 18), (70001, 51)])
def test_tensor_gram_as_accurate_as_fp64(n, nblk):
    """Tiles of one or two blocks (nblk 1, 2 and the last tile of 17 or 18) take the
    stacked-digit MMA, the others one MMA per digit; both are exact digit sums."""
    import torch
    import paper_1809_06574_gb300 as sg
    Q, W = _blocks(n, nblk, seed=n + nblk)
    # extended-precision reference on a subset of basis columns (first and last block)
    cols = np.r_[0:8, nblk * 8 - 8:nblk * 8]
    ref = _ref(Q[:, cols], W)
    wn = np.linalg.norm(W, axis=0)
    scale = np.where(wn > 0, wn, 1.0)
    with context() as ctx:
        Vd = _to_dev_blocks(Q, n, nblk)
        Wd = torch.as_tensor(np.ascontiguousarray(W), device="cuda:0")
        outs = {}
        for method in (sg.ORTH_FP64, sg.ORTH_TENSOR):
            Hd = torch.full((nblk, 8, 8), np.nan, dtype=torch.float64, device="cuda:0")
            sg.spai_block_gram(ctx, 8, n, nblk, Vd, Wd, Hd, method)
            outs[method] = Hd.cpu().numpy().reshape(nblk * 8, 8)
    e64 = np.max(np.abs(outs[sg.ORTH_FP64][cols] - ref) / scale)
    etc = np.max(np.abs(outs[sg.ORTH_TENSOR][cols] - ref) / scale)
    assert np.all(outs[sg.ORTH_TENSOR][:, 7] == 0.0)              # zero column stays exact
    assert e64 <= 1e-14 and etc <= 1e-14, (e64, etc)
    assert etc <= 4 * max(e64, 1e-16), (e64, etc)
    # and the two methods agree on every entry
    assert np.max(np.abs(outs[sg.ORTH_TENSOR] - outs[sg.ORTH_FP64]) / scale) <= 2e-14


@pytest.mark.parametrize("n,nblk,sign", [(1000, 1, -1.0), (4999, 3, -1.0), (20000, 16, 1.0), (70001, 51, -1.0)])
def test_tensor_block_update_as_accurate_as_fp64(n, nblk, sign):
    import torch
    import paper_1809_06574_gb300 as sg
    Q, W = _blocks(n, nblk, seed=7 * n + nblk)
    rng = np.random.default_rng(n)
    H = rng.standard_normal((nblk * 8, 8)) * np.array([1.0, 1e-3, 1e4, 0.0, 1e-9, 2.0, 5.0, 1.0])
    rows = np.r_[0:257, n - 300:n]  # extended-precision reference on a subset of rows
    ref = (W[rows].astype(np.longdouble) +
           sign * (Q[rows].astype(np.longdouble) @ H.astype(np.longdouble))).astype(np.float64)
    scale = np.linalg.norm(H, axis=0) + np.abs(W[rows]).max(axis=0)
    scale = np.where(scale > 0, scale, 1.0)
    outs = {}
    with context() as ctx:
        Vd = _to_dev_blocks(Q, n, nblk)
        Hd = torch.as_tensor(np.ascontiguousarray(H), device="cuda:0")
        for method in (sg.ORTH_FP64, sg.ORTH_TENSOR):
            Wd = torch.as_tensor(np.ascontiguousarray(W), device="cuda:0")
            sg.spai_block_update(ctx, 8, n, nblk, Vd, Hd, Wd, sign, method)
            outs[method] = Wd.cpu().numpy()
    e64 = np.max(np.abs(outs[sg.ORTH_FP64][rows] - ref) / scale)
    etc = np.max(np.abs(outs[sg.ORTH_TENSOR][rows] - ref) / scale)
    assert e64 <= 1e-14 and etc <= 1e-14, (e64, etc)
    assert etc <= 4 * max(e64, 1e-16), (e64, etc)
    assert np.max(np.abs(outs[sg.ORTH_TENSOR] - outs[sg.ORTH_FP64]) / scale) <= 2e-14


def test_tensor_gram_rejects_out_of_range_basis():
    import torch
    import paper_1809_06574_gb300 as sg
    n = 2048
    Q, W = _blocks(n, 4, seed=1)
    Q[5, 3] = 3.0                                               # |v| >= 2 is outside the digits
    with context() as ctx:
        Vd = _to_dev_blocks(Q, n, 4)
        Wd = torch.as_tensor(np.ascontiguousarray(W), device="cuda:0")
        Hd = torch.zeros((4, 8, 8), dtype=torch.float64, device="cuda:0")
        with pytest.raises(sg.SpaiError) as ei:
            sg.spai_block_gram(ctx, 8, n, 4, Vd, Wd, Hd, sg.ORTH_TENSOR)
        assert ei.value.status == sg.SPAI_EINVAL


@pytest.mark.parametrize("nrhs,restart,side", [(8, 50, 24), (16, 30, 24), (16, 20, 23)])
def test_solve_with_tensor_orthogonalisation_matches_fp64(nrhs, restart, side):
    """8 columns run on the digit kernels directly, 16 columns as two 8-column halves
    against all half-blocks of the basis (side 23: n = 12,167, a ragged last sub-tile);
    both must give the FP64 iterates to rounding."""
    import paper_1809_06574_gb300 as sg
    w = synth.grid3d_7pt(side=side, nparams=2, nrhs=nrhs)
    n = w.n
    A = oracle.assemble(w.terms, oracle.coefficients(w.params[0], 0.5), n)
    P = oracle.spai_build(A, n)
    Xo, io = oracle.block_gmres(oracle.csr_apply(A, n), P.apply, w.B, restart, 1e-8, 20)
    res = {}
    with context() as ctx:
        Ad = dev_csr(A, n)
        pc, _ = sg.spai_build(ctx, Ad)
        for orth in (sg.ORTH_FP64, sg.ORTH_TENSOR, sg.ORTH_AUTO):
            X = np.zeros((n, nrhs), order="F")
            st, info, rel = sg.block_solve(ctx, Ad, pc, nrhs, np.asfortranarray(w.B), n, X, n, restart, 1e-8, 20,
                                           orth=orth)
            res[orth] = (X, info)
        sg.spai_pc_destroy(pc)
    for orth, (X, info) in res.items():
        assert info["converged"]
        true_rel = np.linalg.norm(w.B - oracle.spmm(A, X, n), axis=0) / np.linalg.norm(w.B, axis=0)
        assert np.all(true_rel <= 1e-8)
        assert np.linalg.norm(X - Xo) <= 1e-6 * np.linalg.norm(Xo)
    X64, i64 = res[sg.ORTH_FP64]
    Xtc, itc = res[sg.ORTH_TENSOR]
    assert itc["iterations"] == i64["iterations"]
    assert np.linalg.norm(Xtc - X64) <= 1e-10 * np.linalg.norm(X64)


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    """Failure detection of the tensor-core kernels without a fault: with a 2 ms wait limit,
    an injected stall (a bounded wait on a barrier that nothing completes) makes the Gram
    product and the block update give up -- each stops, drains its own copies and MMAs,
    frees its tensor memory and returns -- and the call returns SPAI_ETIMEOUT.  The next
    calls on the same context run normally and match the FP64 kernels; a block solve with a
    stall stops with SPAI_ETIMEOUT and the next solve converges."""
    import torch
    import paper_1809_06574_gb300 as sg
    n, nblk = 65536, 6
    Q, W = _blocks(n, nblk, seed=3)
    H = np.random.default_rng(5).standard_normal((nblk * 8, 8))
    with context() as ctx:
        sg.spai_ctx_set_wait_limit(ctx, 2e-3)
        Vd = _to_dev_blocks(Q, n, nblk)
        Wd = torch.as_tensor(np.ascontiguousarray(W), device="cuda:0")
        Hd = torch.zeros((nblk, 8, 8), dtype=torch.float64, device="cuda:0")
        for _ in range(2):  # twice in a row: each give-up leaves the context clean
            sg.spai_ctx_inject_stall(ctx, 1)
            with pytest.raises(sg.SpaiError) as ei:
                sg.spai_block_gram(ctx, 8, n, nblk, Vd, Wd, Hd, sg.ORTH_TENSOR)
            assert ei.value.status == sg.SPAI_ETIMEOUT
        H64 = torch.zeros_like(Hd)
        sg.spai_block_gram(ctx, 8, n, nblk, Vd, Wd, Hd, sg.ORTH_TENSOR)
        sg.spai_block_gram(ctx, 8, n, nblk, Vd, Wd, H64, sg.ORTH_FP64)
        wn = np.maximum(np.linalg.norm(W, axis=0), 1e-300)
        assert np.max(np.abs((Hd - H64).cpu().numpy().reshape(-1, 8)) / wn) <= 2e-14
        Hu = torch.as_tensor(np.ascontiguousarray(H), device="cuda:0")
        Wt = Wd.clone()
        sg.spai_ctx_inject_stall(ctx, 1)
        with pytest.raises(sg.SpaiError) as ei:
            sg.spai_block_update(ctx, 8, n, nblk, Vd, Hu, Wt, -1.0, sg.ORTH_TENSOR)
        assert ei.value.status == sg.SPAI_ETIMEOUT
        Wt, W64 = Wd.clone(), Wd.clone()
        sg.spai_block_update(ctx, 8, n, nblk, Vd, Hu, Wt, -1.0, sg.ORTH_TENSOR)
        sg.spai_block_update(ctx, 8, n, nblk, Vd, Hu, W64, -1.0, sg.ORTH_FP64)
        assert torch.max(torch.abs(Wt - W64)).item() <= 2e-14 * torch.max(torch.abs(W64)).item()
        # a block solve: the stalled product ends it with SPAI_ETIMEOUT; the next one converges
        w = synth.grid3d_7pt(side=20, nparams=2, nrhs=8)
        A = oracle.assemble(w.terms, oracle.coefficients(w.params[0], 1.0), w.n)
        Ad = dev_csr(A, w.n)
        pc, _ = sg.spai_build(ctx, Ad)
        X = np.zeros((w.n, 8), order="F")
        sg.spai_ctx_inject_stall(ctx, 1)
        with pytest.raises(sg.SpaiError) as ei:
            sg.block_solve(ctx, Ad, pc, 8, np.asfortranarray(w.B), w.n, X, w.n, 30, 1e-8, 20, orth=sg.ORTH_TENSOR)
        assert ei.value.status == sg.SPAI_ETIMEOUT
        sg.spai_ctx_set_wait_limit(ctx, 1.0)
        X = np.zeros((w.n, 8), order="F")
        st, info, rel = sg.block_solve(ctx, Ad, pc, 8, np.asfortranarray(w.B), w.n, X, w.n, 30, 1e-8, 20,
                                       orth=sg.ORTH_TENSOR)
        assert info["converged"] and max(rel) <= 1e-8
        true_rel = np.linalg.norm(w.B - oracle.spmm(A, X, w.n), axis=0) / np.linalg.norm(w.B, axis=0)
        assert np.all(true_rel <= 1e-8)
        with pytest.raises(sg.SpaiError):
            sg.spai_ctx_set_wait_limit(ctx, 0.0)
        sg.spai_pc_destroy(pc)
