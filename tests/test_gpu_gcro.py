"""Block GCRO with a recycled outer space (block_solve_gcro) against the oracle's block_gcro.

A sequence of systems A(p_1), A(p_2), ... (SPAI built at p_1, updated for the others, Table
1 first approach), solved one after another with the recycle space carried along: every
solution within 1e-6 of the oracle's (which carries its own space along the same sequence),
every true residual <= tol recomputed here in FP64, the iteration counts the oracle's (the
recycled spaces of the two sides differ only by rounding).  Without a recycled space the
solve is block_solve's; a space that holds the solution needs no Arnoldi step."""

import numpy as np
import pytest

import oracle
import synth
from gpu_util import context, dev_csr

pytestmark = pytest.mark.gpu


def _sg():
    import paper_1809_06574_gb300 as sg
    return sg


def _sequence(side=12, s=8, nparams=4, seed=2):
    w = synth.grid3d_7pt(side=side, nparams=nparams, nrhs=s, seed=seed)
    n = w.n
    As = [oracle.assemble(w.terms, oracle.coefficients(p, 1.0), n) for p in w.params]
    return w, n, As


def test_empty_recycle_space_is_block_gmres():
    sg = _sg()
    w, n, As = _sequence()
    with context() as ctx:
        Ad = dev_csr(As[0], n)
        pc, _ = sg.spai_build(ctx, Ad)
        rc = sg.spai_recycle_create(ctx, n, 8, 16)
        X1 = np.zeros((n, 8), order="F")
        X2 = np.zeros((n, 8), order="F")
        _, i1, _ = sg.block_solve(ctx, Ad, pc, 8, np.asfortranarray(w.B), n, X1, n, 30, 1e-8, 20)
        _, i2, _ = sg.block_solve_gcro(ctx, Ad, pc, 8, np.asfortranarray(w.B), n, X2, n, 30, 1e-8, 20, rc)
        k = sg.spai_recycle_info(rc)
        sg.spai_recycle_destroy(rc)
        sg.spai_pc_destroy(pc)
    assert i1["iterations"] == i2["iterations"] and i1["cycles"] == i2["cycles"]
    assert np.array_equal(X1, X2)
    assert k == 8  # the solve's iterate joined the space


@pytest.mark.parametrize("orth,precision", [(1, 0), (2, 0), (0, 1)], ids=["fp64", "tensor", "mixed"])
def test_sequence_matches_oracle(orth, precision):
    sg = _sg()
    w, n, As = _sequence()
    s, kmax, m = 8, 16, 30
    B = np.asfortranarray(w.B)
    P1 = oracle.spai_build(As[0], n)
    pcs_o = [P1] + [oracle.spai_update(P1, A, n) for A in As[1:]]
    U = None
    ref = []
    for A, Pq in zip(As, pcs_o):
        X, info, U = oracle.block_gcro(oracle.csr_apply(A, n), Pq.apply, B, m, 1e-8, 20, U=U, kmax=kmax)
        ref.append((X, info))
    got = []
    with context() as ctx:
        Ads = [dev_csr(A, n) for A in As]
        p1, _ = sg.spai_build(ctx, Ads[0])
        pcs = [p1] + [sg.spai_update(ctx, p1, Ad)[0] for Ad in Ads[1:]]
        rc = sg.spai_recycle_create(ctx, n, s, kmax)
        for Ad, pc in zip(Ads, pcs):
            X = np.zeros((n, s), order="F")
            st, info, rel = sg.block_solve_gcro(ctx, Ad, pc, s, B, n, X, n, m, 1e-8, 20, rc, orth=orth,
                                                precision=precision)
            got.append((X, info, sg.spai_recycle_info(rc)))
        sg.spai_recycle_destroy(rc)
        for pc in pcs[1:]:
            sg.spai_pc_destroy(pc)
        sg.spai_pc_destroy(p1)
    gmres_its = oracle.block_gmres(oracle.csr_apply(As[-1], n), pcs_o[-1].apply, B, m, 1e-8, 20)[1]["iterations"]
    for q, ((Xo, io), (X, info, k)) in enumerate(zip(ref, got)):
        assert info["converged"]
        true_rel = np.linalg.norm(B - oracle.spmm(As[q], X, n), axis=0) / np.linalg.norm(B, axis=0)
        sol = np.linalg.norm(X - Xo) / np.linalg.norm(Xo)
        print(f"system {q}: {info['iterations']} iterations ({info['cycles']} cycles), oracle {io['iterations']}; "
              f"true residual {true_rel.max():.2e}; solution vs oracle {sol:.2e}; recycled columns {k}")
        assert np.all(true_rel <= 1e-8)
        assert sol <= 1e-6
        if precision == 0:
            assert abs(info["iterations"] - io["iterations"]) <= 1
        assert k == min(kmax, 8 * (q + 1))
    print(f"block GMRES on the last system: {gmres_its} iterations")
    assert got[-1][1]["iterations"] < gmres_its


def test_a_space_holding_the_solution_needs_no_arnoldi_step():
    sg = _sg()
    w, n, As = _sequence(side=10)
    B = np.asfortranarray(w.B)
    with context() as ctx:
        Ad = dev_csr(As[1], n)
        pc, _ = sg.spai_build(ctx, Ad)
        rc = sg.spai_recycle_create(ctx, n, 8, 8)
        X1 = np.zeros((n, 8), order="F")
        sg.block_solve_gcro(ctx, Ad, pc, 8, B, n, X1, n, 30, 1e-10, 20, rc)
        X2 = np.zeros((n, 8), order="F")
        st, info, rel = sg.block_solve_gcro(ctx, Ad, pc, 8, B, n, X2, n, 30, 1e-8, 20, rc)
        sg.spai_recycle_destroy(rc)
        sg.spai_pc_destroy(pc)
    assert info["iterations"] == 0 and info["converged"]
    assert np.linalg.norm(X2 - X1) <= 1e-8 * np.linalg.norm(X1)


def test_recycle_space_keeps_the_latest_solutions():
    """kmax = 2 s: after three solves the space holds the last two iterates (exported
    columns span them), the oldest having left; clear empties it; sizes are checked."""
    import torch
    sg = _sg()
    w, n, As = _sequence(side=9, s=4, nparams=3)
    B = np.asfortranarray(w.B)
    with context() as ctx:
        Ads = [dev_csr(A, n) for A in As]
        pcs = [sg.spai_build(ctx, Ad)[0] for Ad in Ads]
        rc = sg.spai_recycle_create(ctx, n, 4, 8)
        Xs = []
        for Ad, pc in zip(Ads, pcs):
            X = np.zeros((n, 4), order="F")
            sg.block_solve_gcro(ctx, Ad, pc, 4, B, n, X, n, 30, 1e-10, 20, rc)
            Xs.append(X)
        assert sg.spai_recycle_info(rc) == 8
        Ud = torch.zeros((8, n), dtype=torch.float64, device="cuda:0")  # column-major n x 8
        sg.spai_recycle_export(ctx, rc, Ud, n)
        sg.spai_ctx_sync(ctx)
        U = Ud.cpu().numpy().T
        # P X~ of the last solve is its X: the last block of U maps to X through its own P
        Y = torch.zeros((4, n), dtype=torch.float64, device="cuda:0")
        Ul = torch.as_tensor(np.ascontiguousarray(U[:, 4:].T), device="cuda:0")
        sg.spai_pc_apply(ctx, pcs[-1], 4, Ul, n, Y, n)
        sg.spai_ctx_sync(ctx)
        assert np.linalg.norm(Y.cpu().numpy().T - Xs[-1]) <= 1e-9 * np.linalg.norm(Xs[-1])
        sg.spai_recycle_clear(rc)
        assert sg.spai_recycle_info(rc) == 0
        with pytest.raises(sg.SpaiError):
            sg.spai_recycle_create(ctx, n, 4, 6)  # not a multiple of s
        with pytest.raises(sg.SpaiError):  # made for s = 4
            sg.block_solve_gcro(ctx, Ads[0], pcs[0], 8, np.asfortranarray(np.zeros((n, 8))), n,
                                np.zeros((n, 8), order="F"), n, 30, 1e-8, 20, rc)
        sg.spai_recycle_destroy(rc)
        for pc in pcs:
            sg.spai_pc_destroy(pc)
