"""Batched SPAI build (spai_build_batch): the column problems of many independent systems
in one persistent launch per tile shape, with the team size picked by the autotuner; and
the batched block GMRES (block_solve_batch) that solves many systems in lockstep.

Bars: patterns, index sets and column status bit-exact against the oracle; entries within
1e-10 of the largest oracle entry of their column (FP64), within the FP32 / BF16 bars of
the mixed-precision tests otherwise; and against the single-system spai_build of the same
matrix, which may use another team size, within 1e-13 (rounding of the reductions only).
"""

import numpy as np
import pytest

import oracle
import synth
from gpu_util import column_rel_err, context, dev_csr, export

pytestmark = pytest.mark.gpu


def _sg():
    import paper_1809_06574_gb300 as sg
    return sg


def _systems():
    """(name, A, n, kind, precision flag) of a heterogeneous batch."""
    sg = _sg()
    out = []
    rng = np.random.default_rng(3)
    for i, side in enumerate((8, 13, 21, 34, 40, 17)):
        w = synth.grid_workload((side, side), "5pt", seed=i, nrhs=4, params=[0.5])
        A = oracle.assemble(w.terms, oracle.coefficients(float(rng.uniform(0.1, 1.0)), 1.0), w.n)
        kind = oracle.PATTERN_A if i % 2 == 0 else oracle.PATTERN_A2
        out.append((f"2d-{side}-{'A' if kind == 0 else 'A2'}", A, w.n, kind, 0))
    for seed in (0, 1):
        A, _ = synth.random_sparse(90 + 17 * seed, 0.04, seed=seed)
        out.append((f"random-{seed}", A, 90 + 17 * seed, oracle.PATTERN_A2 if seed else oracle.PATTERN_A, 0))
    w = synth.grid3d_7pt(side=9, nparams=2)
    out.append(("3d-9-7pt", oracle.assemble(w.terms, oracle.coefficients(0.4, 2.0), w.n), w.n, oracle.PATTERN_A, 0))
    w = synth.grid3d_27pt(side=5, nparams=2)
    out.append(("3d-5-27pt", oracle.assemble(w.terms, oracle.coefficients(0.4, 1.0), w.n), w.n, oracle.PATTERN_A, 0))
    # pattern A^2 of the 27-point grid: |J_k| up to 125, the widest union lists (32-lane teams)
    out.append(("3d-5-27pt-A2", out[-1][1], w.n, oracle.PATTERN_A2, 0))
    # the same shapes again in FP32 and BF16
    out.append(("2d-21-A-fp32", out[2][1], out[2][2], oracle.PATTERN_A, sg.PREC_FP32))
    out.append(("2d-34-A2-bf16", out[3][1], out[3][2], oracle.PATTERN_A2, sg.PREC_BF16))
    return out


def test_batch_matches_oracle_and_single_builds():
    sg = _sg()
    systems = _systems()
    with context() as ctx:
        Ads = [dev_csr(A, n) for _, A, n, _, _ in systems]
        pcs, st = sg.spai_build_batch(ctx, Ads, [k | p for _, _, _, k, p in systems])
        assert st == 0
        got = [export(ctx, pc) for pc in pcs]
        single = []
        for (name, A, n, k, p), Ad in zip(systems, Ads):
            pc, _ = sg.spai_build(ctx, Ad, k | p)
            single.append(export(ctx, pc))
            sg.spai_pc_destroy(pc)
        # a second batch reuses the tuned team sizes: identical bits
        pcs2, _ = sg.spai_build_batch(ctx, Ads, [k | p for _, _, _, k, p in systems])
        again = [export(ctx, pc) for pc in pcs2]
        for pc in pcs + pcs2:
            sg.spai_pc_destroy(pc)
    for (name, A, n, k, p), g, g1, g2 in zip(systems, got, single, again):
        ref = oracle.spai_build(A, n, k)
        for key in ("Jptr", "Jind", "Iptr", "Ilist", "status"):
            assert np.array_equal(g[key], getattr(ref, key)), (name, key)
            assert np.array_equal(g[key], g1[key]), (name, key)
        assert np.array_equal(g["val"], g2["val"]), name
        err = column_rel_err(ref.Jptr, g["val"], ref.val)
        bar = {0: 1e-10, sg.PREC_FP32: 1e-4, sg.PREC_BF16: 2 * 2.0 ** -8 + 1e-4}[p]
        print(f"batch {name}: column-relative error vs oracle {err:.2e}")
        assert err <= bar, name
        if p == 0:
            assert column_rel_err(ref.Jptr, g["val"], g1["val"]) <= 1e-13, name


def test_batch_handles_update_and_solve():
    import torch
    sg = _sg()
    ws = [synth.grid_workload((s, s), "5pt", seed=10 + s, nrhs=4, params=[0.2, 0.3]) for s in (20, 31, 26)]
    kinds = [oracle.PATTERN_A, oracle.PATTERN_A2, oracle.PATTERN_A]
    with context() as ctx:
        A1 = [oracle.assemble(w.terms, oracle.coefficients(w.params[0], 1.0), w.n) for w in ws]
        A2 = [oracle.assemble(w.terms, oracle.coefficients(w.params[1], 1.0), w.n) for w in ws]
        d1 = [dev_csr(A, w.n) for A, w in zip(A1, ws)]
        d2 = [dev_csr(A, w.n) for A, w in zip(A2, ws)]
        pcs, _ = sg.spai_build_batch(ctx, d1, kinds)
        for w, a1, a2, dd2, pc, k in zip(ws, A1, A2, d2, pcs, kinds):
            q, _ = sg.spai_update(ctx, pc, dd2)
            Bd = torch.as_tensor(np.ascontiguousarray(w.B.T), device="cuda:0")
            Xd = torch.zeros((4, w.n), dtype=torch.float64, device="cuda:0")
            st, info, rel = sg.block_solve(ctx, dd2, q, 4, Bd, w.n, Xd, w.n, 30, 1e-8, 50)
            X = Xd.cpu().numpy().T
            sg.spai_pc_destroy(q)
            sg.spai_pc_destroy(pc)
            Q = oracle.spai_update(oracle.spai_build(a1, w.n, k), a2, w.n)
            Xo, io = oracle.block_gmres(oracle.csr_apply(a2, w.n), Q.apply, w.B, 30, 1e-8, 50)
            assert info["converged"] and io["converged"]
            assert np.linalg.norm(X - Xo) <= 1e-6 * np.linalg.norm(Xo)


def test_batch_reports_singular_system():
    sg = _sg()
    w = synth.grid_workload((10, 10), "5pt", seed=1, nrhs=4, params=[0.5])
    A = oracle.assemble(w.terms, oracle.coefficients(0.5, 1.0), w.n)
    # a matrix with an empty column 7 (its values zeroed, pattern kept)
    rp, ci, va = A
    Z = (rp, ci, np.where(ci == 7, 0.0, va))
    with context() as ctx:
        pcs, st = sg.spai_build_batch(ctx, [dev_csr(A, w.n), dev_csr(Z, w.n)], [0, 0], allow_singular=True)
        assert st == sg.SPAI_ESINGULAR and "system 1" in sg.spai_last_error(ctx)
        g0, g1 = export(ctx, pcs[0]), export(ctx, pcs[1])
        for pc in pcs:
            sg.spai_pc_destroy(pc)
    ref = oracle.spai_build(Z, w.n)
    assert not g0["status"].any()
    assert np.array_equal(g1["status"], ref.status) and g1["status"][7] == 1


def test_batched_solve_matches_oracle_and_single_solves():
    """block_solve_batch: every system against the oracle's block GMRES (solution bar 1e-6),
    its own true residual recomputed on the host, and the single-system block_solve.  A
    system leaves the lockstep once its residual estimate meets tol, so it takes the steps
    the single solve takes (one step apart at most where rounding moves the estimate across
    tol) and, with the same steps, reaches the single solve's iterate to rounding."""
    import torch
    sg = _sg()
    ws = [synth.grid_workload((d, d), "5pt", seed=20 + d, nrhs=4, params=[0.3, 0.45]) for d in (17, 30, 23, 41)]
    w3 = synth.grid3d_7pt(side=9, nparams=2, seed=3, nrhs=4)
    ws.append(w3)
    kinds = [oracle.PATTERN_A, oracle.PATTERN_A2, oracle.PATTERN_A, oracle.PATTERN_A2, oracle.PATTERN_A]
    s = 4
    A1 = [oracle.assemble(w.terms, oracle.coefficients(w.params[0], 1.0), w.n) for w in ws]
    A2 = [oracle.assemble(w.terms, oracle.coefficients(w.params[1], 1.0), w.n) for w in ws]
    # a zero right-hand-side column in one system
    ws[2].B[:, 1] = 0.0
    with context() as ctx:
        d1 = [dev_csr(A, w.n) for A, w in zip(A1, ws)]
        d2 = [dev_csr(A, w.n) for A, w in zip(A2, ws)]
        base, _ = sg.spai_build_batch(ctx, d1, kinds)
        upd = [sg.spai_update(ctx, b, d)[0] for b, d in zip(base, d2)]
        Bd = [torch.as_tensor(np.ascontiguousarray(w.B.T), device="cuda:0") for w in ws]
        Xd = [torch.zeros((s, w.n), dtype=torch.float64, device="cuda:0") for w in ws]
        st, infos = sg.block_solve_batch(ctx, d2, upd, s, Bd, Xd, 30, 1e-8, 50)
        Xb = [x.cpu().numpy().T.copy() for x in Xd]
        single, single_info = [], []
        for w, d, q in zip(ws, d2, upd):
            X = np.zeros((w.n, s), order="F")
            _, sinf, _ = sg.block_solve(ctx, d, q, s, np.asfortranarray(w.B), w.n, X, w.n, 30, 1e-8, 50)
            single.append(X)
            single_info.append(sinf)
        for q in upd + base:
            sg.spai_pc_destroy(q)
    assert st == 0
    its = [inf["iterations"] for inf in infos]
    assert len(set(its)) > 1  # the systems stop after different numbers of steps
    for i, (w, a1, a2, k, X, Xs, inf, sinf) in enumerate(zip(ws, A1, A2, kinds, Xb, single, infos, single_info)):
        assert inf["converged"] and inf["max_rel_residual"] <= 1e-8, (i, inf)
        assert abs(inf["iterations"] - sinf["iterations"]) <= 1 and inf["cycles"] == sinf["cycles"], (i, inf, sinf)
        if inf["iterations"] == sinf["iterations"]:
            assert np.linalg.norm(X - Xs) <= 1e-8 * np.linalg.norm(Xs), i
        bn = np.linalg.norm(w.B, axis=0)
        rel = np.linalg.norm(w.B - oracle.spmm(a2, X, w.n), axis=0) / np.where(bn > 0, bn, 1.0)
        assert np.all(rel <= 1e-8), (i, rel)
        Q = oracle.spai_update(oracle.spai_build(a1, w.n, k), a2, w.n)
        Xo, io = oracle.block_gmres(oracle.csr_apply(a2, w.n), Q.apply, w.B, 30, 1e-8, 50)
        assert np.linalg.norm(X - Xo) <= 1e-6 * np.linalg.norm(Xo), i
        assert np.linalg.norm(X - Xs) <= 1e-6 * np.linalg.norm(Xs), i
        assert not X[:, 1].any() if i == 2 else True


def test_batched_solve_restarts_without_preconditioner():
    """No preconditioner and a short restart: several cycles; the per-system cycle counts
    and the solutions against the oracle."""
    import torch
    sg = _sg()
    ws = [synth.grid_workload((d, d), "5pt", seed=40 + d, nrhs=2, params=[0.5]) for d in (12, 19, 15)]
    As = [oracle.assemble(w.terms, oracle.coefficients(0.5, 1.0), w.n) for w in ws]
    with context() as ctx:
        ds = [dev_csr(A, w.n) for A, w in zip(As, ws)]
        Bd = [torch.as_tensor(np.ascontiguousarray(w.B.T), device="cuda:0") for w in ws]
        Xd = [torch.zeros((2, w.n), dtype=torch.float64, device="cuda:0") for w in ws]
        st, infos = sg.block_solve_batch(ctx, ds, None, 2, Bd, Xd, 4, 1e-8, 200)
        Xb = [x.cpu().numpy().T.copy() for x in Xd]
    assert st == 0
    assert max(inf["cycles"] for inf in infos) > 1
    for w, A, X, inf in zip(ws, As, Xb, infos):
        Xo, io = oracle.block_gmres(oracle.csr_apply(A, w.n), None, w.B, 4, 1e-8, 200)
        assert inf["converged"] and io["converged"]
        assert np.linalg.norm(X - Xo) <= 1e-6 * np.linalg.norm(Xo)


def test_stacked_batch_handles_outlive_each_other():
    """The stacked analysis carves every handle of a batch from one allocation: destroying
    some handles of the batch leaves the others intact (exports and products against the
    oracle after the others are gone), and an update, which shares its base's analysis, may
    be destroyed after its base (a base must stay alive while its update is USED; the
    shared allocation goes with the last handle)."""
    import torch
    sg = _sg()
    ws = [synth.grid_workload((d, d), "5pt", seed=60 + d, nrhs=4, params=[0.25, 0.4]) for d in (14, 27, 19)]
    kinds = [oracle.PATTERN_A2, oracle.PATTERN_A, oracle.PATTERN_A2]
    A1 = [oracle.assemble(w.terms, oracle.coefficients(w.params[0], 1.0), w.n) for w in ws]
    A2 = [oracle.assemble(w.terms, oracle.coefficients(w.params[1], 1.0), w.n) for w in ws]
    X = [np.asfortranarray(np.random.default_rng(d).standard_normal((w.n, 4))) for d, w in enumerate(ws)]
    with context() as ctx:
        d1 = [dev_csr(A, w.n) for A, w in zip(A1, ws)]
        d2 = [dev_csr(A, w.n) for A, w in zip(A2, ws)]
        pcs, _ = sg.spai_build_batch(ctx, d1, kinds)
        q1, _ = sg.spai_update(ctx, pcs[1], d2[1])

        def apply(h, x, w):
            Xd = torch.as_tensor(x.T.copy(), device="cuda:0")
            Yd = torch.empty_like(Xd)
            sg.spai_pc_apply(ctx, h, 4, Xd, w.n, Yd, w.n)
            sg.spai_ctx_sync(ctx)
            return Yd.cpu().numpy().T

        sg.spai_pc_destroy(pcs[0])
        g2 = export(ctx, pcs[2])
        Y = [apply(pcs[2], X[2], ws[2])]
        sg.spai_pc_destroy(pcs[2])
        gq = export(ctx, q1)
        Y.append(apply(q1, X[1], ws[1]))
        sg.spai_pc_destroy(pcs[1])  # the base first: its update still holds the shared allocation
        sg.spai_pc_destroy(q1)
    P2 = oracle.spai_build(A1[2], ws[2].n, kinds[2])
    Q1 = oracle.spai_update(oracle.spai_build(A1[1], ws[1].n, kinds[1]), A2[1], ws[1].n)
    for g, ref in ((g2, P2), (gq, Q1)):
        for key in ("Jptr", "Jind", "Iptr", "Ilist", "status"):
            assert np.array_equal(g[key], getattr(ref, key)), key
        assert column_rel_err(ref.Jptr, g["val"], ref.val) <= 1e-10
    for y, ref, x in ((Y[0], P2, X[2]), (Y[1], Q1, X[1])):
        yr = ref.apply(x)
        assert np.max(np.abs(y - yr)) <= 1e-10 * np.max(np.abs(yr))


def test_stacked_batch_checks_every_system():
    """Each system's CSR arrays are checked in its own index range: a column index equal to
    that system's n (inside the stacked matrix's range) and a row pointer that does not end
    at its nnz are both rejected, with no handle returned."""
    sg = _sg()
    ws = [synth.grid_workload((d, d), "5pt", seed=d, nrhs=4, params=[0.5]) for d in (9, 12)]
    As = [oracle.assemble(w.terms, oracle.coefficients(0.5, 1.0), w.n) for w in ws]
    rp, ci, va = As[0]
    bad_col = (rp, np.concatenate([ci[:-1], [ws[0].n]]).astype(np.int32), va)
    bad_ptr = (np.concatenate([rp[:-1], [rp[-1] - 1]]).astype(np.int32), ci, va)
    with context() as ctx:
        good = dev_csr(As[1], ws[1].n)
        for bad in (bad_col, bad_ptr):
            with pytest.raises(sg.SpaiError) as e:
                sg.spai_build_batch(ctx, [dev_csr(bad, ws[0].n), good], [0, 0])
            assert e.value.status == sg.SPAI_EINVAL
        # the context stays usable
        pcs, st = sg.spai_build_batch(ctx, [dev_csr(As[0], ws[0].n), good], [0, 1])
        g = [export(ctx, pc) for pc in pcs]
        for pc in pcs:
            sg.spai_pc_destroy(pc)
    assert st == 0
    for gg, A, w, k in zip(g, As, ws, (0, 1)):
        ref = oracle.spai_build(A, w.n, k)
        assert np.array_equal(gg["Jind"], ref.Jind) and np.array_equal(gg["Ilist"], ref.Ilist)
        assert column_rel_err(ref.Jptr, gg["val"], ref.val) <= 1e-10


def test_batch_with_an_empty_system():
    """A batch that holds an n = 0 system takes the per-system analysis; the other systems'
    results are those of the oracle and the empty system's handle is valid (n = 0)."""
    import torch
    sg = _sg()
    ws = [synth.grid_workload((d, d), "5pt", seed=d, nrhs=4, params=[0.5]) for d in (10, 15)]
    As = [oracle.assemble(w.terms, oracle.coefficients(0.3, 1.0), w.n) for w in ws]
    with context() as ctx:
        rp0 = torch.zeros(1, dtype=torch.int32, device="cuda:0")
        empty = sg.csr(0, rp0, None, None, nnz=0)
        pcs, st = sg.spai_build_batch(ctx, [dev_csr(As[0], ws[0].n), empty, dev_csr(As[1], ws[1].n)], [0, 0, 1])
        assert st == 0
        info = sg.spai_pc_info(pcs[1])
        g = [export(ctx, pcs[0]), export(ctx, pcs[2])]
        for pc in pcs:
            sg.spai_pc_destroy(pc)
    assert info["n"] == 0 and info["nnz"] == 0
    for gg, A, w, k in zip(g, As, ws, (0, 1)):
        ref = oracle.spai_build(A, w.n, k)
        assert np.array_equal(gg["Jind"], ref.Jind) and np.array_equal(gg["Ilist"], ref.Ilist)
        assert column_rel_err(ref.Jptr, gg["val"], ref.val) <= 1e-10
