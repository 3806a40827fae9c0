"""Adaptive SPAI (spai_build_adaptive) against the oracle's adaptive pattern search.

Patterns J_k, row sets I_k and column status bit-exact; entries within 1e-10 of the
largest oracle entry of their column (FP64); the update from an adaptive base (which keeps
the base's pattern, so it skips the search) against the oracle's update on the oracle's
pattern; a solve with the adaptive preconditioner.  The pattern search compares its
scores quantised to 2^-30 of ||r||^2, so both sides take the same decisions unless a score
falls within rounding of a quantisation boundary; the cases here are checked to agree."""

import numpy as np
import pytest

import oracle
import synth
from gpu_util import column_rel_err, context, dev_csr, export

pytestmark = pytest.mark.gpu


def _cases():
    out = []
    for seed in (0, 1):
        A, _ = synth.random_sparse(180 + 40 * seed, 0.03, seed=seed)
        out.append((f"random-{seed}", A, 180 + 40 * seed, dict(eps=1e-6, max_steps=3, max_new=3)))
    w = synth.grid_workload((14, 14), "5pt", seed=2, nrhs=4, params=[0.35])
    out.append(("2d-14-5pt", oracle.assemble(w.terms, oracle.coefficients(0.35, 1.0), w.n), w.n,
                dict(eps=1e-4, max_steps=5, max_new=5)))
    w = synth.grid3d_7pt(side=7, nparams=2, seed=4)
    out.append(("3d-7-7pt", oracle.assemble(w.terms, oracle.coefficients(0.5, 0.5), w.n), w.n,
                dict(eps=1e-4, max_steps=5, max_new=5)))
    w = synth.grid3d_7pt(side=6, nparams=2, seed=5)
    out.append(("3d-6-7pt-tight-rows", oracle.assemble(w.terms, oracle.coefficients(0.5, 2.0), w.n), w.n,
                dict(eps=1e-8, max_steps=6, max_new=5, max_rows=48)))
    return out


@pytest.mark.parametrize("name,A,n,opts", _cases(), ids=[c[0] for c in _cases()])
def test_adaptive_build_matches_oracle(name, A, n, opts):
    import paper_1809_06574_gb300 as sg
    ref = oracle.spai_build_adaptive(A, n, **opts)
    with context() as ctx:
        pc, st = sg.spai_build_adaptive(ctx, dev_csr(A, n), **opts)
        g = export(ctx, pc)
        sg.spai_pc_destroy(pc)
    assert st == 0
    sizes = np.diff(ref.Jptr)
    print(f"{name}: |J| mean {sizes.mean():.2f} max {sizes.max()}, |I| max {np.diff(ref.Iptr).max()}")
    for key in ("Jptr", "Jind", "Iptr", "Ilist", "status"):
        assert np.array_equal(g[key], getattr(ref, key)), key
    assert column_rel_err(ref.Jptr, g["val"], ref.val) <= 1e-10


def test_adaptive_update_and_solve():
    """P_1 adaptive at p_1; Q_2 from it (the base's pattern: no search) at p_2, against the
    oracle; the factored P_2 = Q_2 P_1 in a block GMRES solve against the oracle's."""
    import torch
    import paper_1809_06574_gb300 as sg
    w = synth.grid3d_7pt(side=9, nparams=3, seed=6)
    n = w.n
    A1 = oracle.assemble(w.terms, oracle.coefficients(w.params[0], 1.0), n)
    A2 = oracle.assemble(w.terms, oracle.coefficients(w.params[2], 1.0), n)
    P1 = oracle.spai_build_adaptive(A1, n)
    Q2 = oracle.spai_update(P1, A2, n)
    Xo, io = oracle.block_gmres(oracle.csr_apply(A2, n), Q2.apply, w.B, 30, 1e-8, 50)
    with context() as ctx:
        d1, d2 = dev_csr(A1, n), dev_csr(A2, n)
        pc1, _ = sg.spai_build_adaptive(ctx, d1)
        q2, _ = sg.spai_update(ctx, pc1, d2)
        g1, g2 = export(ctx, pc1), export(ctx, q2)
        X = np.zeros((n, w.B.shape[1]), order="F")
        st, info, rel = sg.block_solve(ctx, d2, q2, w.B.shape[1], np.asfortranarray(w.B), n, X, n, 30, 1e-8, 50)
        sg.spai_pc_destroy(q2)
        sg.spai_pc_destroy(pc1)
    for g, ref in ((g1, P1), (g2, Q2)):
        assert np.array_equal(g["Jptr"], ref.Jptr) and np.array_equal(g["Jind"], ref.Jind)
        assert column_rel_err(ref.Jptr, g["val"], ref.val) <= 1e-10
    assert info["converged"] and io["converged"]
    assert np.linalg.norm(X - Xo) <= 1e-6 * np.linalg.norm(Xo)
    print(f"adaptive 3d-9: {info['iterations']} iterations (oracle {io['iterations']})")


def test_adaptive_more_candidates_than_one_window():
    """A bordered matrix (row 0 full, n = 1,200): every column's row set holds row 0, so
    each step of every column has ~1,199 candidates, more than the kernel's window of 1,024.
    The kernel scores all of them in windows, so its patterns, row sets and entries equal
    the oracle's (which has no cap) on sampled column ranges, and the build reports no
    error."""
    import paper_1809_06574_gb300 as sg
    n = 1200
    A, _ = synth.bordered_sparse(n, 0.002, seed=7)
    opts = dict(eps=1e-10, max_steps=2, max_new=3)
    with context() as ctx:
        pc, st = sg.spai_build_adaptive(ctx, dev_csr(A, n), **opts)
        g = export(ctx, pc)
        sg.spai_pc_destroy(pc)
    assert st == 0
    for k0, k1 in ((0, 40), (600, 640), (n - 40, n)):
        Jptr, Jind = oracle.spai_adaptive_pattern(A, n, k0=k0, k1=k1, **opts)
        Iptr, Ilist = oracle.index_sets(A, n, Jptr, Jind)
        ref = oracle.spai_build(A, n, oracle.PATTERN_A, k0=k0, k1=k1, sets=(Jptr, Jind, Iptr, Ilist))
        for k in range(k0, k1):
            a, b = g["Jptr"][k], g["Jptr"][k + 1]
            assert b - a > 1, k  # the pattern grew despite the candidate count
            assert np.array_equal(g["Jind"][a:b], Jind[Jptr[k]:Jptr[k + 1]]), k
            ia, ib = g["Iptr"][k], g["Iptr"][k + 1]
            assert np.array_equal(g["Ilist"][ia:ib], Ilist[Iptr[k]:Iptr[k + 1]]), k
            got, want = g["val"][a:b], ref.val[Jptr[k]:Jptr[k + 1]]
            assert np.max(np.abs(got - want)) <= 1e-10 * np.max(np.abs(want)), k


def test_adaptive_options_are_checked():
    import paper_1809_06574_gb300 as sg
    w = synth.plain_2d_32()
    A = oracle.assemble(w.terms, oracle.coefficients(0.1, 1.0), w.n)
    with context() as ctx:
        d = dev_csr(A, w.n)
        for bad in (dict(max_steps=8, max_new=4), dict(max_rows=129), dict(max_new=0), dict(eps=-1.0)):
            with pytest.raises(sg.SpaiError) as e:
                sg.spai_build_adaptive(ctx, d, **bad)
            assert e.value.status == sg.SPAI_EINVAL
        pc, st = sg.spai_build_adaptive(ctx, d, max_steps=0)  # no growth: the diagonal pattern
        g = export(ctx, pc)
        sg.spai_pc_destroy(pc)
    assert st == 0 and np.array_equal(g["Jind"], np.arange(w.n))


def test_adaptive_full_size_sampled_columns():
    """The benchmark's matrix (3D 64^3 7-point, n = 262,144) with the default options, as
    bench.py's adaptive leg builds it: the oracle grows the patterns of three sampled column
    ranges (a boundary plane, the interior, the last plane); the GPU's patterns, row sets
    and entries on those columns match it (patterns bit-exact, entries within 1e-10)."""
    import torch
    import paper_1809_06574_gb300 as sg
    w = synth.grid3d_7pt(side=64, nparams=20)
    n = w.n
    A = oracle.assemble(w.terms, oracle.coefficients(w.params[0], w.shifts[0]), n)
    ranges = [(0, 200), (n // 2 + 31, n // 2 + 231), (n - 200, n)]
    with context() as ctx:
        pc, st = sg.spai_build_adaptive(ctx, dev_csr(A, n))
        g = export(ctx, pc)
        sg.spai_pc_destroy(pc)
    assert st == 0
    for k0, k1 in ranges:
        Jptr, Jind = oracle.spai_adaptive_pattern(A, n, k0=k0, k1=k1)
        Iptr, Ilist = oracle.index_sets(A, n, Jptr, Jind)
        ref = oracle.spai_build(A, n, oracle.PATTERN_A, k0=k0, k1=k1, sets=(Jptr, Jind, Iptr, Ilist))
        for k in range(k0, k1):
            a, b = g["Jptr"][k], g["Jptr"][k + 1]
            assert np.array_equal(g["Jind"][a:b], Jind[Jptr[k]:Jptr[k + 1]]), k
            ia, ib = g["Iptr"][k], g["Iptr"][k + 1]
            assert np.array_equal(g["Ilist"][ia:ib], Ilist[Iptr[k]:Iptr[k + 1]]), k
            got, want = g["val"][a:b], ref.val[Jptr[k]:Jptr[k + 1]]
            assert np.max(np.abs(got - want)) <= 1e-10 * np.max(np.abs(want)), k
