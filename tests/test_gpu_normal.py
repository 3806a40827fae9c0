"""The column least-squares problems by their normal equations (SPAI_LS_NORMAL): the same
minimiser as Householder QR (Sec. 2.2, and Sec. 2.4 for the update), so every factor is
compared with the oracle's QR solution -- index sets and status bit-exact, entries within
a bar set by the normal equations' error, which grows with cond(Ahat)^2 times the unit
roundoff: the test's tiles have cond(Ahat) below 4 (measured here on the oracle's tiles),
so 1e-12 in FP64 and the mixed-precision bar 5e-6 in FP32 hold with room to spare.  Tiles
beyond the normal-equations kernels (25 x 13 here) fall back to QR and give the QR build's
bits.  Exactly dependent columns are reported like QR reports them."""

import numpy as np
import pytest

import oracle
import synth
from gpu_util import column_rel_err, context, dev_csr, export

pytestmark = pytest.mark.gpu


def _sg():
    import paper_1809_06574_gb300 as sg
    return sg


def _cases():
    w2 = synth.grid_workload((14, 14), "5pt", seed=3, nrhs=4, params=[0.2, 0.7])
    w3 = synth.grid3d_7pt(side=9, nparams=3, seed=2)
    return [("2d-5pt-A", w2, oracle.PATTERN_A), ("3d-7pt-A", w3, oracle.PATTERN_A),
            ("2d-5pt-A2", w2, oracle.PATTERN_A2)]


def _max_tile_cond(A, n, P):
    """Largest condition number of the tiles A(I_k, J_k) of the oracle's factor P."""
    rp, ci, va = A
    D = np.zeros((n, n))
    for r in range(n):
        D[r, ci[rp[r]:rp[r + 1]]] = va[rp[r]:rp[r + 1]]
    worst = 1.0
    for k in range(n):
        I = P.Ilist[P.Iptr[k]:P.Iptr[k + 1]]
        J = P.Jind[P.Jptr[k]:P.Jptr[k + 1]]
        worst = max(worst, np.linalg.cond(D[np.ix_(I, J)]))
    return worst


@pytest.mark.parametrize("name,w,kind", _cases(), ids=[c[0] for c in _cases()])
@pytest.mark.parametrize("low", [0, 1], ids=["fp64", "fp32"])
def test_normal_equations_against_oracle(name, w, kind, low):
    sg = _sg()
    n = w.n
    A1 = oracle.assemble(w.terms, oracle.coefficients(w.params[0], 1.0), n)
    A2 = oracle.assemble(w.terms, oracle.coefficients(w.params[1], 1.0), n)
    P1 = oracle.spai_build(A1, n, kind)
    Q2 = oracle.spai_update(P1, A2, n)
    assert _max_tile_cond(A1, n, P1) < 4.0
    prec = sg.PREC_FP32 if low else 0
    bar = 5e-6 if low else 1e-12
    with context() as ctx:
        d1, d2 = dev_csr(A1, n), dev_csr(A2, n)
        pc, _ = sg.spai_build(ctx, d1, kind | prec | sg.LS_NORMAL)
        q, _ = sg.spai_update(ctx, pc, d2, sg.UPDATE_FIRST | prec | sg.LS_NORMAL)
        g1, g2 = export(ctx, pc), export(ctx, q)
        pq, _ = sg.spai_build(ctx, d1, kind | prec)  # QR, for the fallback's bits
        gq = export(ctx, pq)
        for h in (q, pc, pq):
            sg.spai_pc_destroy(h)
    for g, ref in ((g1, P1), (g2, Q2)):
        for key in ("Jptr", "Jind", "Iptr", "Ilist", "status"):
            assert np.array_equal(g[key], getattr(ref, key)), key
    e = max(column_rel_err(P1.Jptr, g1["val"], P1.val), column_rel_err(Q2.Jptr, g2["val"], Q2.val))
    assert e <= bar, e
    maxJ = int(np.diff(P1.Jptr).max())
    if maxJ > 8:  # no normal-equations kernel holds this tile: the QR path's own bits
        assert np.array_equal(g1["val"], gq["val"])
    print(f"{name} {'fp32' if low else 'fp64'} normal equations: {e:.1e}")


@pytest.mark.parametrize("low", [0, 1], ids=["fp64", "fp32"])
def test_normal_equations_report_dependent_columns(low):
    sg = _sg()
    D = np.array([[1.0, 1.0, 0.0], [2.0, 2.0, 0.0], [0.0, 0.0, 3.0]])
    A = synth.dense_to_csr(D, D != 0)
    ref = oracle.spai_build(A, 3)
    with context() as ctx:
        pc, st = sg.spai_build(ctx, dev_csr(A, 3), sg.PATTERN_A | sg.LS_NORMAL | (sg.PREC_FP32 if low else 0),
                               allow_singular=True)
        g = export(ctx, pc)
        sg.spai_pc_destroy(pc)
    assert st == sg.SPAI_ESINGULAR
    assert np.array_equal(g["status"], ref.status)
    bad = np.flatnonzero(ref.status)
    for k in bad:  # a rank-deficient column is set to 0
        assert not np.any(g["val"][g["Jptr"][k]:g["Jptr"][k + 1]])


def test_normal_equations_in_a_batch():
    """spai_build_batch with SPAI_LS_NORMAL: every system equals its single build bit for
    bit (one kernel per tile shape either way), FP32 and FP64 systems mixed."""
    sg = _sg()
    ws = [synth.grid_workload((d, d), "5pt", seed=60 + d, nrhs=2, params=[0.4]) for d in (11, 17, 14)]
    ws.append(synth.grid3d_7pt(side=7, nparams=1, seed=5))
    kinds = [sg.PATTERN_A | sg.LS_NORMAL, sg.PATTERN_A | sg.LS_NORMAL | sg.PREC_FP32,
             sg.PATTERN_A | sg.LS_NORMAL, sg.PATTERN_A | sg.LS_NORMAL | sg.PREC_FP32]
    As = [oracle.assemble(w.terms, oracle.coefficients(w.params[0], 1.0), w.n) for w in ws]
    with context() as ctx:
        ds = [dev_csr(A, w.n) for A, w in zip(As, ws)]
        pcs, st = sg.spai_build_batch(ctx, ds, kinds)
        assert st == 0
        got = [export(ctx, p) for p in pcs]
        single = []
        for d, k in zip(ds, kinds):
            p, _ = sg.spai_build(ctx, d, k)
            single.append(export(ctx, p))
            sg.spai_pc_destroy(p)
        for p in pcs:
            sg.spai_pc_destroy(p)
    for w, A, k, g, s1 in zip(ws, As, kinds, got, single):
        assert np.array_equal(g["val"], s1["val"])
        ref = oracle.spai_build(A, w.n, oracle.PATTERN_A)
        bar = 5e-6 if k & sg.PREC_FP32 else 1e-12
        assert column_rel_err(ref.Jptr, g["val"], ref.val) <= bar
