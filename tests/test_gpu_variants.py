"""Every column-kernel variant (shared-memory teams of 1 ... 32 lanes, register-tiled
kernels) on its own: the variant is pinned with spai_column_variant_set, and the build
and the update it computes are compared with the oracle -- index sets and status
bit-exact, entries within 1e-10 of the largest oracle entry of their column (FP64) or
within the FP32 bar of the mixed-precision tests (5e-6 for the stencils).  The autotuner
picks one of these variants per shape by timing, so each must be correct on its own."""

import numpy as np
import pytest

import oracle
import synth
from gpu_util import column_rel_err, context, dev_csr, export

pytestmark = pytest.mark.gpu


def _cases():
    out = []
    w = synth.grid_workload((14, 14), "5pt", seed=3, nrhs=4, params=[0.2, 0.7])
    out.append(("2d-5pt-A", w, oracle.PATTERN_A))
    out.append(("2d-5pt-A2", w, oracle.PATTERN_A2))
    out.append(("3d-7pt-A", synth.grid3d_7pt(side=9, nparams=3, seed=2), oracle.PATTERN_A))
    out.append(("3d-27pt-A", synth.grid3d_27pt(side=6, nparams=3, seed=2), oracle.PATTERN_A))
    return out


@pytest.mark.parametrize("name,w,kind", _cases(), ids=[c[0] for c in _cases()])
@pytest.mark.parametrize("low", [0, 1], ids=["fp64", "fp32"])
def test_every_variant_against_oracle(name, w, kind, low):
    import paper_1809_06574_gb300 as sg
    n = w.n
    A1 = oracle.assemble(w.terms, oracle.coefficients(w.params[0], 1.0), n)
    A2 = oracle.assemble(w.terms, oracle.coefficients(w.params[1], 1.0), n)
    P1 = oracle.spai_build(A1, n, kind)
    Q2 = oracle.spai_update(P1, A2, n)
    maxI, maxJ = int(np.diff(P1.Iptr).max()), int(np.diff(P1.Jptr).max())
    codes = sg.spai_column_variants(low, maxI, maxJ)
    assert codes
    bar = 5e-6 if low else 1e-10
    prec = sg.PREC_FP32 if low else 0
    before = sg.spai_column_variant_get(low, maxI, maxJ)
    errs = {}
    try:
        with context() as ctx:
            d1, d2 = dev_csr(A1, n), dev_csr(A2, n)
            for code in codes:
                sg.spai_column_variant_set(low, maxI, maxJ, code)
                pc, _ = sg.spai_build(ctx, d1, kind | prec)
                q, _ = sg.spai_update(ctx, pc, d2, sg.UPDATE_FIRST | prec)
                g1, g2 = export(ctx, pc), export(ctx, q)
                sg.spai_pc_destroy(q)
                sg.spai_pc_destroy(pc)
                for g, ref in ((g1, P1), (g2, Q2)):
                    for key in ("Jptr", "Jind", "Iptr", "Ilist", "status"):
                        assert np.array_equal(g[key], getattr(ref, key)), (code, key)
                e = max(column_rel_err(P1.Jptr, g1["val"], P1.val), column_rel_err(Q2.Jptr, g2["val"], Q2.val))
                errs[code] = e
                assert e <= bar, (code, e)
    finally:
        sg.spai_column_variant_set(low, maxI, maxJ, before)
    print(f"{name} {'fp32' if low else 'fp64'} {maxI}x{maxJ}:",
          ", ".join(f"{c}: {e:.1e}" for c, e in errs.items()))
