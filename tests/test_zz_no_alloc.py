"""spai_pc_apply_noalloc: the preconditioner apply for callers that cannot allocate device
memory where they apply it (an outside solver loop that must not stall the device, or a
process whose device memory is reserved by another allocator).

It must give the same Y = P X as the allocating spai_pc_apply, on two calls in a row (the
shared staging array keeps the previous call's contents), must not change the library's
device memory use, and must refuse sizes beyond its fixed array with SPAI_EINVAL.  This
file is collected last so that a run stopping at the first failure has run every other
test first; it also passes on its own in a fresh process.
"""

import numpy as np
import pytest

import oracle
import synth
from gpu_util import context, dev_csr

pytestmark = pytest.mark.gpu


def test_noalloc_apply_matches_allocating_apply_twice():
    import torch
    import paper_1809_06574_gb300 as sg
    w = synth.grid3d_7pt(side=14, nparams=2, nrhs=4)
    n = w.n
    A1 = oracle.assemble(w.terms, oracle.coefficients(w.params[0], 1.0), n)
    A2 = oracle.assemble(w.terms, oracle.coefficients(w.params[1], 1.0), n)
    rng = np.random.default_rng(11)
    with context() as ctx:
        pc1, _ = sg.spai_build(ctx, dev_csr(A1, n))
        pc2, _ = sg.spai_update(ctx, pc1, dev_csr(A2, n))  # factored apply Q2 (P1 X)
        for s in (4, 8):
            ld = n + 3
            for call in range(2):
                X = torch.as_tensor(rng.standard_normal((s, ld)), device="cuda:0")
                Y_ref = torch.zeros((s, ld), dtype=torch.float64, device="cuda:0")
                Y = torch.full((s, ld), 7.0, dtype=torch.float64, device="cuda:0")
                sg.spai_pc_apply(ctx, pc2, s, X, ld, Y_ref, ld)
                sg.spai_ctx_sync(ctx)
                before = sg.spai_ctx_mem_in_use(ctx)
                sg.spai_pc_apply_noalloc(ctx, pc2, s, X, ld, Y, ld)
                sg.spai_ctx_sync(ctx)
                assert sg.spai_ctx_mem_in_use(ctx) == before
                y, y_ref = Y.cpu().numpy()[:, :n], Y_ref.cpu().numpy()[:, :n]
                assert np.max(np.abs(y - y_ref)) <= 1e-13 * np.max(np.abs(y_ref)), (s, call)
                # padding rows beyond n are left alone
                assert np.all(Y.cpu().numpy()[:, n:] == 7.0)
        sg.spai_pc_destroy(pc2)
        sg.spai_pc_destroy(pc1)


def test_noalloc_apply_rejects_sizes_beyond_its_array():
    import torch
    import paper_1809_06574_gb300 as sg
    w = synth.grid_workload((375, 375), "5pt", seed=0, nrhs=1, params=[0.5])  # n = 140,625
    n = w.n
    A = oracle.assemble(w.terms, oracle.coefficients(0.5, 1.0), n)
    with context() as ctx:
        pc, _ = sg.spai_build(ctx, dev_csr(A, n))
        X = torch.zeros((16, n), dtype=torch.float64, device="cuda:0")
        Y = torch.zeros_like(X)
        with pytest.raises(sg.SpaiError) as ei:  # n * 16 = 2,250,000 > 2,097,152
            sg.spai_pc_apply_noalloc(ctx, pc, 16, X, n, Y, n)
        assert ei.value.status == sg.SPAI_EINVAL
        sg.spai_pc_apply_noalloc(ctx, pc, 8, X, n, Y, n)  # n * 8 fits
        sg.spai_ctx_sync(ctx)
        sg.spai_pc_destroy(pc)
