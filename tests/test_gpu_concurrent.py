"""Concurrent use of the C ABI: several contexts, each on its own stream and host thread,
sharing one base preconditioner (the way bench.py runs a shift's independent solves).

Every kernel reduces in a fixed order, so a system solved in the mix must give exactly
the bits it gives when solved alone; the sequential run is itself checked against the
oracle.
"""

import threading

import numpy as np
import pytest

import oracle
import synth
from gpu_util import context, dev_csr

pytestmark = pytest.mark.gpu


def _solve(sg, torch, ctx, stream, Ad, pc, B, restart, tol):
    n, s = B.shape
    with torch.cuda.stream(stream):
        Bd = torch.as_tensor(np.ascontiguousarray(B.T), device="cuda:0")
        Xd = torch.zeros((s, n), dtype=torch.float64, device="cuda:0")
    stream.synchronize()
    st, info, rel = sg.block_solve(ctx, Ad, pc, s, Bd, n, Xd, n, restart, tol, 50)
    stream.synchronize()
    return Xd.cpu().numpy().T.copy(), info


def test_concurrent_solves_match_sequential_bitwise():
    import torch
    import paper_1809_06574_gb300 as sg
    w = synth.grid3d_7pt(side=16, nparams=7, seed=3)
    n, s0 = w.n, w.shifts[1]
    As = [oracle.assemble(w.terms, oracle.coefficients(p, s0), n) for p in w.params]
    Ad = [dev_csr(A, n) for A in As]
    torch.cuda.synchronize()
    restart, tol = 20, 1e-8
    with context() as ctx0:
        base, _ = sg.spai_build(ctx0, Ad[0])
        main = torch.cuda.current_stream()
        # alone: one context, one system after another
        seq = []
        for i in range(len(As)):
            pc = base if i == 0 else sg.spai_update(ctx0, base, Ad[i])[0]
            seq.append(_solve(sg, torch, ctx0, main, Ad[i], pc, w.B, restart, tol))
            if i:
                sg.spai_pc_destroy(pc)
        P1 = oracle.spai_build(As[0], n)
        Pref = oracle.spai_update(P1, As[3], n)
        Xo, io = oracle.block_gmres(oracle.csr_apply(As[3], n), Pref.apply, w.B, restart, tol, 50)
        assert io["converged"] and seq[3][1]["converged"]
        assert np.linalg.norm(seq[3][0] - Xo) <= 1e-6 * np.linalg.norm(Xo)

        # in the mix: three worker threads, each with its own stream and context
        nw = 3
        out = [None] * len(As)
        errors = []
        streams = [torch.cuda.Stream(device="cuda:0") for _ in range(nw)]
        ctxs = [sg.spai_ctx_create(st.cuda_stream, 0) for st in streams]
        start = threading.Barrier(nw)

        def run(k):
            try:
                start.wait()
                for i in range(k, len(As), nw):
                    pc = base if i == 0 else sg.spai_update(ctxs[k], base, Ad[i])[0]
                    out[i] = _solve(sg, torch, ctxs[k], streams[k], Ad[i], pc, w.B, restart, tol)
                    if i:
                        sg.spai_pc_destroy(pc)
            except Exception as e:  # reported on the main thread
                errors.append(e)

        threads = [threading.Thread(target=run, args=(k,)) for k in range(nw)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        assert not errors, errors
        for k in range(nw):
            sg.spai_ctx_sync(ctxs[k])
            sg.spai_ctx_destroy(ctxs[k])
        for i in range(len(As)):
            Xs, infos = seq[i]
            Xc, infoc = out[i]
            assert infoc["converged"] and infoc["iterations"] == infos["iterations"]
            assert np.array_equal(Xc, Xs), f"system {i} differs in the mix"
        sg.spai_pc_destroy(base)
