"""Helpers for the GPU tests: move seeded CSR inputs to the device and read results back.

Only marshalling lives here; every computation under test runs through the C ABI of
libspai_gb300 (via the ctypes binding), and every expected value comes from the oracle.
"""

import contextlib

import numpy as np

DEV = "cuda:0"


def torch_mod():
    import torch
    return torch


@contextlib.contextmanager
def context(mem_budget=0):
    import paper_1809_06574_gb300 as sg
    torch = torch_mod()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctx = sg.spai_ctx_create(stream.cuda_stream, mem_budget)
    try:
        yield ctx
    finally:
        sg.spai_ctx_sync(ctx)
        sg.spai_ctx_destroy(ctx)


def dev_csr(A, n):
    """spai_csr over device copies of the numpy CSR triplet A (keeps the tensors alive)."""
    import paper_1809_06574_gb300 as sg
    torch = torch_mod()
    rp = torch.as_tensor(np.ascontiguousarray(A[0], dtype=np.int32), device=DEV)
    ci = torch.as_tensor(np.ascontiguousarray(A[1], dtype=np.int32), device=DEV)
    va = torch.as_tensor(np.ascontiguousarray(A[2], dtype=np.float64), device=DEV)
    return sg.csr(n, rp, ci, va, nnz=len(A[1]))


def export(ctx, pc):
    """All of a handle's exported arrays as numpy."""
    import paper_1809_06574_gb300 as sg
    torch = torch_mod()
    info = sg.spai_pc_info(pc)
    n, nnz, nI = info["n"], info["nnz"], info["nI"]
    Jptr = torch.empty(n + 1, dtype=torch.int32, device=DEV)
    Jind = torch.empty(max(nnz, 1), dtype=torch.int32, device=DEV)
    val = torch.empty(max(nnz, 1), dtype=torch.float64, device=DEV)
    Iptr = torch.empty(n + 1, dtype=torch.int32, device=DEV)
    Ilist = torch.empty(max(nI, 1), dtype=torch.int32, device=DEV)
    st = torch.empty(max(n, 1), dtype=torch.int32, device=DEV)
    sg.spai_pc_export(ctx, pc, Jptr, Jind, val, Iptr, Ilist, st)
    sg.spai_ctx_sync(ctx)
    return {"Jptr": Jptr.cpu().numpy(), "Jind": Jind.cpu().numpy()[:nnz],
            "val": val.cpu().numpy()[:nnz], "Iptr": Iptr.cpu().numpy(),
            "Ilist": Ilist.cpu().numpy()[:nI], "status": st.cpu().numpy()[:n], **info}


def column_rel_err(Jptr, got, ref):
    """max over columns of max|got - ref| / max|ref| within the column (0 for empty)."""
    worst = 0.0
    for k in range(len(Jptr) - 1):
        a, b = Jptr[k], Jptr[k + 1]
        if a == b:
            continue
        scale = np.max(np.abs(ref[a:b]))
        d = np.max(np.abs(got[a:b] - ref[a:b]))
        if scale == 0:
            worst = max(worst, d)
        else:
            worst = max(worst, d / scale)
    return worst


def column_rel_err_vec(Jptr, got, ref):
    """Vectorised column_rel_err for large patterns."""
    lens = np.diff(Jptr)
    keep = lens > 0
    idx = np.repeat(np.arange(len(lens)), lens)
    scale = np.zeros(len(lens))
    np.maximum.at(scale, idx, np.abs(ref))
    diff = np.zeros(len(lens))
    np.maximum.at(diff, idx, np.abs(got - ref))
    s = np.where(scale[keep] > 0, scale[keep], 1.0)
    return float(np.max(diff[keep] / s)) if keep.any() else 0.0
