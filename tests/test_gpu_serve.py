"""Request server (the "Serving" part of the C ABI): requests for several parametric
systems run concurrently on several slots, routed to a new SPAI build, an update of a
cached build (Table 1, first approach) or a cached build itself.

The server adds no arithmetic of its own, and every kernel reduces in a fixed order, so a
request served in the mix must give exactly the bits of the same route (build at its base
parameter, update, solve) run alone through the plain entry points; those are checked
against the oracle.
"""

import numpy as np
import pytest

import oracle
import synth
from gpu_util import context, dev_csr

pytestmark = pytest.mark.gpu

RESTART, TOL = 20, 1e-8


def _systems(sides=(8, 10, 12), seed=5):
    return [synth.grid_workload((d, d, d), "7pt", seed=seed + i, nrhs=8, params=[0.5]) for i, d in enumerate(sides)]


def _trace(nreq, nsys, seed=11, near=0.7):
    """(system, p, s, nrhs) requests: a share `near` lies within 0.05 of an earlier p."""
    rng = np.random.default_rng(seed)
    out, seen = [], []
    for _ in range(nreq):
        if seen and rng.random() < near:
            sy, p0, s = seen[rng.integers(len(seen))]
            p = float(np.clip(p0 + rng.uniform(-0.05, 0.05), 0.1, 1.0))
        else:
            sy, p, s = int(rng.integers(nsys)), float(rng.uniform(0.1, 1.0)), float(rng.choice([0.5, 1.0, 2.0]))
        seen.append((sy, p, s))
        out.append((sy, p, s, int(rng.choice([1, 4, 8]))))
    return out


def _plain_route(sg, ctx, w, res, p, s, nrhs):
    """The request's route through the plain calls, alone: build at base_p, update to p, solve."""
    n = w.n
    A_base = oracle.assemble(w.terms, oracle.coefficients(res["base_p"], s), n)
    A = oracle.assemble(w.terms, oracle.coefficients(p, s), n)
    Ab, Ad = dev_csr(A_base, n), dev_csr(A, n)
    base, _ = sg.spai_build(ctx, Ab)
    pc = base
    if res["route"] == sg.ROUTE_UPDATE:
        pc, _ = sg.spai_update(ctx, base, Ad)
    X = np.zeros((n, nrhs), order="F")
    B = np.asfortranarray(w.B[:, :nrhs])
    sg.block_solve(ctx, Ad if res["route"] != sg.ROUTE_BUILD else Ab, pc, nrhs, B, n, X, n, RESTART, TOL, 50)
    if pc is not base:
        sg.spai_pc_destroy(pc)
    sg.spai_pc_destroy(base)
    return X, A


def _serve(sg, systems, trace, **kw):
    srv = sg.spai_server_create(restart=RESTART, tol=TOL, **kw)
    try:
        ids = [sg.spai_server_add_shifted_system(srv, [sg.csr(w.n, *t) for t in w.terms], w.alpha, w.beta) for w in systems]
        Bs = [np.asfortranarray(w.B) for w in systems]
        Xs, tickets = [], []
        for sy, p, s, nrhs in trace:
            w = systems[sy]
            X = np.zeros((w.n, nrhs), order="F")
            Xs.append(X)
            tickets.append(sg.spai_server_submit(srv, ids[sy], nrhs, p, s, None,
                                                 Bs[sy], X))
        res = [sg.spai_server_wait(srv, t) for t in tickets]
        stats = sg.spai_server_stats_get(srv)
    finally:
        sg.spai_server_destroy(srv)
    return res, Xs, stats


def test_served_requests_equal_their_route_alone_and_the_oracle():
    import paper_1809_06574_gb300 as sg
    systems = _systems()
    trace = _trace(30, len(systems))
    res, Xs, stats = _serve(sg, systems, trace, slots=3, reuse=True, radius=0.05)
    assert stats["completed"] == len(trace) and stats["failed"] == 0
    assert stats["builds"] + stats["updates"] + stats["reuses"] == len(trace)
    assert stats["updates"] > 0 and stats["builds"] > 0
    assert len({r["slot"] for r in res}) > 1  # the mix really ran on several slots
    with context() as ctx:
        for i, ((sy, p, s, nrhs), r, X) in enumerate(zip(trace, res, Xs)):
            assert r["status"] == 0, (i, r)
            assert r["max_rel_residual"] <= TOL
            if r["route"] == sg.ROUTE_BUILD:
                assert r["base_p"] == p
            else:
                assert abs(r["base_p"] - p) <= 0.05
            w = systems[sy]
            Xa, A = _plain_route(sg, ctx, w, r, p, s, nrhs)
            assert np.array_equal(X, Xa), f"request {i} differs from its route run alone"
            # independent FP64 check of the true residual
            rel = np.linalg.norm(w.B[:, :nrhs] - oracle.spmm(A, X, w.n), axis=0) / np.linalg.norm(w.B[:, :nrhs], axis=0)
            assert np.all(rel <= TOL), (i, rel)
    # two requests against the oracle's own build / update / block GMRES
    for i in [k for k, r in enumerate(res) if r["route"] == sg.ROUTE_UPDATE][:2]:
        sy, p, s, nrhs = trace[i]
        w = systems[sy]
        A1 = oracle.assemble(w.terms, oracle.coefficients(res[i]["base_p"], s), w.n)
        A = oracle.assemble(w.terms, oracle.coefficients(p, s), w.n)
        Q = oracle.spai_update(oracle.spai_build(A1, w.n), A, w.n)
        Xo, io = oracle.block_gmres(oracle.csr_apply(A, w.n), Q.apply, w.B[:, :nrhs], RESTART, TOL, 50)
        assert io["converged"]
        assert np.linalg.norm(Xs[i] - Xo) <= 1e-6 * np.linalg.norm(Xo)


def test_plain_mode_builds_every_request_and_fp32_factors_converge():
    import paper_1809_06574_gb300 as sg
    systems = _systems(sides=(8, 9))
    trace = _trace(10, len(systems), seed=3)
    res, Xs, stats = _serve(sg, systems, trace, slots=1, reuse=False)
    assert stats["builds"] == len(trace) and stats["updates"] == 0 and stats["cached_builds"] == 0
    assert all(r["route"] == sg.ROUTE_BUILD and r["status"] == 0 for r in res)
    # FIFO on one slot: requests start in arrival order
    starts = [r["t_start"] for r in res]
    assert starts == sorted(starts)
    # FP32 factors, by QR and by the normal equations (SPAI_LS_NORMAL), each with the
    # mixed-precision solve too: every solution meets tol and the FP64 solution's bar
    for kind, prec in ((sg.PREC_FP32, sg.SOLVE_FP64), (sg.PREC_FP32 | sg.LS_NORMAL, sg.SOLVE_FP64),
                       (sg.PREC_FP32 | sg.LS_NORMAL, sg.SOLVE_MIXED)):
        res32, Xs32, _ = _serve(sg, systems, trace, slots=2, reuse=True, pattern_kind=kind, precision=prec)
        for (sy, p, s, nrhs), r, X, X64 in zip(trace, res32, Xs32, Xs):
            assert r["status"] == 0 and r["max_rel_residual"] <= TOL
            w = systems[sy]
            A = oracle.assemble(w.terms, oracle.coefficients(p, s), w.n)
            rel = np.linalg.norm(w.B[:, :nrhs] - oracle.spmm(A, X, w.n), axis=0) / np.linalg.norm(w.B[:, :nrhs], axis=0)
            assert np.all(rel <= TOL)
            assert np.linalg.norm(X - X64) <= 1e-6 * np.linalg.norm(X64)


def test_memory_budget_evicts_and_refuses():
    import paper_1809_06574_gb300 as sg
    systems = _systems(sides=(10,))
    w = systems[0]
    # distinct p far apart (radius 0.01): every request builds and caches its own base
    trace = [(0, p, 1.0, 4) for p in (0.1, 0.3, 0.5, 0.7, 0.9, 0.2, 0.4)]
    res0, _, st0 = _serve(sg, systems, trace, slots=1, reuse=True, radius=0.01)
    assert st0["cached_builds"] == len(trace) and st0["evictions"] == 0
    with context() as ctx:
        pc, _ = sg.spai_build(ctx, dev_csr(oracle.assemble(w.terms, oracle.coefficients(0.1, 1.0), w.n), w.n))
        build_bytes = sg.spai_pc_mem_size(pc, True)
        sg.spai_pc_destroy(pc)
    fixed = st0["mem_in_use"] - len(trace) * build_bytes  # the system and the slot's buffers
    # one slot (no idle workspace to release): room for four builds and the transient
    # pattern-analysis reservation of the build in flight (16 nnz + 16 (n + 1) + 1 MiB):
    # at most three cached while one is built
    nnz = int(oracle.assemble(w.terms, oracle.coefficients(0.1, 1.0), w.n)[0][-1])
    transient = 16 * nnz + 16 * (w.n + 1) + (1 << 20)
    budget = fixed + 4 * build_bytes + transient
    res, Xs, stats = _serve(sg, systems, trace, slots=1, reuse=True, radius=0.01, mem_budget=budget)
    assert all(r["status"] == 0 for r in res), res
    assert stats["mem_peak"] <= budget
    assert stats["evictions"] >= 3 and stats["cached_builds"] <= 4
    for X, X0 in zip(Xs, _serve(sg, systems, trace, slots=1, reuse=True, radius=0.01)[1]):
        assert np.array_equal(X, X0)  # eviction changes nothing in the results (same routes)
    # a budget below one request's workspace: the request fails with SPAI_ENOMEM, the server survives
    ws = sg.spai_solve_workspace_size(w.n, 4, RESTART)
    res2, _, stats2 = _serve(sg, systems, trace[:2], slots=2, reuse=True, mem_budget=ws // 2)
    assert all(r["status"] == sg.SPAI_ENOMEM for r in res2)
    assert stats2["failed"] == 2


def test_fullsize_served_trace():
    """The serving workload at full size for one second of arrivals (200 requests/s over the
    16-grid pool, n up to 884,736, FP32 factors, 40 GiB budget, 4 slots), submitted at once:
    every request converges; for a sample (one per system that has a request) the
    solution's true residual is recomputed on the host and the route is checked."""
    import paper_1809_06574_gb300 as sg
    pool = synth.serving_pool()
    trace = synth.serving_trace(200.0, 1.0, len(pool))
    srv = sg.spai_server_create(slots=4, reuse=True, radius=0.05, pattern_kind=sg.PREC_FP32, restart=30,
                                max_cycles=100, tol=TOL, mem_budget=40 << 30)
    try:
        ids = [sg.spai_server_add_shifted_system(srv, [sg.csr(w.n, *t) for t in w.terms], w.alpha, w.beta) for w in pool]
        Bs = [np.asfortranarray(w.B) for w in pool]
        sampled, tickets, Xs = set(), [], {}
        for k, (_, sy, p, s, nrhs) in enumerate(trace):
            X = None
            if sy not in sampled:
                sampled.add(sy)
                X = np.zeros((pool[sy].n, nrhs), order="F")
                Xs[k] = X
            tickets.append(sg.spai_server_submit(srv, ids[sy], nrhs, p, s, None, Bs[sy], X))
        res = [sg.spai_server_wait(srv, t) for t in tickets]
        stats = sg.spai_server_stats_get(srv)
    finally:
        sg.spai_server_destroy(srv)
    assert stats["failed"] == 0 and stats["mem_peak"] <= 40 << 30
    assert all(r["status"] == 0 and r["max_rel_residual"] <= TOL for r in res)
    assert stats["updates"] > 0
    for k, X in Xs.items():
        _, sy, p, s, nrhs = trace[k]
        w, r = pool[sy], res[k]
        assert r["route"] == sg.ROUTE_BUILD and r["base_p"] == p  # first request of its system builds
        A = oracle.assemble(w.terms, oracle.coefficients(p, s), w.n)
        rel = np.linalg.norm(w.B[:, :nrhs] - oracle.spmm(A, X, w.n), axis=0) / np.linalg.norm(w.B[:, :nrhs], axis=0)
        assert np.all(rel <= TOL), (k, rel)


def test_failed_requests_do_not_stop_the_server():
    """A restart length and cycle cap too small to reach the tolerance: every request
    completes with SPAI_ENOTCONV and its residual report, the server keeps serving, and a
    second server with the normal settings solves the same requests."""
    import paper_1809_06574_gb300 as sg
    systems = _systems(sides=(8, 9))
    trace = _trace(6, len(systems), seed=9)
    srv = sg.spai_server_create(slots=2, restart=1, max_cycles=1, tol=1e-12, reuse=True)
    try:
        ids = [sg.spai_server_add_shifted_system(srv, [sg.csr(w.n, *t) for t in w.terms], w.alpha, w.beta) for w in systems]
        Bs = [np.asfortranarray(w.B) for w in systems]  # read by the workers: kept alive here
        tickets = [sg.spai_server_submit(srv, ids[sy], nrhs, p, s, None, Bs[sy])
                   for sy, p, s, nrhs in trace]
        res = [sg.spai_server_wait(srv, t) for t in tickets]
        stats = sg.spai_server_stats_get(srv)
        assert "request" in sg.spai_server_last_error(srv)
    finally:
        sg.spai_server_destroy(srv)
    assert all(r["status"] == sg.SPAI_ENOTCONV and r["max_rel_residual"] > 1e-12 for r in res)
    assert stats["failed"] == len(trace) and stats["completed"] == len(trace)
    res2, _, st2 = _serve(sg, systems, trace, slots=2, reuse=True)
    assert all(r["status"] == 0 for r in res2) and st2["failed"] == 0
