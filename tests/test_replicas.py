"""Multi-GPU form of the benchmark: independent replicas (one sweep per rank, seeded by
its rank, no collective on the data path).  The host-side aggregation -- slowest rank's
time, all ranks' solves -- runs here on CPU with two gloo ranks; no GPU is used."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_local = [0.25, 0.75][rank]
    solves = [60, 57][rank]
    t_max, total = bench.aggregate_replicas(dist, torch, "cpu", t_local, solves)
    out[rank] = (t_max, total)
    dist.barrier()
    dist.destroy_process_group()


def test_aggregation_over_two_gloo_ranks():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
    for rank in range(2):
        t_max, total = out[rank]
        assert t_max == pytest.approx(0.75)
        assert total == pytest.approx(117.0)


def test_single_process_aggregation_is_identity():
    import bench
    assert bench.aggregate_replicas(None, torch, "cpu", 0.5, 60) == (0.5, 60.0)


def test_replicas_get_independent_inputs():
    """bench.py seeds every rank's sweep with its rank: the replicas solve different
    systems (parameters and right-hand sides) of the same shape."""
    w0 = synth.grid3d_7pt(side=8, nparams=4, seed=0)
    w1 = synth.grid3d_7pt(side=8, nparams=4, seed=1)
    assert w0.n == w1.n and w0.B.shape == w1.B.shape
    assert not np.array_equal(w0.B, w1.B)
    assert not np.allclose(w0.params, w1.params)
