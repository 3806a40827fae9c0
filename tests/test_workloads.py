"""Host-side checks of the benchmark workloads' generators (no GPU): the serving trace's
arrival rate and share of requests near an already-served parameter, and the batched
workload's sizes and pattern split."""

import numpy as np

import synth


def test_serving_trace_rate_and_update_share():
    tr = synth.serving_trace(200.0, 20.0, 16, seed=0)
    t = np.array([r[0] for r in tr])
    assert np.all(np.diff(t) > 0) and t[-1] < 20.0
    assert abs(len(tr) / 20.0 - 200.0) < 200.0 * 0.05          # Poisson count within 5 %
    gaps = np.diff(t)
    assert abs(gaps.mean() * 200.0 - 1.0) < 0.05 and abs(gaps.std() / gaps.mean() - 1.0) < 0.1  # exponential
    near = 0
    seen = []
    for _, sy, p, s, nrhs in tr:
        assert 0.1 <= p <= 1.0 and s in (0.5, 1.0, 2.0) and nrhs in (1, 4, 8) and 0 <= sy < 16
        if any(sy == a and s == c and abs(p - b) <= 0.05 for a, b, c in seen):
            near += 1
        seen.append((sy, p, s))
    # 70 % are drawn near a served (system, s, p); fresh draws land near one by chance too
    assert 0.67 <= near / len(tr) <= 0.95


def test_serving_pool_sizes():
    assert synth.SERVE_SIDES[0] == 24 and synth.SERVE_SIDES[-1] == 96 and len(synth.SERVE_SIDES) == 16
    assert synth.SERVE_SIDES == sorted(synth.SERVE_SIDES)


def test_batched_workload_sizes_and_patterns():
    ws = synth.batched_2d(256)
    sides = np.array([w.dims[0] for w in ws])
    assert sides.min() >= 48 and sides.max() <= 256
    assert [w.extra["pattern"] for w in ws[:4]] == ["A", "A2", "A", "A2"]
    assert all(0.1 <= w.params[0] <= 1.0 for w in ws)
    assert all(w.B.shape == (w.n, 4) for w in ws)
    # every system has its own seed: the K1 diagonals differ
    assert not np.array_equal(ws[0].K1[2][:100], ws[1].K1[2][:100])
