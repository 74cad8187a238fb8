"""Host logic of the serving loop on CPU: the seeded Poisson request trace
the served benchmark replays, and the latency statistics it reports."""
import math
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from paper_2507_19718_gb300 import serve  # noqa: E402


def test_poisson_trace_rate_mix_and_seed():
    rate, duration, scenes = 2000.0, 5.0, 8
    tr = serve.poisson_trace(rate, duration, scenes, seed=11, tf_fraction=0.1)
    n = len(tr)
    # Poisson count: mean and variance rate x duration (10,000); 5 sigma
    assert abs(n - rate * duration) < 5 * math.sqrt(rate * duration)
    t = np.array([r.arrival for r in tr])
    assert np.all(np.diff(t) > 0) and t[0] > 0 and t[-1] < duration
    # exponential gaps: mean 1/rate, coefficient of variation 1
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() * rate - 1) < 5 / math.sqrt(n)
    assert abs(gaps.std() / gaps.mean() - 1) < 0.05
    tf = [r for r in tr if r.kind == "tf"]
    views = [r for r in tr if r.kind == "view"]
    p = len(tf) / n
    assert abs(p - 0.1) < 5 * math.sqrt(0.1 * 0.9 / n)
    assert {(r.width, r.height) for r in views} == set(serve.VIEW_RESOLUTIONS)
    assert {r.scene for r in tr} == set(range(scenes))
    assert all(0.0 <= r.angle < 360.0 for r in views)
    assert [r.rid for r in tr] == list(range(n))
    again = serve.poisson_trace(rate, duration, scenes, seed=11, tf_fraction=0.1)
    assert [(r.kind, r.scene, r.arrival, r.width, r.tf_seed) for r in again] == \
           [(r.kind, r.scene, r.arrival, r.width, r.tf_seed) for r in tr]
    assert serve.poisson_trace(rate, duration, scenes, seed=12)[0].arrival != tr[0].arrival


def test_latency_stats_of_a_known_trace():
    tr = []
    for i in range(200):
        r = serve.Request(i, "view", 0, arrival=0.01 * i)
        r.done = r.arrival + 0.001 * (i + 1)   # latencies 1 .. 200 ms
        tr.append(r)
    lost = serve.Request(200, "view", 0, arrival=3.0)          # never completed: not counted
    tf = serve.Request(201, "tf", 0, arrival=3.0)
    tf.done = 3.5
    s = serve.latency_stats(tr + [lost, tf])
    lat = np.arange(1, 201, dtype=np.float64)
    assert s["n"] == 200
    assert math.isclose(s["p50_ms"], np.percentile(lat, 50), rel_tol=1e-9)
    assert math.isclose(s["p99_ms"], np.percentile(lat, 99), rel_tol=1e-9)
    assert math.isclose(s["max_ms"], 200.0, rel_tol=1e-9)
    assert serve.latency_stats(tr + [tf], kind="tf")["p50_ms"] == 500.0
    assert serve.latency_stats([lost]) == {"n": 0}
