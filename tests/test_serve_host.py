"""Host logic of the serving driver (no GPU): rate steps, Poisson schedules, summaries."""
import types

import numpy as np

from paper_2003_00575_gb300 import serve


def test_rate_steps_log_spaced():
    r = serve.rate_steps(100, 20000, 12)
    assert len(r) == 12 and abs(r[0] - 100) < 1e-9 and abs(r[-1] - 20000) < 1e-6
    ratios = np.array(r[1:]) / np.array(r[:-1])
    assert np.allclose(ratios, ratios[0])


def test_poisson_schedule_seeded_rates_and_mix():
    a = serve.poisson_schedule(4000.0, 2.0, 4, seed=7)
    b = serve.poisson_schedule(4000.0, 2.0, 4, seed=7)
    assert a == b
    ts = [t for t, _, _ in a]
    assert ts == sorted(ts) and 0 <= ts[0] and ts[-1] < 2.0
    n = len(a)
    assert abs(n - 8000) < 5 * np.sqrt(8000)          # Poisson count
    per = np.bincount([s for _, s, _ in a], minlength=4)
    assert np.all(np.abs(per - 2000) < 5 * np.sqrt(2000))
    clouds = sum(k for _, _, k in a)
    assert abs(clouds - n / 2) <= 4                    # alternating per sensor
    gaps = np.diff([t for t, s, _ in a if s == 0])
    assert abs(gaps.mean() - 1 / 1000) < 0.1 / 1000   # exponential inter-arrivals, mean 1/rate


def test_summarize_percentiles():
    # frame i waits i/2 ms for its launch and takes i/2 ms of service
    recs = [types.SimpleNamespace(t_submit=0.0, t_launch=i / 2000.0, t_done=i / 1000.0,
                                  batch_size=2, status=0) for i in range(1, 101)]
    s = serve.summarize(recs, 0.0, 1.0)
    assert s["completed"] == 100 and s["frames_per_s"] == 100.0
    assert abs(s["latency_ms_p50"] - 50.5) < 1e-6 and s["latency_ms_max"] == 100.0
    assert abs(s["queue_ms_p50"] - 25.25) < 1e-6 and abs(s["service_ms_p50"] - 25.25) < 1e-6
    assert s["queue_ms_p99"] <= s["latency_ms_p99"]
    assert serve.summarize([], 0, 1) == {"completed": 0}
