"""Host-side logic of the serving layer (no GPU): the Poisson request
stream and the latency summary."""
import numpy as np

from paper_2501_06121_b300 import serving as S


def test_poisson_stream_rate_mix_and_determinism():
    Q = {"a": np.zeros((50, 4), np.float32), "b": np.ones((20, 4), np.float32)}
    r1 = S.poisson_requests(10000.0, 2.0, Q, seed=3)
    r2 = S.poisson_requests(10000.0, 2.0, Q, seed=3)
    assert [(r["t"], r["index"], r["qid"], r["k"], r["ef"]) for r in r1] == \
           [(r["t"], r["index"], r["qid"], r["k"], r["ef"]) for r in r2]
    n = len(r1)
    assert abs(n - 20000) < 5 * np.sqrt(20000)        # Poisson count
    t = np.array([r["t"] for r in r1])
    assert np.all(np.diff(t) > 0) and t[-1] <= 2.0
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1e-4) < 5e-6               # exponential gaps, mean 1/rate
    assert abs(np.std(gaps) / gaps.mean() - 1.0) < 0.05
    assert {r["k"] for r in r1} == {10, 100}
    efs = np.array([r["ef"] for r in r1])
    assert efs.min() >= 64 and efs.max() <= 512
    frac_a = np.mean([r["index"] == "a" for r in r1])
    assert abs(frac_a - 0.5) < 0.02
    assert all(np.array_equal(r["query"], Q[r["index"]][r["qid"]]) for r in r1[:100])


def test_latency_summary():
    done = [{"latency": x / 1000.0} for x in range(1, 101)]
    s = S.latency_summary(done, 2.0)
    assert s["completed"] == 100 and s["qps"] == 50.0
    assert abs(s["p50_ms"] - 50.5) < 1e-9 and abs(s["p99_ms"] - 99.01) < 1e-9
    assert S.latency_summary([], 1.0) == {"completed": 0}


def test_status_counts():
    from paper_2501_06121_b300 import kann as K
    done = [{"status": 0}, {"status": K.KANN_QSTAT_HOPCAP | K.KANN_QSTAT_FORGOT}, {"status": K.KANN_QSTAT_FORGOT},
            {}]
    c = S.status_counts(done)
    assert c == {"hop_cap": 1, "forgot": 2, "bad_id": 0, "query_truncated": 0}
