"""Host logic of the served form that needs no GPU: the seeded session generator."""
import numpy as np

from paper_1611_03631_gb300 import serve


def _sessions(n=4000, rate=32.0, seed=5):
    return serve.poisson_sessions(
        n,
        ["room", "lidar_terrain"],
        {"room": 3, "lidar_terrain": 2},
        {"room": 8, "lidar_terrain": 8},
        sessions_per_s=rate,
        scans_per_session=16,
        seed=seed,
    )


def test_sessions_are_seeded_and_arrive_as_a_poisson_process():
    a, b = _sessions(), _sessions()
    assert [(s.kind, s.seq, s.offset, s.start, s.rate_hz) for s in a] == [(s.kind, s.seq, s.offset, s.start, s.rate_hz) for s in b]
    assert _sessions(seed=6)[0].start != a[0].start
    t = np.array([s.start for s in a])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert (gaps > 0).all()
    # exponential inter-arrival times: mean 1/rate and coefficient of variation 1
    assert abs(gaps.mean() * 32.0 - 1.0) < 0.05
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.08


def test_sessions_stay_inside_the_pool_and_rate_range():
    ss = _sessions()
    kinds = [s.kind for s in ss]
    assert set(kinds) == {"room", "lidar_terrain"}
    assert abs(kinds.count("room") / len(kinds) - 0.5) < 0.05
    for s in ss:
        assert 0 <= s.seq < (3 if s.kind == "room" else 2)
        assert 0 <= s.offset < 8
        assert 10.0 <= s.rate_hz <= 30.0
        assert s.n_scans == 16
    assert [s.sid for s in ss] == list(range(len(ss)))
