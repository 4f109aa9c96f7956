"""Host-side serving logic (no GPU): the per-request memory estimate and the
latency/throughput summary."""
import pytest

import synthetic as S

pytest.importorskip("torch")


def test_estimate_grows_with_pixels_and_scene():
    from paper_2609_13397_b300.serving import estimate_bytes
    small = S.pinhole(160, 120, 150.0)
    big = S.pinhole(3840, 2160, 3600.0)
    assert estimate_bytes(big, 1000) > 100 * estimate_bytes(small, 1000) / 2
    assert estimate_bytes(small, 5_000_000) - estimate_bytes(small, 0) >= 5_000_000 * 128


def test_summary_percentiles_and_rate():
    from paper_2609_13397_b300.serving import Result, summarize
    res = [Result(i, 10, 10, 100, t_arrival=0.01 * i, t_admit=0.01 * i, t_done=0.01 * i + 0.001 * (i + 1))
           for i in range(100)]
    res.append(Result(100, 10, 10, 0, 1.0, 1.0, 1.0, error="ERR_ARG: bad"))
    st = summarize(res)
    assert st["requests"] == 101 and st["errors"] == 1
    assert abs(st["p50_ms"] - 51.0) < 1.01 and abs(st["p99_ms"] - 99.0) < 1.01
    assert st["rays"] == 100 * 100
    assert st["mrays_per_s"] == pytest.approx(1e4 / (0.99 + 0.1 - 0.0) / 1e6, rel=1e-6)


def test_request_stream_shape():
    reqs = list(S.c5_requests(400, rate_hz=200.0, seed=0))
    assert all(b.arrival_s > a.arrival_s for a, b in zip(reqs, reqs[1:]))
    rate = len(reqs) / reqs[-1].arrival_s
    assert 150 < rate < 260
    models = [r.camera.model for r in reqs]
    assert 0.35 < sum(models) / len(models) < 0.65
    assert min(r.camera.width for r in reqs) >= 160 and max(r.camera.width for r in reqs) <= 3840
