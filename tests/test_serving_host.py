"""Host-side serving logic (no GPU): memory admission and the latency/throughput
summary."""
import pytest

import synthetic as S

pytest.importorskip("torch")


def test_memory_gate_admits_within_budget_without_head_of_line_blocking():
    """A request whose memory does not fit waits; a later, smaller one that fits is
    admitted past it; the waiting one runs once memory frees up; a request larger
    than the whole budget runs alone."""
    import threading
    import time
    from paper_2609_13397_b300.serving import MemoryGate
    gate = MemoryGate(100)
    assert gate.acquire(60)                       # in flight: 60
    order = []
    big = threading.Thread(target=lambda: (gate.acquire(70), order.append("big")))
    big.start()
    time.sleep(0.2)
    assert order == []                            # 60 + 70 > 100: waits
    assert gate.acquire(30)                       # 60 + 30 fits: passes the waiting one
    order.append("small")
    gate.release(60)
    gate.release(30)
    big.join(2.0)
    assert order == ["small", "big"] and gate.in_use == 70
    gate.release(70)
    assert gate.acquire(500) and gate.in_use == 500   # larger than the budget: alone
    gate.release(500)
    assert gate.in_use == 0


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
