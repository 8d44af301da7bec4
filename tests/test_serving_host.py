"""Host-side pieces of serving: the request record and the latency summary
(no GPU)."""

import paper_2306_07795_gb300 as bm
from paper_2306_07795_gb300 import serving


def _done(rid, arrival_ms, done_ms, n=10, e=4, status=0):
    r = serving.Request(rid, arrival_ms / 1e3, n, e, [1 << i for i in range(n)], 0, None)
    r.arrival_ms = arrival_ms
    r.done_ms = done_ms
    r.status = status
    r.late_ms = 0.0
    return r


def test_request_converts_rows_once():
    r = serving.Request(7, 0.5, 3, 8, [4, 1, 2], 5, None)
    assert list(r.rows_c) == [4, 1, 2]
    # an already converted array passes through the binding unchanged
    assert bm._binding._rows(r.rows_c) is r.rows_c


def test_summary_percentiles_and_throughput():
    # 100 requests, one per ms, latency 1 + (i % 10) / 10 ms
    reqs = [_done(i, float(i), i + 1.0 + (i % 10) / 10.0) for i in range(100)]
    reqs.append(_done(100, 100.0, 200.0, status=bm.BMMC_ERR_OOM))  # failed: not counted
    s = serving.summarize(reqs)
    assert s["requests"] == 101 and s["completed"] == 100
    assert abs(s["p50_ms"] - 1.45) < 0.06
    assert abs(s["p99_ms"] - 1.9) < 1e-9
    span_ms = (99 + 1.9) - 0.0
    assert abs(s["throughput_req_s"] - 100 / (span_ms / 1e3)) < 1e-6
    assert abs(s["effective_gbs"] - 100 * 2 * (1 << 10) * 4 / (span_ms / 1e3) / 1e9) < 1e-9
