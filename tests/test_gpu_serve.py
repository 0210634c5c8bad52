"""Served stream: requests that overlap on the GPU give the same result as alone."""
import numpy as np
import pytest

from paper_2107_09879_b300 import workloads as W

pytestmark = pytest.mark.gpu


def test_results_same_alone_and_in_the_mix():
    from paper_2107_09879_b300 import serve
    reqs = W.served_stream(6, seed=W.BASE_SEED + 3, rate_per_s=1000.0, k_lo=6, k_hi=14)
    srv = serve.Server(slots=3, mem_budget=4 << 30)
    mixed = srv.run(reqs, keep_solutions=True)
    srv.close()
    assert all("E" in r and r["rc"] == 0 for r in mixed), mixed
    # the runs overlapped: some request was admitted before another one finished
    assert any(a["admit"] < b["finish"] and b["admit"] < a["finish"] for a in mixed for b in mixed if a is not b)
    for req in reqs:
        alone = serve.Server(slots=1, mem_budget=4 << 30)
        req1 = dict(req, arrival=0.0)
        rec = alone.run([req1], keep_solutions=True)[0]
        alone.close()
        mix = mixed[req["rid"]]
        assert np.array_equal(rec["E"], mix["E"])
        assert np.array_equal(rec["s"], mix["s"])


def test_admission_respects_memory_budget():
    """The sum of the memory estimates of the requests in flight never exceeds the
    budget; a budget that fits one request at a time serialises the stream."""
    from paper_2107_09879_b300 import serve
    reqs = W.served_stream(5, seed=W.BASE_SEED + 4, rate_per_s=1000.0, k_lo=8, k_hi=8)
    for r in reqs:
        r["nmax"] = 4  # equal estimates: a budget of one request admits one at a time
    est = [serve.request_bytes(r["side"], r["nmax"]) for r in reqs]
    budget = max(est)
    assert 2 * min(est) > budget  # so no two requests fit together
    srv = serve.Server(slots=4, mem_budget=budget)
    recs = srv.run(reqs)
    srv.close()
    assert all("E" in r for r in recs)
    assert srv.mem_high <= budget
    spans = sorted((r["admit"], r["finish"]) for r in recs)
    assert all(spans[i][1] <= spans[i + 1][0] + 1e-3 for i in range(len(spans) - 1))  # one at a time
