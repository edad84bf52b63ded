"""Continuous-batching server: every request's pairs equal the pairs of the
same request solved alone (and the oracle's), whatever else was in flight."""
import numpy as np
import pytest

import oracle
from paper_2401_11029_gb300 import gen
from paper_2401_11029_gb300.cflr import Solver
from paper_2401_11029_gb300.serve import Server, summarize

pytestmark = pytest.mark.gpu


def _requests(count, rate, lo, hi, seed):
    reqs = gen.serving_stream(n_req=count, rate=rate, seed=seed, n_lo=lo, n_hi=hi)
    return [(r.rid, r.arrival_s, r.graph()) for r in reqs]


@pytest.mark.parametrize("budget_mb", [4096, 160])
def test_served_results_equal_solved_alone(budget_mb):
    text = gen.grammar_text("fica")
    reqs = _requests(24, rate=400.0, lo=300, hi=4000, seed=55)
    srv = Server(text, mem_budget_bytes=budget_mb << 20, max_active=8, keep_pairs=True)
    try:
        done = srv.run(reqs)
    finally:
        srv.close()
    assert sorted(f.rid for f in done) == [r[0] for r in reqs]
    by_id = {r[0]: r[2] for r in reqs}
    names = oracle.parse(text).nts[:5]
    for f in done:
        g = by_id[f.rid]
        with Solver(text) as s:
            s.load(g)
            st = s.solve()
            assert st["iterations"] == f.iterations
            for x, name in enumerate(names):
                assert np.array_equal(f.keys[x], s.pairs(name)), (f.rid, name)
    for f in done[:3]:
        want = oracle.solve(text, by_id[f.rid])
        for x, name in enumerate(names):
            assert np.array_equal(f.keys[x], want.pairs[name])
    s = summarize(done)
    assert s["requests"] == len(reqs) and s["p99_s"] >= s["p50_s"] > 0
