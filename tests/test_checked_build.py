"""The bounds-checked build (libcflr_checked.so, CFLR_CHECKED): the product
kernels and the merge test every index that comes from data before they use
it, and a failed test ends the solve with CFLR_ECUDA.  These runs load that
library in a child process (CFLR_LIBRARY=checked) and require the oracle's
pairs on workloads that reach every kernel path: plain and family groups, the
split of large families, growth of every buffer, the graph form, a batch of
instances, epsilon and unit productions.  No check may fire on them."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
sys.path.insert(0, "tests")
import numpy as np
import oracle
from paper_2401_11029_gb300 import cflr, gen
from paper_2401_11029_gb300.cflr import Solver
assert cflr.LIB_PATH.endswith("libcflr_checked.so"), cflr.LIB_PATH

def check(text, g, **cfg):
    want = oracle.solve(text, g)
    with Solver(text, **cfg) as s:
        s.load(g)
        s.solve()
        for x in want.grammar.nts:
            assert np.array_equal(s.pairs(x), want.pairs[x]), x

check(gen.grammar_text("fica"), gen.fica_like(n=6000, n_a=12_000, n_d=4500, seed=31),
      form=cflr.CFLR_FORM_GRAPH)
check(gen.grammar_text("fica"), gen.fica_like(n=5000, n_a=10_000, n_d=3750, seed=11),
      initial_capacity=64)
check(gen.grammar_text("fsjpt"), gen.fsjpt_like(n=6000, n_edges=24_000, fields=64, seed=13))
with Solver(gen.grammar_text("fsjpt")) as s:       # large families split into members
    cflr.cflr_set_tuning(s.ctx, 1, [16, 64, 256], [1, 1, 1, 1])
    g = gen.fsjpt_like(n=6000, n_edges=24_000, fields=64, seed=13)
    want = oracle.solve(gen.grammar_text("fsjpt"), g)
    s.load(g)
    s.solve()
    for x in want.grammar.nts[:want.grammar.n_user]:
        assert np.array_equal(s.pairs(x), want.pairs[x]), x
check(gen.grammar_text("fsca", index_hi=63), gen.fsca_like(n=3000, n_edges=4000, fields=64, seed=21))
check(gen.grammar_text("cscvf", index_hi=255),
      gen.cscvf_like(n=4000, n_edges=6700, calls=256, seed=22), form=cflr.CFLR_FORM_GRAPH)
check(gen.grammar_text("dyck1"), gen.dyck1_er())
text = gen.grammar_text("dyck3")
graphs = gen.dyck3_batch(count=6, seed0=4200, n_lo=500, n_hi=3000)
solvers = [Solver(text, form=cflr.CFLR_FORM_GRAPH) for _ in graphs]
for s, g in zip(solvers, graphs):
    s.load(g)
cflr.cflr_solve_batch([s.ctx for s in solvers])
for s, g in zip(solvers, graphs):
    want = oracle.solve(text, g)
    for x in want.grammar.nts:
        assert np.array_equal(s.pairs(x), want.pairs[x]), x
    s.close()
print("checked build: all parity cases clean")
'''


def test_checked_build_runs_clean_and_exact():
    env = dict(os.environ, CFLR_LIBRARY="checked")
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "all parity cases clean" in r.stdout
