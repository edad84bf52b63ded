"""The seeded workload generators (CPU): shapes, determinism, and the oracle
against Algorithm 1 run as printed on small program-shaped graphs of the
field-sensitive alias and context-sensitive value-flow families."""
import numpy as np

import oracle
from paper_2401_11029_gb300 import gen
from pins import naive_alg1, read_grammar


def _triples(g):
    return set(zip(g.src.tolist(), g.lab.tolist(), g.dst.tolist()))


def test_fsca_like_shape_reverses_and_determinism():
    g = gen.fsca_like(n=2000, n_edges=3000, fields=16, seed=3)
    assert g.n_edges == 6000 and len(g.labels) == 4 + 2 * 16
    t = _triples(g)
    assert len(t) == g.n_edges                       # distinct triples
    idx = {x: i for i, x in enumerate(g.labels)}
    fwd = {"a": "a_r", "d": "d_r"}
    fwd.update({f"f_{i}": f"f_r_{i}" for i in range(16)})
    rev = dict(fwd)
    rev.update({r: f for f, r in fwd.items()})
    for s, l, d in t:                                # every edge has its reverse
        assert (d, idx[rev[g.labels[l]]], s) in t
    cnt = g.label_counts()
    assert cnt["a"] == 3000 * 45 // 100 and cnt["d"] == 3000 * 25 // 100
    assert cnt["f_0"] >= cnt["f_15"]                  # Zipf over fields
    assert g.edge_digest() == gen.fsca_like(n=2000, n_edges=3000, fields=16, seed=3).edge_digest()


def test_cscvf_like_call_structure():
    W = 64
    g = gen.cscvf_like(n=5000, n_edges=8000, calls=300, seed=4, window=W)
    assert g.n_edges == 8000 and len(g.labels) == 1 + 2 * 300
    cnt = g.label_counts()
    assert cnt["a"] == 8000 - 600
    assert all(cnt[f"call_{i}"] == 1 and cnt[f"ret_{i}"] == 1 for i in range(300))
    # a call enters a procedure at its entry vertex and the return leaves it
    # from its exit vertex: both ends of call site i lie in the same callee
    lab = {x: i for i, x in enumerate(g.labels)}
    call_dst = {int(l) - lab["call_0"]: int(d) for l, d in zip(g.lab, g.dst)
                if lab["call_0"] <= l < lab["ret_0"]}
    ret_src = {int(l) - lab["ret_0"]: int(s) for l, s in zip(g.lab, g.src) if l >= lab["ret_0"]}
    assert len(call_dst) == len(ret_src) == 300
    assert g.edge_digest() == gen.cscvf_like(n=5000, n_edges=8000, calls=300, seed=4,
                                             window=W).edge_digest()


def _check_alg1(text, g):
    res = oracle.solve(text, g)
    ref = naive_alg1(text, g)
    nts, _ = read_grammar(text)
    for x in nts:
        assert (res.dense(x, g.n) == ref[x]).all(), x


def test_oracle_equals_algorithm1_on_fsca_program_graph():
    g = gen.fsca_like(n=48, n_edges=70, fields=4, seed=8, window=16)
    _check_alg1(gen.grammar_text("fsca", index_hi=3), g)


def test_oracle_equals_algorithm1_on_cscvf_program_graph():
    g = gen.cscvf_like(n=48, n_edges=70, calls=6, seed=9, window=16)
    _check_alg1(gen.grammar_text("cscvf", index_hi=5), g)
