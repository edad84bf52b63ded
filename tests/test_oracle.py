"""Pins of the CPU oracle (no GPU needed).

Each test checks the oracle against something other than itself: Algorithm 1
run as printed, brute-force path enumeration with CYK, breadth-first search,
closed forms of Dyck languages, and the invariants and grammar equivalences
the paper's figures imply.  Inputs are tiny so the whole file runs in well
under a minute.
"""
import numpy as np
import pytest

import oracle
from oracle.grammar import GrammarError, parse
from paper_2401_11029_gb300 import gen
from pins import bfs_reach, brute_force, dyck_balanced, naive_alg1, read_grammar

from common import GRAMMARS, RANDOM_GRAMMARS  # noqa: E402


def dense_of(res, name, n):
    return res.dense(name, n)


def check_against_naive(text, g):
    res = oracle.solve(text, g)
    ref = naive_alg1(text, g)
    nts, _ = read_grammar(text)
    for x in nts:
        got = dense_of(res, x, g.n)
        assert (got == ref[x]).all(), f"{x}: oracle {got.sum()} pairs, Algorithm 1 {ref[x].sum()}"
    return res


@pytest.mark.parametrize("name", list(GRAMMARS))
@pytest.mark.parametrize("seed", [11, 12, 13])
def test_oracle_equals_algorithm1(name, seed):
    text, labels = GRAMMARS[name]
    g = gen.random_graph(n=14, n_edges=30, labels=labels, seed=seed)
    check_against_naive(text, g)


@pytest.mark.parametrize("text", RANDOM_GRAMMARS)
@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_oracle_equals_algorithm1_random_grammars(text, seed):
    g = gen.random_graph(n=10, n_edges=24, labels=["a", "b", "c"], seed=seed)
    check_against_naive(text, g)


def _tiny_dag(seed, labels, n=6, m=10):
    rng = np.random.default_rng(seed)
    src, dst, lab = [], [], []
    seen = set()
    while len(src) < m:
        u, v = sorted(rng.choice(n, size=2, replace=False).tolist())
        l = int(rng.integers(0, len(labels)))
        if (u, l, v) in seen:
            continue
        seen.add((u, l, v))
        src.append(u); dst.append(v); lab.append(l)
    return gen.Graph(n=n, labels=list(labels), src=np.array(src, np.uint32),
                     lab=np.array(lab, np.uint32), dst=np.array(dst, np.uint32))


@pytest.mark.parametrize("name", ["dyck1", "dyck3", "fica", "fica_cfg", "fsjpt2", "fsca2", "cscvf2"])
@pytest.mark.parametrize("seed", [5, 6])
def test_oracle_equals_brute_force_on_dags(name, seed):
    text, labels = GRAMMARS[name]
    g = _tiny_dag(seed, labels)
    res = oracle.solve(text, g)
    bf = brute_force(text, g, max_len=g.n)      # a DAG path has < n edges
    nts, _ = read_grammar(text)
    for x in nts:
        got = {(int(k >> 32), int(k & 0xFFFFFFFF)) for k in res.pairs[x]}
        assert got == bf.get(x, set()), x


@pytest.mark.parametrize("text", RANDOM_GRAMMARS)
def test_oracle_equals_brute_force_random_grammar_dag(text):
    g = _tiny_dag(3, ["a", "b", "c"], n=6, m=11)
    res = oracle.solve(text, g)
    bf = brute_force(text, g, max_len=g.n)
    for x in read_grammar(text)[0]:
        got = {(int(k >> 32), int(k & 0xFFFFFFFF)) for k in res.pairs[x]}
        assert got == bf.get(x, set()), x


@pytest.mark.parametrize("name", ["dyck1", "fica"])
def test_brute_force_on_cyclic_graph_is_contained_and_grows_to_oracle(name):
    text, labels = GRAMMARS[name]
    g = gen.random_graph(n=5, n_edges=9, labels=labels, seed=21)
    res = oracle.solve(text, g)
    full = {x: {(int(k >> 32), int(k & 0xFFFFFFFF)) for k in res.pairs[x]}
            for x in read_grammar(text)[0]}
    prev = 0
    for L in (2, 4, 6, 8):
        bf = brute_force(text, g, max_len=L)
        for x in full:
            assert bf.get(x, set()) <= full[x]
        tot = sum(len(v) for v in bf.values())
        assert tot >= prev
        prev = tot


def test_transitive_closure_grammar_equals_bfs():
    text = "S -> S S | a\n"
    for seed in (1, 2, 3):
        g = gen.random_graph(n=30, n_edges=45, labels=["a", "b"], seed=seed)
        res = oracle.solve(text, g)
        got = {(int(k >> 32), int(k & 0xFFFFFFFF)) for k in res.pairs["S"]}
        assert got == bfs_reach(g, "a")


def test_dyck1_on_path_graphs_matches_balanced_counter():
    rng = np.random.default_rng(7)
    text = GRAMMARS["dyck1"][0]
    for _ in range(20):
        L = int(rng.integers(1, 24))
        word = ["a" if x else "b" for x in rng.integers(0, 2, size=L)]
        g = gen.path_graph(word, labels=["a", "b"])
        res = oracle.solve(text, g)
        got = {(int(k >> 32), int(k & 0xFFFFFFFF)) for k in res.pairs["S"]}
        want = {(i, j) for i in range(L + 1) for j in range(i + 1, L + 1)
                if dyck_balanced(word[i:j], {"a": "b"})}
        assert got == want


def test_dyck3_on_path_graphs_matches_balanced_counter():
    rng = np.random.default_rng(8)
    text = GRAMMARS["dyck3"][0]
    labels = GRAMMARS["dyck3"][1]
    for _ in range(20):
        L = int(rng.integers(1, 20))
        word = [labels[int(x)] for x in rng.integers(0, 6, size=L)]
        g = gen.path_graph(word, labels=labels)
        res = oracle.solve(text, g)
        got = {(int(k >> 32), int(k & 0xFFFFFFFF)) for k in res.pairs["S"]}
        want = {(i, j) for i in range(L + 1) for j in range(i + 1, L + 1)
                if dyck_balanced(word[i:j], {"a_1": "b_1", "a_2": "b_2", "a_3": "b_3"})}
        assert got == want


def test_dyck_pairs_join_equal_heights_on_layered_graph():
    g = gen.layered_graph(n=60, n_edges=150, seed=4,
                          pairs=(("a_1", "b_1"), ("a_2", "b_2"), ("a_3", "b_3")))
    res = oracle.solve(GRAMMARS["dyck3"][0], g)
    h = g.meta["height"]
    k = res.pairs["S"]
    assert k.size > 0
    assert (h[(k >> np.uint64(32)).astype(np.int64)] ==
            h[(k & np.uint64(0xFFFFFFFF)).astype(np.int64)]).all()


def _with_reverse(g, pairs):
    src, dst, lab = [g.src], [g.dst], [g.lab]
    labels = list(g.labels)
    for f, r in pairs.items():
        sel = g.lab == labels.index(f)
        src.append(g.dst[sel]); dst.append(g.src[sel])
        lab.append(np.full(int(sel.sum()), labels.index(r), np.uint32))
    return gen.Graph(n=g.n, labels=labels, src=np.concatenate(src),
                     dst=np.concatenate(dst), lab=np.concatenate(lab))


def test_fica_alias_relation_is_symmetric():
    # closed under reversal + the grammar maps to itself under reverse-and-bar
    for seed in (1, 2):
        base = gen.random_graph(n=40, n_edges=70, labels=["a", "d", "a_r", "d_r"], seed=seed)
        keep = (base.lab == 0) | (base.lab == 1)
        fwd = gen.Graph(n=base.n, labels=base.labels, src=base.src[keep], lab=base.lab[keep],
                        dst=base.dst[keep])
        g = _with_reverse(fwd, {"a": "a_r", "d": "d_r"})
        m = oracle.solve(GRAMMARS["fica"][0], g).dense("M", g.n)
        assert m.sum() > 0
        assert (m == m.T).all()


def test_fsjpt_flows_to_is_points_to_transposed():
    text, labels = GRAMMARS["fsjpt2"]
    fwd_labels = ["alloc", "assign", "load_0", "load_1", "store_0", "store_1"]
    for seed in (3, 4):
        base = gen.random_graph(n=40, n_edges=90, labels=fwd_labels, seed=seed)
        pairs = {x: (x.replace("_", "_r_") if x[-1].isdigit() else x + "_r") for x in fwd_labels}
        g = _with_reverse(gen.Graph(n=base.n, labels=fwd_labels + list(pairs.values()),
                                    src=base.src, lab=base.lab, dst=base.dst), pairs)
        res = oracle.solve(text, g)
        pt, ft = res.dense("PT", g.n), res.dense("FT", g.n)
        assert pt.sum() > 0
        assert (ft == pt.T).all()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_optimisation5_fica_grammars_agree(seed):
    g = gen.random_graph(n=30, n_edges=60, labels=["a", "d", "a_r", "d_r"], seed=seed)
    m1 = oracle.solve(GRAMMARS["fica"][0], g).dense("M", g.n)
    m2 = oracle.solve(GRAMMARS["fica_cfg"][0], g).dense("M", g.n)
    assert m1.sum() > 0
    assert (m1 == m2).all()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_optimisation5_fsjpt_grammars_agree(seed):
    text, labels = GRAMMARS["fsjpt2"]
    g = gen.random_graph(n=30, n_edges=110, labels=labels, seed=seed)
    r1 = oracle.solve(text, g)
    r2 = oracle.solve(GRAMMARS["fsjpt2_cfg"][0], g)
    for x in ("PT", "FT"):
        assert (r1.dense(x, g.n) == r2.dense(x, g.n)).all()
    assert r1.dense("PT", g.n).sum() > 0


def test_fixpoint_is_closed_and_idempotent_on_workload_sample():
    """One more full (non-delta) application of every production adds nothing."""
    import scipy.sparse as sp
    g = gen.fica_like(n=3000, n_a=6000, n_d=2250, seed=9)
    res = oracle.solve(GRAMMARS["fica"][0], g)
    pg = res.grammar
    n = g.n

    def mat(X):
        k = res.pairs[pg.nts[X]]
        r = (k >> np.uint64(32)).astype(np.int64)
        c = (k & np.uint64(0xFFFFFFFF)).astype(np.int64)
        return sp.csr_matrix((np.ones(k.size, np.int64), (r, c)), shape=(n, n))
    for c, a, b in pg.binary:
        prod = (mat(a) @ mat(b)).tocoo()
        have = set((res.pairs[pg.nts[c]]).tolist())
        keys = (prod.row.astype(np.uint64) << np.uint64(32)) | prod.col.astype(np.uint64)
        assert set(keys.tolist()) <= have
    # monotone: the terminal initialisation is contained in the result
    init = oracle.terminal_init(pg, g).astype(np.uint64)
    for A in np.unique(init[:, 1]).tolist():
        sel = init[:, 1] == A
        keys = (init[sel, 0] << np.uint64(32)) | init[sel, 2]
        assert np.isin(keys, res.pairs[pg.nts[A]]).all()


def test_oracle_grammar_reader_counts():
    g = parse(gen.grammar_text("fsjpt"))
    F = 64
    assert g.n_user == 2 + 6 * F            # PT, FT, LPFS_i, LP_i, FS_i, SPFL_i, SP_i, FL_i
    assert len(g.binary) == 2 + 8 * F        # the binary productions of Fig. wcnf:fsjpt
    assert len(g.nts) - g.n_user == 2 + 4 * F  # wrapped terminals of binary productions
    assert len(g.term) == 4 + 4 * F          # terminal labels
    f = parse(gen.grammar_text("fica"))
    assert f.nts[:f.n_user] == ["M", "N1", "N2", "N3", "AM"]
    names = f.nts
    got = sorted((names[c], names[a], names[b]) for c, a, b in f.binary)
    assert got == sorted([("M", "N1", "N3"), ("M", "N2", "N3"), ("N1", "N1", "<a_r>"),
                          ("N1", "N2", "<a_r>"), ("N2", "N1", "M"), ("N3", "<a>", "N3"),
                          ("N3", "AM", "N3"), ("AM", "<a>", "M")])
    assert sorted((k, [names[x] for x in v]) for k, v in f.term.items()) == sorted(
        [("d_r", ["N1"]), ("d", ["N3"]), ("a_r", ["<a_r>"]), ("a", ["<a>"])])


@pytest.mark.parametrize("bad", ["S -> a b c\n", "S a b\n", "%index i 3 1\nS -> a_{i}\n",
                                 "S -> a_{j}\n", "S -> A eps\n"])
def test_oracle_grammar_reader_rejects(bad):
    with pytest.raises(GrammarError):
        parse(bad)


def test_epsilon_gives_identity_and_unit_copies():
    text = "A -> eps | a\nB -> A\n"
    g = gen.random_graph(n=5, n_edges=4, labels=["a"], seed=1)
    res = oracle.solve(text, g)
    a = res.dense("A", g.n)
    assert a.diagonal().all()
    assert (res.dense("B", g.n) == a).all()
