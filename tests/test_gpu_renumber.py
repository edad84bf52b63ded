"""The breadth-first vertex order found on the GPU.

It must be the order a one-thread queue search of the undirected edges gives
(components in the order of their smallest vertex, each searched from it,
a vertex's neighbours in edge order), the same as the host search; the
solve's pairs must not depend on where the order was found."""
from collections import deque

import numpy as np
import pytest

import oracle
from common import GRAMMARS
from paper_2401_11029_gb300 import cflr, gen
from paper_2401_11029_gb300.cflr import Solver

pytestmark = pytest.mark.gpu


def queue_order(n, src, dst):
    """The order by definition: a plain queue search."""
    adj = [[] for _ in range(n)]
    for s, d in zip(src.tolist(), dst.tolist()):
        adj[s].append(d)
        adj[d].append(s)
    seen = bytearray(n)
    order = []
    for s in range(n):
        if seen[s]:
            continue
        seen[s] = 1
        q = deque([s])
        while q:
            u = q.popleft()
            order.append(u)
            for v in adj[u]:
                if not seen[v]:
                    seen[v] = 1
                    q.append(v)
    return np.asarray(order, dtype=np.uint32)


def stored_order(text, g, where):
    with Solver(text, order_on_device=where) as s:
        s.load(g)
        return cflr.cflr_get_vertex_order(s.ctx, g.n)


def check_order(text, g, reference=True):
    dev = stored_order(text, g, 1)
    host = stored_order(text, g, -1)
    assert np.array_equal(np.sort(dev), np.arange(g.n, dtype=np.uint32))
    assert np.array_equal(dev, host)
    if reference:
        assert np.array_equal(dev, queue_order(g.n, g.src, g.dst))
    return dev


def _graph(n, src, dst):
    src = np.asarray(src, np.uint32)
    return gen.Graph(n=n, labels=["a"], src=src, lab=np.zeros(src.size, np.uint32),
                     dst=np.asarray(dst, np.uint32))


@pytest.mark.parametrize("name", ["fica", "fsca2", "dyck3"])
def test_device_order_and_parity_with_oracle(name):
    text, labels = GRAMMARS[name]
    g = gen.random_graph(n=400, n_edges=1200, labels=labels, seed=41)
    check_order(text, g)
    want = oracle.solve(text, g)
    with Solver(text, form=cflr.CFLR_FORM_GRAPH, order_on_device=1) as s:
        s.load(g)
        s.solve()
        got = s.pairs_many(want.grammar.nts)
    for x in want.grammar.nts:
        assert np.array_equal(got[x], want.pairs[x]), x


def test_program_graphs_many_components():
    # thousands of components, isolated vertices, lists longer than 32
    check_order(gen.grammar_text("fica"), gen.fica_like(n=20_000, n_a=40_000, n_d=15_000,
                                                        seed=42))
    check_order(gen.grammar_text("fsca", index_hi=15),
                gen.fsca_like(n=6000, n_edges=9000, fields=16, seed=43))


def test_self_loops_repeated_edges_and_isolated_vertices():
    rng = np.random.default_rng(44)
    src = rng.integers(0, 300, 900)
    dst = rng.integers(0, 300, 900)
    loops = rng.integers(0, 300, 40)
    src = np.concatenate([src, loops, src[:100]])
    dst = np.concatenate([dst, loops, dst[:100]])        # vertices 300.. stay isolated
    check_order("S -> a | S S\n", _graph(500, src, dst))


def test_no_edges_and_one_vertex():
    check_order("S -> a\n", _graph(7, [], []))
    check_order("S -> a\n", _graph(1, [0], [0]))


def test_long_path_numbered_backwards():
    # one component of 3000 levels, searched from its smallest vertex
    n = 3000
    src = np.arange(n - 1, 0, -1)
    check_order("S -> a\n", _graph(n, src, src - 1))


def test_star_lists_sorted_in_shared_memory():
    # a hub of 5000 edge ends (its list sorted by one CTA), edges in a mixed order
    n = 6000
    leaves = np.arange(1, 5001)
    src = np.concatenate([np.zeros(5000, np.int64), leaves[:-1]])
    dst = np.concatenate([leaves, leaves[1:]])
    p = np.random.default_rng(45).permutation(src.size)
    check_order("S -> a\n", _graph(n, src[p], dst[p]))


def test_hub_beyond_the_device_list_limit_is_ordered_on_the_host():
    src = np.zeros(9000, np.int64)
    g = _graph(10_000, src, np.arange(1, 9001))
    check_order("S -> a\n", g)
    with Solver("S -> a\nT -> S S\n", order_on_device=1) as s:
        s.load(g)
        s.solve()
        assert s.count("S") == 9000 and s.count("T") == 0


def test_full_size_workloads_default_to_the_device_order():
    # 1.1 M and 4 M edges: the default (0) searches on the GPU
    g = gen.fica_like()
    auto = stored_order(gen.grammar_text("fica"), g, 0)
    assert np.array_equal(auto, stored_order(gen.grammar_text("fica"), g, -1))
    g = gen.fsjpt_like()
    text = gen.grammar_text("fsjpt")
    assert np.array_equal(stored_order(text, g, 0), stored_order(text, g, -1))


def test_vertex_order_errors_and_kept_order():
    g = _graph(5, [0, 3], [4, 1])
    with Solver("S -> a\n", keep_vertex_order=1) as s:
        s.load(g)
        assert np.array_equal(cflr.cflr_get_vertex_order(s.ctx, 5), np.arange(5))
        lib = cflr.load_library()
        buf = np.zeros(4, np.uint32)
        assert lib.cflr_get_vertex_order(s.ctx, buf.ctypes.data, 4) == cflr.CFLR_EINVAL
        assert lib.cflr_get_vertex_order(s.ctx, None, 5) == cflr.CFLR_EINVAL
    with Solver("S -> a\n") as s:
        with pytest.raises(cflr.CflrError) as e:
            cflr.cflr_get_vertex_order(s.ctx, 5)
        assert e.value.code == cflr.CFLR_ESTATE
