"""Parity of the CUDA path with the CPU oracle (bit-exact pair sets).

All calls go through the C ABI (the ctypes binding).  Sizes are chosen so the
oracle finishes in seconds while the GPU work still spans many work-list
groups, every shared-memory bin and ragged tails; the full-size workloads are
compared through fingerprints the oracle wrote (tests/golden).
"""
import json
import os

import numpy as np
import pytest

import oracle
from common import GRAMMARS, RANDOM_GRAMMARS, fingerprint, keys_of
from paper_2401_11029_gb300 import cflr, gen
from paper_2401_11029_gb300.cflr import CflrError, Solver

pytestmark = pytest.mark.gpu


def gpu_pairs(text, g, names=None, **cfg):
    with Solver(text, **cfg) as s:
        s.load(g)
        st = s.solve()
        if names is None:
            names = oracle.parse(text).nts
        return {x: s.pairs(x) for x in names}, st


def assert_parity(text, g, include_wrappers=True, **cfg):
    want = oracle.solve(text, g)
    pg = want.grammar
    names = pg.nts if include_wrappers else pg.nts[:pg.n_user]
    got, st = gpu_pairs(text, g, names, **cfg)
    for x in names:
        a, b = got[x], want.pairs[x]
        if not np.array_equal(a, b):
            extra = np.setdiff1d(a, b)[:5]
            missing = np.setdiff1d(b, a)[:5]
            raise AssertionError(f"{x}: gpu {a.size} vs oracle {b.size} pairs; "
                                 f"extra {[(int(k >> 32), int(k & 0xFFFFFFFF)) for k in extra]} "
                                 f"missing {[(int(k >> 32), int(k & 0xFFFFFFFF)) for k in missing]}")
    assert st["total_pairs"] == want.total()
    return st, want


@pytest.mark.parametrize("name", list(GRAMMARS))
@pytest.mark.parametrize("seed", [1, 2])
@pytest.mark.parametrize("n,m", [(30, 70), (300, 900)])
def test_paper_grammars_random_graphs(name, seed, n, m):
    text, labels = GRAMMARS[name]
    assert_parity(text, gen.random_graph(n=n, n_edges=m, labels=labels, seed=seed))


@pytest.mark.parametrize("text", RANDOM_GRAMMARS)
@pytest.mark.parametrize("seed", [3, 4])
def test_epsilon_unit_and_terminal_operands(text, seed):
    assert_parity(text, gen.random_graph(n=60, n_edges=150, labels=["a", "b", "c"], seed=seed))


def test_dyck1_erdos_renyi_full_size():
    """Dyck-1 on the 1000-vertex Erdos-Renyi graph (dense closure, bitmap bin)."""
    st, want = assert_parity(gen.grammar_text("dyck1"), gen.dyck1_er())
    assert want.pairs["S"].size > 100_000


def test_fica_program_graph():
    g = gen.fica_like(n=20_000, n_a=40_000, n_d=15_000, seed=2)
    st, want = assert_parity(gen.grammar_text("fica"), g)
    assert st["iterations"] > 3


def test_fsjpt_program_graph_64_fields():
    g = gen.fsjpt_like(n=12_000, n_edges=48_000, fields=64, seed=3)
    st, want = assert_parity(gen.grammar_text("fsjpt"), g, include_wrappers=False)
    assert want.pairs["PT"].size > 0


def test_growth_paths_give_identical_pairs():
    """Tiny first buffers force every re-run-after-growth path."""
    g = gen.fica_like(n=5000, n_a=10_000, n_d=3750, seed=11)
    st, _ = assert_parity(gen.grammar_text("fica"), g, initial_capacity=64)
    assert st["regrows"] > 0
    assert st["regrow_buffers"] + st["regrow_sets"] + st["regrow_pools"] == st["regrows"]


def test_batch_equals_alone_and_oracle():
    text = gen.grammar_text("dyck3")
    graphs = gen.dyck3_batch(count=12, seed0=4000, n_lo=500, n_hi=5000)
    solvers = [Solver(text) for _ in graphs]
    try:
        for s, g in zip(solvers, graphs):
            s.load(g)
        cflr.cflr_solve_batch([s.ctx for s in solvers])
        for s, g in zip(solvers, graphs):
            want = oracle.solve(text, g)
            for x in want.grammar.nts:
                assert np.array_equal(s.pairs(x), want.pairs[x]), x
    finally:
        for s in solvers:
            s.close()


# ---------------------------------------------------------------------------
# edge cases and error handling
# ---------------------------------------------------------------------------

def test_empty_graph_and_isolated_vertices():
    text = gen.grammar_text("fica")
    g = gen.Graph(n=10, labels=["a"], src=np.zeros(0, np.uint32), lab=np.zeros(0, np.uint32),
                  dst=np.zeros(0, np.uint32))
    got, st = gpu_pairs(text, g, ["M", "N1"])
    assert got["M"].size == 0 and st["total_pairs"] == 0


def test_single_vertex_self_loops():
    assert_parity("S -> S S | a\n", gen.Graph(n=1, labels=["a"], src=np.zeros(1, np.uint32),
                                               lab=np.zeros(1, np.uint32),
                                               dst=np.zeros(1, np.uint32)))


def test_duplicate_edges_and_unknown_labels():
    text, labels = GRAMMARS["dyck1"]
    g = gen.random_graph(n=50, n_edges=120, labels=labels + ["zzz"], seed=5)
    dup = gen.Graph(n=g.n, labels=g.labels, src=np.concatenate([g.src, g.src]),
                    lab=np.concatenate([g.lab, g.lab]), dst=np.concatenate([g.dst, g.dst]))
    want = oracle.solve(text, g)
    got, st = gpu_pairs(text, dup, ["S", "S1"])
    for x in ("S", "S1"):
        assert np.array_equal(got[x], want.pairs[x])
    assert st["ignored_edges"] == 2 * int((g.lab == 2).sum())


def test_epsilon_identity_on_every_vertex():
    got, _ = gpu_pairs("A -> eps\n", gen.Graph(n=1000, labels=["a"], src=np.zeros(0, np.uint32),
                                               lab=np.zeros(0, np.uint32),
                                               dst=np.zeros(0, np.uint32)), ["A"])
    assert np.array_equal(got["A"], keys_of(np.arange(1000), np.arange(1000)))


def test_call_order_and_argument_errors():
    ctx = cflr.cflr_create()
    try:
        with pytest.raises(CflrError) as e:
            cflr.cflr_load_graph(ctx, 3, [0], [0], [1])
        assert e.value.code == cflr.CFLR_ESTATE
        with pytest.raises(CflrError) as e:
            cflr.cflr_load_grammar(ctx, "S -> a b c\n")
        assert e.value.code == cflr.CFLR_EGRAMMAR
        cflr.cflr_load_grammar(ctx, "S -> S S | a\n")
        with pytest.raises(CflrError) as e:
            cflr.cflr_solve(ctx)
        assert e.value.code == cflr.CFLR_ESTATE
        with pytest.raises(CflrError) as e:
            cflr.cflr_load_graph(ctx, 3, [0], [0], [3])
        assert e.value.code == cflr.CFLR_EGRAPH
        cflr.cflr_load_graph(ctx, 3, [0, 1], [0, 0], [1, 2])
        cflr.cflr_solve(ctx)
        s, d = cflr.cflr_get_pairs(ctx, 0)
        assert list(zip(s.tolist(), d.tolist())) == [(0, 1), (0, 2), (1, 2)]
        with pytest.raises(CflrError) as e:
            cflr.cflr_get_pairs(ctx, 7)
        assert e.value.code == cflr.CFLR_EINVAL
    finally:
        cflr.cflr_destroy(ctx)


def test_iteration_limit_then_resume_reaches_same_fixpoint():
    text = gen.grammar_text("fica")
    g = gen.fica_like(n=4000, n_a=8000, n_d=3000, seed=12)
    want = oracle.solve(text, g)
    with Solver(text, max_iterations=2) as s:
        s.load(g)
        with pytest.raises(CflrError) as e:
            s.solve()
        assert e.value.code == cflr.CFLR_ELIMIT
        partial = s.count("M")
        assert partial <= want.pairs["M"].size
        for _ in range(1000):
            try:
                s.solve()
                break
            except CflrError as err:
                assert err.code == cflr.CFLR_ELIMIT
        assert np.array_equal(s.pairs("M"), want.pairs["M"])


def test_memory_budget_is_enforced_and_context_survives():
    text = gen.grammar_text("fica")
    g = gen.fica_like(n=20_000, n_a=40_000, n_d=15_000, seed=2)
    with Solver(text, mem_budget_bytes=48 << 20) as s:    # the 20k graph needs ~450 MB
        with pytest.raises(CflrError) as e:
            s.load(g)
            s.solve()
        assert e.value.code == cflr.CFLR_ENOMEM
        small = gen.random_graph(n=20, n_edges=30, labels=["a", "d", "a_r", "d_r"], seed=1)
        s.load(small)
        s.solve()
        want = oracle.solve(text, small)
        assert np.array_equal(s.pairs("M"), want.pairs["M"])


# ---------------------------------------------------------------------------
# full-size workloads against the oracle's stored fingerprints
# ---------------------------------------------------------------------------

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden(name):
    path = os.path.join(GOLDEN, name + ".json")
    if not os.path.exists(path):
        pytest.skip(f"no stored oracle fingerprints for {name}")
    with open(path) as f:
        return json.load(f)


def _check_full(name, grammar, g, **cfg):
    gold = _golden(name)
    if g.edge_digest() != gold["edge_digest"]:
        pytest.skip("the generator made a different graph on this machine")
    with Solver(gen.grammar_text(grammar), **cfg) as s:
        s.load(g)
        st = s.solve()
        for x, fp in gold["pairs"].items():
            assert fingerprint(s.pairs(x)) == fp, x
    assert st["total_pairs"] == gold["total_pairs"]
    return st


def test_full_size_dyck1_er():
    _check_full("dyck1_er_1000", "dyck1", gen.dyck1_er())


def test_full_size_fica_200k():
    _check_full("fica_like_200k", "fica", gen.fica_like())


def _check_timed_configuration(kind, n_vertices):
    """The exact launch configuration bench.py times (graph form, the cached
    tuned schedule through cflr_autotune, reset + solve + extraction to
    device buffers, twice on the same context) against the oracle's stored
    fingerprints of every named non-terminal."""
    import torch
    import bench
    g = bench.workload_graph(bench.WORKLOAD["seed"] if kind == "fica" else bench.FSJPT["seed"],
                             n_vertices, kind)
    gold = _golden(bench.golden_name(kind, g.n))
    if g.edge_digest() != gold["edge_digest"]:
        pytest.skip("the generator made a different graph on this machine")
    stream = torch.cuda.current_stream()
    ctx, tuning = bench.timed_context(g, bench.grammar_of(kind), 0, stream.cuda_stream)
    try:
        # the schedule is the cached one the bench line reports
        assert open(bench.TUNING_CACHE).read().count(f"_{g.n}_{g.n_edges} ") >= 1
        n_nt, n_named, _ = cflr.cflr_grammar_sizes(ctx)
        cap = gold["total_pairs"]
        out = (torch.empty(cap, dtype=torch.int32, device="cuda"),
               torch.empty(cap, dtype=torch.int32, device="cuda"))
        for _ in range(2):                       # second pass runs on reused buffers
            total = bench.device_step(ctx, n_named, out)
            assert total == gold["total_pairs"]
            fps = bench.device_fingerprints(ctx, list(gold["pairs"]), out)
            for x, fp in gold["pairs"].items():
                assert fps[x] == fp, x
    finally:
        cflr.cflr_destroy(ctx)
    return tuning


def test_full_size_fica_200k_launch_config_of_bench():
    t = _check_timed_configuration("fica", 200_000)
    assert t["bin_limit"][2] == t["bin_limit"][1] + 1      # bin 2 routed to the bitmap bin


def test_full_size_fsjpt_500k_launch_config_of_bench():
    _check_timed_configuration("fsjpt", 500_000)


def test_full_size_dyck3_batch_256_graph_form():
    """The 256 Dyck-3 instances as bench.py times them: graph-form contexts
    solved together by cflr_solve_batch after cflr_reset, twice."""
    gold = _golden("dyck3_batch_256")
    text = gen.grammar_text("dyck3")
    graphs = gen.dyck3_batch(count=256, seed0=4000)
    solvers = [Solver(text, form=cflr.CFLR_FORM_GRAPH) for _ in graphs]
    try:
        for s, g, gi in zip(solvers, graphs, gold["instances"]):
            assert g.edge_digest() == gi["edge_digest"]
            s.load(g)
        for _ in range(2):
            for s in solvers:
                cflr.cflr_reset(s.ctx)
            cflr.cflr_solve_batch([s.ctx for s in solvers])
            for s, gi in zip(solvers, gold["instances"]):
                for x, fp in gi["pairs"].items():
                    assert fingerprint(s.pairs(x)) == fp, (gi["seed"], x)
    finally:
        for s in solvers:
            s.close()


def test_full_size_fsjpt_500k():
    _check_full("fsjpt_like_500k", "fsjpt", gen.fsjpt_like())


def test_full_size_dyck3_batch_256():
    gold = _golden("dyck3_batch_256")
    text = gen.grammar_text("dyck3")
    graphs = gen.dyck3_batch(count=256, seed0=4000)
    solvers = [Solver(text) for _ in graphs]
    try:
        for s, g, gi in zip(solvers, graphs, gold["instances"]):
            assert g.edge_digest() == gi["edge_digest"]
            s.load(g)
        cflr.cflr_solve_batch([s.ctx for s in solvers])
        for s, gi in zip(solvers, gold["instances"]):
            for x, fp in gi["pairs"].items():
                assert fingerprint(s.pairs(x)) == fp, (gi["seed"], x)
    finally:
        for s in solvers:
            s.close()


@pytest.mark.parametrize("form", [cflr.CFLR_FORM_PLAIN, cflr.CFLR_FORM_BATCHED,
                                  cflr.CFLR_FORM_GRAPH])
def test_execution_forms_agree(form):
    text = gen.grammar_text("fica")
    g = gen.fica_like(n=8000, n_a=16_000, n_d=6000, seed=21)
    st, want = assert_parity(text, g, form=form)
    # one more solve of a finished context is a no-op with the same pairs
    with Solver(text, form=form) as s:
        s.load(g)
        first = s.solve()
        again = s.solve()
        assert again["total_pairs"] == first["total_pairs"] == want.total()
        assert first["iterations"] == st["iterations"]


def test_graph_form_growth_and_limit_paths():
    """The device-driven loop stops for every growth and for the iteration
    limit, and the host finishes the iteration."""
    text = gen.grammar_text("fica")
    g = gen.fica_like(n=5000, n_a=10_000, n_d=3750, seed=11)
    st, _ = assert_parity(text, g, form=cflr.CFLR_FORM_GRAPH, initial_capacity=64)
    assert st["regrows"] > 0
    want = oracle.solve(text, g)
    with Solver(text, form=cflr.CFLR_FORM_GRAPH, max_iterations=3) as s:
        s.load(g)
        for _ in range(1000):
            try:
                s.solve()
                break
            except CflrError as err:
                assert err.code == cflr.CFLR_ELIMIT
        assert np.array_equal(s.pairs("M"), want.pairs["M"])


def test_graph_form_batch_of_instances():
    text = gen.grammar_text("dyck3")
    graphs = gen.dyck3_batch(count=8, seed0=4100, n_lo=500, n_hi=4000)
    solvers = [Solver(text, form=cflr.CFLR_FORM_GRAPH) for _ in graphs]
    try:
        for s, g in zip(solvers, graphs):
            s.load(g)
        stats = cflr.cflr_solve_batch([s.ctx for s in solvers])
        for s, g, st in zip(solvers, graphs, stats):
            want = oracle.solve(text, g)
            for x in want.grammar.nts:
                assert np.array_equal(s.pairs(x), want.pairs[x]), x
            alone = Solver(text)
            alone.load(g)
            assert alone.solve()["iterations"] == st["iterations"]
            alone.close()
    finally:
        for s in solvers:
            s.close()


# ---------------------------------------------------------------------------
# product-kernel schedules
# ---------------------------------------------------------------------------

def test_tuning_roundtrip_and_validation():
    with Solver("S -> S S | a\n") as s:
        t = cflr.cflr_get_tuning(s.ctx)
        assert t["bin_limit"] == [128, 1024, 4096]
        cflr.cflr_set_tuning(s.ctx, 2, [64, 512, 2048], [4, 2, 2, 4])
        assert cflr.cflr_get_tuning(s.ctx) == {"probe_ratio": 2, "bin_limit": [64, 512, 2048],
                                               "ctas_per_sm": [4, 2, 2, 4]}
        for bad in ((0, [64, 512, 2048], [4, 2, 2, 4]), (2, [256, 512, 2048], [4, 2, 2, 4]),
                    (2, [64, 32, 2048], [4, 2, 2, 4]), (2, [64, 512, 2048], [0, 2, 2, 4])):
            with pytest.raises(CflrError) as e:
                cflr.cflr_set_tuning(s.ctx, *bad)
            assert e.value.code == cflr.CFLR_EINVAL


@pytest.mark.parametrize("tuning", [(1, [16, 64, 256], [1, 1, 1, 1]),
                                    (1000, [128, 1024, 4096], [32, 8, 8, 8]),
                                    (1, [128, 129, 130], [8, 3, 3, 2])])
def test_extreme_schedules_give_identical_pairs(tuning):
    """Groups pushed into other bins and accumulator modes still give the
    oracle's pairs."""
    text = gen.grammar_text("fica")
    g = gen.fica_like(n=6000, n_a=12_000, n_d=4500, seed=31)
    want = oracle.solve(text, g)
    with Solver(text, form=cflr.CFLR_FORM_GRAPH) as s:
        cflr.cflr_set_tuning(s.ctx, *tuning)
        s.load(g)
        s.solve()
        for x in want.grammar.nts:
            assert np.array_equal(s.pairs(x), want.pairs[x]), x


def test_autotune_measures_caches_and_stays_exact(tmp_path):
    text = gen.grammar_text("fica")
    g = gen.fica_like(n=20_000, n_a=40_000, n_d=15_000, seed=2)
    want = oracle.solve(text, g)
    cache = str(tmp_path / "tuning.txt")
    with Solver(text, autotune_cache=cache.encode()) as s:
        s.load(g)
        best = cflr.cflr_autotune(s.ctx, 10)
        s.solve()
        for x in want.grammar.nts[:want.grammar.n_user]:
            assert np.array_equal(s.pairs(x), want.pairs[x]), x
    assert open(cache).read().count("\n") == 1
    with Solver(text, autotune_cache=cache.encode()) as s2:
        s2.load(g)
        assert cflr.cflr_autotune(s2.ctx, 10) == best      # read from the cache
        s2.solve()
        assert np.array_equal(s2.pairs("M"), want.pairs["M"])
    assert open(cache).read().count("\n") == 1


def test_size_hint_presizes_and_stays_exact():
    text = gen.grammar_text("fica")
    g = gen.fica_like(n=8000, n_a=16_000, n_d=6000, seed=41)
    st_hint, _ = assert_parity(text, g, size_hint=100)
    st_none, _ = assert_parity(text, g)
    assert st_hint["regrows"] <= st_none["regrows"]


@pytest.mark.parametrize("keep", [0, 1])
@pytest.mark.parametrize("name", ["dyck1", "fica", "fsca2"])
def test_vertex_order_kept_or_renumbered(keep, name):
    """The internal breadth-first renumbering is invisible in the results."""
    text, labels = GRAMMARS[name]
    for seed, (n, m) in enumerate([(1, 1), (7, 12), (500, 1400)]):
        g = gen.random_graph(n=n, n_edges=m, labels=labels, seed=50 + seed)
        assert_parity(text, g, keep_vertex_order=keep)
    g = gen.fica_like(n=6000, n_a=12_000, n_d=4500, seed=43)
    assert_parity(gen.grammar_text("fica"), g, keep_vertex_order=keep)


@pytest.mark.parametrize("keep", [0, 1])
def test_rows_beyond_the_shared_memory_bitmap(keep):
    """Over 1.6M vertices the row bitmaps (product bin 3, folding of large
    rows) no longer fit shared memory and take their global-memory forms."""
    n = 1_700_000
    rng = np.random.default_rng(71)
    ids = rng.choice(n, size=700, replace=False).astype(np.uint32)
    # a path of 600 'a' edges over scattered ids (closure rows up to 600 long)
    # and 100 'a' edges into the path (more rows that grow every iteration)
    src = np.concatenate([ids[:600], ids[600:700]])
    dst = np.concatenate([ids[1:601], ids[rng.integers(0, 600, size=100)]])
    g = gen.Graph(n=n, labels=["a"], src=src, lab=np.zeros(src.size, np.uint32), dst=dst)
    st, want = assert_parity("S -> a | S S\n", g, keep_vertex_order=keep)
    assert want.pairs["S"].size > 150_000


@pytest.mark.parametrize("keep", [0, 1])
def test_extraction_across_row_lengths(keep):
    """Rows of every length class of the extraction: up to 32 entries (sorted
    in registers), up to 1024 (sorted in shared memory, around each power of
    two) and longer (the per-row bitmap), each ending sorted in caller ids."""
    n = 9000
    rng = np.random.default_rng(73)
    lengths = [1, 2, 31, 32, 33, 63, 64, 65, 127, 128, 129, 255, 256, 257, 511, 512, 513,
               1000, 1023, 1024, 1025, 1500, 4000]
    srcs, dsts = [], []
    for r, L in enumerate(lengths):     # sources 0..22 point into 100..n-1 only
        srcs.append(np.full(L, r, np.uint32))
        dsts.append((100 + rng.choice(n - 100, size=L, replace=False)).astype(np.uint32))
    # links among the targets scramble the breadth-first renumbering
    extra = rng.integers(100, n, size=(3000, 2)).astype(np.uint32)
    src = np.concatenate(srcs + [extra[:, 0]])
    dst = np.concatenate(dsts + [extra[:, 1]])
    g = gen.Graph(n=n, labels=["a", "b"], src=src,
                  lab=np.concatenate([np.zeros(src.size - 3000, np.uint32),
                                      np.ones(3000, np.uint32)]), dst=dst)
    st, want = assert_parity("S -> a | S S\nT -> b\n", g, keep_vertex_order=keep)
    rows = np.bincount((want.pairs["S"] >> 32).astype(np.int64), minlength=len(lengths))
    assert list(rows[:len(lengths)]) == lengths


@pytest.mark.parametrize("form", [cflr.CFLR_FORM_PLAIN, cflr.CFLR_FORM_BATCHED,
                                  cflr.CFLR_FORM_GRAPH])
@pytest.mark.parametrize("tuning", [None, (1, [16, 64, 256], [1, 1, 1, 1])])
def test_indexed_families_as_block_products(form, tuning):
    """Optimisation 4: the 64-field points-to grammar runs its families as one
    block product each (batched and graph forms; the plain form keeps one
    product per member).  Small bin limits force the large families apart
    into per-member groups."""
    text = gen.grammar_text("fsjpt")
    g = gen.fsjpt_like(n=6_000, n_edges=24_000, fields=64, seed=13)
    want = oracle.solve(text, g)
    with Solver(text, form=form) as s:
        if tuning:
            cflr.cflr_set_tuning(s.ctx, *tuning)
        s.load(g)
        st = s.solve()
        assert st["total_pairs"] == want.total()
        for x in want.grammar.nts[:want.grammar.n_user]:
            assert np.array_equal(s.pairs(x), want.pairs[x]), x


def test_autotune_cache_path_is_copied_at_create(tmp_path):
    """The context keeps its own copy of cfg.autotune_cache: the caller's
    buffer may be reused right after cflr_create."""
    import ctypes
    text = gen.grammar_text("fica")
    g = gen.fica_like(n=5000, n_a=10_000, n_d=3750, seed=7)
    cache = str(tmp_path / "t.txt")
    buf = ctypes.create_string_buffer(cache.encode(), 4096)
    cfg = cflr.cflr_default_config()
    cfg.autotune_cache = ctypes.cast(buf, ctypes.c_char_p)
    s = Solver.__new__(Solver)
    s.ctx = cflr.cflr_create(cfg)
    try:
        cflr.cflr_load_grammar(s.ctx, text)
        ctypes.memset(buf, ord("x"), 4095)          # the caller's buffer changes
        s.load(g)
        cflr.cflr_autotune(s.ctx, 3)
    finally:
        cflr.cflr_destroy(s.ctx)
    assert open(cache).read().count("\n") == 1


@pytest.mark.parametrize("name", ["dyck1", "fica", "fsca2", "cscvf2", "fsjpt2"])
def test_witness_steps_rebuild_valid_paths(name):
    """Single-path semantics (cfg.witness): the pair sets are unchanged, every
    recorded step of a sampled pair is a production whose operand pairs the
    oracle holds (or an edge of the graph), and the path those steps rebuild
    joins the pair over the graph's edges; short paths' label words are
    checked with CYK too."""
    from pins import CYK
    text, labels = GRAMMARS[name]
    g = gen.random_graph(n=50, n_edges=140, labels=labels, seed=61)
    want = oracle.solve(text, g)
    pg = want.grammar
    binary = set(pg.binary)
    unit = set(pg.unit)
    eps = set(pg.eps)
    term = {(A, x) for x, As in pg.term.items() for A in As}
    edges = {(int(a), g.labels[l], int(b)) for a, l, b in zip(g.src, g.lab, g.dst)}
    pairs = {pg.nt_id(x): set(map(int, want.pairs[x])) for x in pg.nts}
    cyk = CYK(text)
    rng = np.random.default_rng(5)
    with Solver(text, witness=1) as s:
        s.load(g)
        s.solve()
        lib_of = {s.nt_id(x): pg.nt_id(x) for x in pg.nts}     # library id -> oracle id
        ids = s.label_ids(g.labels)
        label_name = {int(i): lab for i, lab in zip(ids, g.labels) if i != 0xFFFFFFFF}
        for x in pg.nts[:pg.n_user]:
            keys = want.pairs[x]
            assert np.array_equal(s.pairs(x), keys), x
            if keys.size == 0:
                continue
            for key in rng.choice(keys, size=min(12, keys.size), replace=False):
                u, v = int(key >> 32), int(key & 0xFFFFFFFF)
                # every step of the derivation, checked against the oracle
                stack = [(s.nt_id(x), u, v)]
                while stack:
                    X, a, b = stack.pop()
                    kind, i1, i2, m = cflr.cflr_get_witness(s.ctx, X, a, b)
                    ox = lib_of[X]
                    if kind == cflr.CFLR_WIT_EDGE:
                        assert (ox, label_name[i1]) in term and (a, label_name[i1], b) in edges
                    elif kind == cflr.CFLR_WIT_EPS:
                        assert a == b and ox in eps
                    elif kind == cflr.CFLR_WIT_UNIT:
                        assert (ox, lib_of[i1]) in unit
                        assert (a << 32) | b in pairs[lib_of[i1]]
                        stack.append((i1, a, b))
                    else:
                        assert (ox, lib_of[i1], lib_of[i2]) in binary
                        assert (a << 32) | m in pairs[lib_of[i1]]
                        assert (m << 32) | b in pairs[lib_of[i2]]
                        stack.append((i2, m, b))
                        stack.append((i1, a, m))
                path = s.path(x, u, v, label_name)
                cur = u
                for a, lab, b in path:
                    assert a == cur and (a, lab, b) in edges
                    cur = b
                assert cur == v
                if len(path) <= 12:
                    assert x in cyk.derives(tuple(lab for _, lab, _ in path))


def test_full_pair_set_stops_the_solve_and_context_stays_usable():
    """Every hash probe is capped at one pass over its table.  With the pair
    sets kept at their first size (a test-only setting) a set fills up: the
    capped probes report it, the solve returns CFLR_ECUDA instead of spinning,
    and the same context then solves a new graph correctly."""
    text = gen.grammar_text("fica")
    big = gen.fica_like(n=5000, n_a=10_000, n_d=3750, seed=11)
    small = gen.random_graph(n=20, n_edges=30, labels=["a", "d", "a_r", "d_r"], seed=1)
    for form in (cflr.CFLR_FORM_BATCHED, cflr.CFLR_FORM_GRAPH):
        with Solver(text, form=form, test_fixed_pair_sets=1) as s:
            s.load(big)
            with pytest.raises(CflrError) as e:
                s.solve()
            assert e.value.code == cflr.CFLR_ECUDA
            assert "filled up" in e.value.message
            with pytest.raises(CflrError) as e:      # the matrices were dropped
                s.solve()
            assert e.value.code == cflr.CFLR_ESTATE
            s.load(small)
            s.solve()
            want = oracle.solve(text, small)
            for x in want.grammar.nts:
                assert np.array_equal(s.pairs(x), want.pairs[x]), x


# ---------------------------------------------------------------------------
# the field-sensitive alias and context-sensitive value-flow workloads
# (Figs. wcnf:fsca and wcnf:cscvf: epsilon, unit productions, indexed
# families over the full index range of the graph)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("form", [cflr.CFLR_FORM_PLAIN, cflr.CFLR_FORM_BATCHED,
                                  cflr.CFLR_FORM_GRAPH])
def test_fsca_program_graph_64_fields(form):
    g = gen.fsca_like(n=3000, n_edges=4000, fields=64, seed=21)
    st, want = assert_parity(gen.grammar_text("fsca", index_hi=63), g, form=form)
    assert want.pairs["M"].size > 1000 and want.pairs["FV_63"].size > 0


@pytest.mark.parametrize("form", [cflr.CFLR_FORM_PLAIN, cflr.CFLR_FORM_BATCHED,
                                  cflr.CFLR_FORM_GRAPH])
def test_cscvf_program_graph_256_call_sites(form):
    g = gen.cscvf_like(n=4000, n_edges=6700, calls=256, seed=22)
    st, want = assert_parity(gen.grammar_text("cscvf", index_hi=255), g, form=form)
    assert want.pairs["AH"].size > 0


def test_fsca_paper_shaped_142_fields():
    """The imagick-shaped field-sensitive alias graph (41,652 vertices, 111,550
    edges, 142 fields) in the timed launch configuration (graph form)."""
    g = gen.fsca_like()
    assert len(g.labels) == 288
    assert_parity(gen.grammar_text("fsca", index_hi=141), g, include_wrappers=False,
                  form=cflr.CFLR_FORM_GRAPH)
