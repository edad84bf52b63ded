"""The allocation-free extraction entry point (cflr_get_pairs_device_noalloc).

It exists for callers that may not allocate device memory when they read
results (a fixed device-memory plan, an embedder's own allocator, or a path
that must not synchronise the device the way cudaMalloc/cudaFree can).  It
keeps its scratch in a static device array inside the library, so it must
return exactly what the allocating cflr_get_pairs_device returns.  This file
is collected last so a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

from paper_2401_11029_gb300 import cflr, gen
from paper_2401_11029_gb300.cflr import CflrError, Solver

pytestmark = pytest.mark.gpu


def _device_pairs(fn, ctx, nt, cnt, torch):
    s = torch.full((max(cnt, 1),), -1, dtype=torch.int32, device="cuda")
    d = torch.full((max(cnt, 1),), -1, dtype=torch.int32, device="cuda")
    got = fn(ctx, nt, s.data_ptr(), d.data_ptr(), cnt)
    assert got == cnt
    return s[:cnt].cpu().numpy(), d[:cnt].cpu().numpy()


def test_noalloc_extraction_equals_allocating_extraction_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    text = gen.grammar_text("fica")
    g = gen.fica_like(n=20_000, n_a=40_000, n_d=15_000, seed=2)
    with Solver(text) as s:
        s.load(g)
        s.solve()
        for name in ("M", "N3"):             # consecutive calls share the static scratch
            nt = s.nt_id(name)
            cnt = cflr.cflr_get_pairs(s.ctx, nt, count_only=True)
            assert cnt > 0
            ref = _device_pairs(cflr.cflr_get_pairs_device, s.ctx, nt, cnt, torch)
            got = _device_pairs(cflr.cflr_get_pairs_device_noalloc, s.ctx, nt, cnt, torch)
            assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1]), name


def test_noalloc_extraction_rejects_graphs_over_the_limit():
    torch = pytest.importorskip("torch")
    n = cflr.CFLR_NOALLOC_MAX_VERTICES + 1
    with Solver("S -> S S | a\n") as s:
        a, _ = cflr.cflr_symbol_id(s.ctx, "a")
        cflr.cflr_load_graph(s.ctx, n, [0, 1], [a, a], [1, n - 1])
        s.solve()
        buf = torch.empty(8, dtype=torch.int32, device="cuda")
        with pytest.raises(CflrError) as e:
            cflr.cflr_get_pairs_device_noalloc(s.ctx, 0, buf.data_ptr(), buf.data_ptr(), 8)
        assert e.value.code == cflr.CFLR_EINVAL
        assert "at most" in e.value.message
        # the allocating entry point still serves this graph
        src, dst = cflr.cflr_get_pairs(s.ctx, 0)
        assert list(zip(src.tolist(), dst.tolist())) == [(0, 1), (0, n - 1), (1, n - 1)]


def test_noalloc_extraction_at_the_vertex_limit_with_long_rows():
    """A graph of exactly CFLR_NOALLOC_MAX_VERTICES vertices: the long-row list
    fills its last slots' region and rows of more than 1024 pairs take the
    per-row bitmap (128 KiB of shared memory at this size); both entry points
    must agree, on two calls in a row."""
    torch = pytest.importorskip("torch")
    n = cflr.CFLR_NOALLOC_MAX_VERTICES
    rng = np.random.default_rng(91)
    ids = rng.choice(n, size=4000, replace=False).astype(np.uint32)
    # 'a': vertex ids[0] reaches 1500 scattered vertices directly and a path
    # of 400 more through them; 'b': a second relation with a 2000-pair row
    hub, fan, path = ids[0], ids[1:1501], ids[1501:1901]
    src_a = np.concatenate([np.full(fan.size, hub, np.uint32), path[:-1], [fan[0]]])
    dst_a = np.concatenate([fan, path[1:], [path[0]]])
    src_b = np.full(2000, ids[1901], np.uint32)
    dst_b = ids[1902:3902]
    g = gen.Graph(n=n, labels=["a", "b"], src=np.concatenate([src_a, src_b]),
                  lab=np.concatenate([np.zeros(src_a.size, np.uint32),
                                      np.ones(src_b.size, np.uint32)]),
                  dst=np.concatenate([dst_a, dst_b]))
    with Solver("S -> S S | a\nT -> b\n") as s:
        s.load(g)
        s.solve()
        for name in ("S", "T"):
            nt = s.nt_id(name)
            cnt = cflr.cflr_get_pairs(s.ctx, nt, count_only=True)
            row_len = np.bincount((s.pairs(name) >> np.uint64(32)).astype(np.int64)).max()
            assert row_len > 1024, (name, row_len)
            ref = _device_pairs(cflr.cflr_get_pairs_device, s.ctx, nt, cnt, torch)
            got = _device_pairs(cflr.cflr_get_pairs_device_noalloc, s.ctx, nt, cnt, torch)
            assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1]), name
