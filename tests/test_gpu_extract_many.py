"""Extraction of several non-terminals in one call (cflr_get_pairs_many and
cflr_get_pairs_device_many) against the oracle and the one-at-a-time calls.

The result of Algorithm 1 for each non-terminal must be the same set, in the
same (src, dst) order, whichever call reads it out."""
import numpy as np
import pytest

import oracle
from common import keys_of
from paper_2401_11029_gb300 import cflr, gen
from paper_2401_11029_gb300.cflr import CflrError, Solver

pytestmark = pytest.mark.gpu


def _solved(text, g):
    s = Solver(text, form=cflr.CFLR_FORM_GRAPH)
    s.load(g)
    s.solve()
    return s


def test_many_equals_oracle_and_single_calls():
    # the field-sensitive alias grammar (Fig. wcnf:fsca) with 8 field indices
    # (dozens of non-terminals); no edge of field 7, so some are empty
    text = gen.grammar_text("fsca", index_hi=7)
    g0 = gen.fsca_like(n=2500, n_edges=3500, fields=8, seed=31)
    gone = [g0.labels.index(x) for x in ("f_7", "f_r_7") if x in g0.labels]
    keep = ~np.isin(g0.lab, gone)
    g = gen.Graph(n=g0.n, labels=g0.labels, src=g0.src[keep], lab=g0.lab[keep],
                  dst=g0.dst[keep])
    want = oracle.solve(text, g)
    names = want.grammar.nts
    with _solved(text, g) as s:
        ids = [s.nt_id(x) for x in names]
        # an id repeated, and the list in an order of its own
        ids = ids[::-1] + ids[:3]
        names = names[::-1] + names[:3]
        src, dst, off = cflr.cflr_get_pairs_many(s.ctx, ids)
        assert off.size == len(ids) + 1 and off[0] == 0 and off[-1] == src.size
        assert np.all(np.diff(off.astype(np.int64)) >= 0)
        assert gone and any(off[i] == off[i + 1] for i in range(len(ids)))   # empty ones
        for i, (x, nt) in enumerate(zip(names, ids)):
            a, b = int(off[i]), int(off[i + 1])
            got = keys_of(src[a:b], dst[a:b])
            assert np.array_equal(got, want.pairs[x]), x
            s1, d1 = cflr.cflr_get_pairs(s.ctx, nt)
            assert np.array_equal(s1, src[a:b]) and np.array_equal(d1, dst[a:b]), x
        # offsets only
        assert np.array_equal(cflr.cflr_get_pairs_many(s.ctx, ids, count_only=True), off)
        # the Solver's name-keyed form
        by_name = s.pairs_many(want.grammar.nts)
        for x in want.grammar.nts:
            assert np.array_equal(by_name[x], want.pairs[x]), x


def test_device_many_equals_host_many():
    import torch
    text = gen.grammar_text("fica")
    g = gen.fica_like(n=6000, n_a=12000, n_d=4500, seed=32)
    with _solved(text, g) as s:
        ids = list(range(s.n_named))
        src, dst, off = cflr.cflr_get_pairs_many(s.ctx, ids)
        total = int(off[-1])
        out = (torch.full((total + 7,), -1, dtype=torch.int32, device="cuda"),
               torch.full((total + 7,), -1, dtype=torch.int32, device="cuda"))
        for _ in range(2):          # the second call runs on reused scratch
            doff = cflr.cflr_get_pairs_device_many(s.ctx, ids, out[0].data_ptr(),
                                                   out[1].data_ptr(), total + 7)
            assert np.array_equal(doff, off)
            ds = out[0].cpu().numpy().view(np.uint32)
            dd = out[1].cpu().numpy().view(np.uint32)
            assert np.array_equal(ds[:total], src) and np.array_equal(dd[:total], dst)
            assert np.all(ds[total:] == 0xFFFFFFFF)        # nothing past the total


def test_many_into_caller_arrays_and_errors():
    text = gen.grammar_text("fica")
    g = gen.fica_like(n=3000, n_a=6000, n_d=2000, seed=33)
    with _solved(text, g) as s:
        ids = list(range(s.n_named))
        src, dst, off = cflr.cflr_get_pairs_many(s.ctx, ids)
        total = int(off[-1])
        assert total > 0
        buf = (np.zeros(total + 5, dtype=np.uint32), np.zeros(total + 5, dtype=np.uint32))
        s2, d2, off2 = cflr.cflr_get_pairs_many(s.ctx, ids, out=buf)
        assert np.array_equal(off2, off) and np.array_equal(s2, src) and np.array_equal(d2, dst)
        # capacity below the total: CFLR_EINVAL, offsets still filled
        lib = cflr.load_library()
        ida = np.asarray(ids, dtype=np.uint32)
        o3 = np.zeros(len(ids) + 1, dtype=np.uint64)
        small = np.zeros(total - 1, dtype=np.uint32)
        rc = lib.cflr_get_pairs_many(s.ctx, len(ids), ida.ctypes.data, small.ctypes.data,
                                     small.ctypes.data, total - 1, o3.ctypes.data)
        assert rc == cflr.CFLR_EINVAL and np.array_equal(o3, off)
        # a bad id, NULL offsets, one array of two
        with pytest.raises(CflrError):
            cflr.cflr_get_pairs_many(s.ctx, [0, 10_000])
        assert lib.cflr_get_pairs_many(s.ctx, len(ids), ida.ctypes.data, None, None, 0,
                                       None) == cflr.CFLR_EINVAL
        assert lib.cflr_get_pairs_many(s.ctx, len(ids), ida.ctypes.data, small.ctypes.data,
                                       None, total, o3.ctypes.data) == cflr.CFLR_EINVAL
        # no non-terminals: one offset, zero
        e_s, e_d, e_off = cflr.cflr_get_pairs_many(s.ctx, [])
        assert e_s.size == 0 and list(e_off) == [0]
        # the context still answers
        s4, d4, off4 = cflr.cflr_get_pairs_many(s.ctx, ids)
        assert np.array_equal(off4, off) and np.array_equal(s4, src)


def test_many_before_a_graph_is_a_state_error():
    with Solver(gen.grammar_text("fica")) as s:
        with pytest.raises(CflrError) as e:
            cflr.cflr_get_pairs_many(s.ctx, [0])
        assert e.value.code == cflr.CFLR_ESTATE


def test_pinned_host_arrays():
    # pinned host arrays (the copies run asynchronously on a second stream)
    # get what pageable ones get
    import torch
    text = gen.grammar_text("fica")
    g = gen.fica_like(n=6000, n_a=12000, n_d=4500, seed=34)
    with _solved(text, g) as s:
        ids = list(range(s.n_named))
        src, dst, off = cflr.cflr_get_pairs_many(s.ctx, ids)          # pageable
        total = int(off[-1])
        ps = torch.full((total + 3,), -1, dtype=torch.int32).pin_memory()
        pd = torch.full((total + 3,), -1, dtype=torch.int32).pin_memory()
        out = (ps.numpy().view(np.uint32), pd.numpy().view(np.uint32))
        s2, d2, off2 = cflr.cflr_get_pairs_many(s.ctx, ids, out=out)
        assert np.array_equal(off2, off) and np.array_equal(s2, src) and np.array_equal(d2, dst)
        assert np.all(out[0][total:] == 0xFFFFFFFF)
        # one non-terminal into a pinned array at an offset inside it
        x = int(np.argmax(np.diff(off.astype(np.int64))))
        a, b = int(off[x]), int(off[x + 1])
        lib = cflr.load_library()
        import ctypes
        n_p = ctypes.c_uint64()
        assert lib.cflr_get_pairs(s.ctx, ids[x], ps.data_ptr() + 12, pd.data_ptr() + 12, b - a,
                                  ctypes.byref(n_p)) == 0
        assert np.array_equal(out[0][3:3 + b - a], src[a:b])
        assert np.array_equal(out[1][3:3 + b - a], dst[a:b])
