"""Python binding of the C ABI in ``include/cflr.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
computation of its own: the grammar compiler, the matrix initialisation, the
closure loop and the extraction all run inside ``libcflr.so`` (host C++ and
CUDA kernels for sm_103a).  If the library cannot be loaded the calls raise;
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# CFLR_LIBRARY=checked selects the bounds-checked build of the same library
LIB_PATH = os.path.join(_HERE, "libcflr_checked.so" if os.environ.get("CFLR_LIBRARY") == "checked"
                        else "libcflr.so")

CFLR_OK = 0
CFLR_EINVAL = -1
CFLR_EGRAMMAR = -2
CFLR_EGRAPH = -3
CFLR_ENOMEM = -4
CFLR_ECUDA = -5
CFLR_ELIMIT = -6
CFLR_ESTATE = -7
CFLR_ETIMEOUT = -8
CODE_NAMES = {0: "CFLR_OK", -1: "CFLR_EINVAL", -2: "CFLR_EGRAMMAR", -3: "CFLR_EGRAPH",
              -4: "CFLR_ENOMEM", -5: "CFLR_ECUDA", -6: "CFLR_ELIMIT", -7: "CFLR_ESTATE",
              -8: "CFLR_ETIMEOUT"}

CFLR_FORM_PLAIN = 0
CFLR_FORM_BATCHED = 1
CFLR_FORM_GRAPH = 2

# Every symbol include/cflr.h declares (checked by the CPU tests).
EXPORTS = ["cflr_default_config", "cflr_create", "cflr_load_grammar", "cflr_symbol_id",
           "cflr_grammar_sizes", "cflr_load_graph", "cflr_solve", "cflr_get_pairs",
           "cflr_get_pairs_device", "cflr_get_pairs_device_noalloc", "cflr_get_pairs_many",
           "cflr_get_pairs_device_many", "cflr_get_vertex_order", "cflr_reset",
           "cflr_solve_batch", "cflr_kernel_stats", "cflr_get_tuning", "cflr_set_tuning",
           "cflr_autotune", "cflr_get_witness", "cflr_last_error", "cflr_destroy"]

# Kinds of a derivation step (cflr_get_witness).
CFLR_WIT_BINARY, CFLR_WIT_EDGE, CFLR_WIT_UNIT, CFLR_WIT_EPS = 0, 1, 2, 3

# Largest graph the allocation-free extraction accepts (CFLR_NOALLOC_MAX_VERTICES).
CFLR_NOALLOC_MAX_VERTICES = 1048576


class CflrError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"{CODE_NAMES.get(code, code)}: {message}")
        self.code = code
        self.message = message


class cflr_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("mem_budget_bytes", ctypes.c_uint64), ("max_iterations", ctypes.c_uint32),
                ("form", ctypes.c_int), ("profile", ctypes.c_int),
                ("autotune_cache", ctypes.c_char_p), ("initial_capacity", ctypes.c_uint32),
                ("size_hint", ctypes.c_uint32), ("stop_on_first_converged", ctypes.c_int),
                ("keep_vertex_order", ctypes.c_int), ("witness", ctypes.c_int),
                ("test_fixed_pair_sets", ctypes.c_int), ("order_on_device", ctypes.c_int)]


class cflr_tuning(ctypes.Structure):
    _fields_ = [("probe_ratio", ctypes.c_uint32), ("bin_limit", ctypes.c_uint32 * 3),
                ("ctas_per_sm", ctypes.c_uint32 * 4)]

    def to_dict(self) -> dict:
        return {"probe_ratio": self.probe_ratio, "bin_limit": list(self.bin_limit),
                "ctas_per_sm": list(self.ctas_per_sm)}


class cflr_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_uint32), ("total_pairs", ctypes.c_uint64),
                ("solve_ms", ctypes.c_double), ("peak_device_bytes", ctypes.c_uint64),
                ("ignored_edges", ctypes.c_uint64), ("flops", ctypes.c_uint64),
                ("candidates", ctypes.c_uint64), ("regrows", ctypes.c_uint64),
                ("converged", ctypes.c_uint32), ("groups", ctypes.c_uint64 * 4),
                ("regrow_buffers", ctypes.c_uint64), ("regrow_sets", ctypes.c_uint64),
                ("regrow_pools", ctypes.c_uint64), ("flops_bin3", ctypes.c_uint64),
                ("mask_tiles_bin3", ctypes.c_uint64)]

    def to_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "groups"}
        d["groups"] = list(self.groups)
        return d


_lib = None


def load_library(path: str = LIB_PATH):
    """Load ``libcflr.so``; build it first when it is missing or stale."""
    global _lib
    if _lib is not None:
        return _lib
    from . import build as _build
    _build.build()
    if not os.path.exists(path):
        raise ImportError(f"CUDA library {path} is missing; run build() first")
    lib = ctypes.CDLL(path)
    vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lib.cflr_default_config.argtypes = [ctypes.POINTER(cflr_config)]
    lib.cflr_default_config.restype = None
    lib.cflr_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(cflr_config)]
    lib.cflr_create.restype = i32
    lib.cflr_load_grammar.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t]
    lib.cflr_load_grammar.restype = i32
    lib.cflr_symbol_id.argtypes = [vp, ctypes.c_char_p, u32p, ctypes.POINTER(i32)]
    lib.cflr_symbol_id.restype = i32
    lib.cflr_grammar_sizes.argtypes = [vp, u32p, u32p, u32p]
    lib.cflr_grammar_sizes.restype = i32
    lib.cflr_load_graph.argtypes = [vp, u32, u64, vp, vp, vp]
    lib.cflr_load_graph.restype = i32
    lib.cflr_solve.argtypes = [vp, ctypes.POINTER(cflr_stats)]
    lib.cflr_solve.restype = i32
    lib.cflr_get_pairs.argtypes = [vp, u32, vp, vp, u64, ctypes.POINTER(u64)]
    lib.cflr_get_pairs.restype = i32
    lib.cflr_get_pairs_device.argtypes = [vp, u32, vp, vp, u64, ctypes.POINTER(u64)]
    lib.cflr_get_pairs_device.restype = i32
    lib.cflr_get_pairs_device_noalloc.argtypes = [vp, u32, vp, vp, u64, ctypes.POINTER(u64)]
    lib.cflr_get_pairs_device_noalloc.restype = i32
    lib.cflr_get_vertex_order.argtypes = [vp, vp, u64]
    lib.cflr_get_vertex_order.restype = i32
    lib.cflr_get_pairs_many.argtypes = [vp, u32, vp, vp, vp, u64, vp]
    lib.cflr_get_pairs_many.restype = i32
    lib.cflr_get_pairs_device_many.argtypes = [vp, u32, vp, vp, vp, u64, vp]
    lib.cflr_get_pairs_device_many.restype = i32
    lib.cflr_get_witness.argtypes = [vp, u32, u32, u32, ctypes.POINTER(i32), u32p, u32p, u32p]
    lib.cflr_get_witness.restype = i32
    lib.cflr_reset.argtypes = [vp]
    lib.cflr_reset.restype = i32
    lib.cflr_solve_batch.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(cflr_stats)]
    lib.cflr_solve_batch.restype = i32
    lib.cflr_kernel_stats.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_char_p),
                                      ctypes.POINTER(u64), ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(u64)]
    lib.cflr_kernel_stats.restype = i32
    tp = ctypes.POINTER(cflr_tuning)
    lib.cflr_get_tuning.argtypes = [vp, tp]
    lib.cflr_get_tuning.restype = i32
    lib.cflr_set_tuning.argtypes = [vp, tp]
    lib.cflr_set_tuning.restype = i32
    lib.cflr_autotune.argtypes = [vp, u32, tp]
    lib.cflr_autotune.restype = i32
    lib.cflr_last_error.argtypes = [vp]
    lib.cflr_last_error.restype = ctypes.c_char_p
    lib.cflr_destroy.argtypes = [vp]
    lib.cflr_destroy.restype = None
    _lib = lib
    return lib


def _check(ctx, rc: int):
    if rc != CFLR_OK:
        msg = load_library().cflr_last_error(ctx).decode() if ctx else ""
        raise CflrError(rc, msg)


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint32).reshape(-1))


def cflr_default_config() -> cflr_config:
    cfg = cflr_config()
    load_library().cflr_default_config(ctypes.byref(cfg))
    return cfg


def cflr_create(cfg: cflr_config | None = None, **overrides):
    """Create a context; keyword overrides set fields of the default config."""
    lib = load_library()
    if cfg is None:
        cfg = cflr_default_config()
    for k, v in overrides.items():
        setattr(cfg, k, v)
    ctx = ctypes.c_void_p()
    rc = lib.cflr_create(ctypes.byref(ctx), ctypes.byref(cfg))
    if rc != CFLR_OK:
        raise CflrError(rc, "cflr_create failed (no usable CUDA device?)")
    return ctx


def cflr_load_grammar(ctx, text: str):
    b = text.encode()
    _check(ctx, load_library().cflr_load_grammar(ctx, b, len(b)))


def cflr_symbol_id(ctx, name: str):
    """Return (id, is_terminal) or raise CflrError for an unknown name."""
    i = ctypes.c_uint32()
    t = ctypes.c_int()
    rc = load_library().cflr_symbol_id(ctx, name.encode(), ctypes.byref(i), ctypes.byref(t))
    if rc != CFLR_OK:
        raise CflrError(rc, f"unknown symbol {name!r}")
    return int(i.value), bool(t.value)


def cflr_grammar_sizes(ctx):
    a, b, c = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    _check(ctx, load_library().cflr_grammar_sizes(ctx, ctypes.byref(a), ctypes.byref(b),
                                                  ctypes.byref(c)))
    return int(a.value), int(b.value), int(c.value)


def cflr_load_graph(ctx, n_vertices: int, src, label, dst):
    s, l, d = _u32(src), _u32(label), _u32(dst)
    if not (s.shape == l.shape == d.shape):
        raise ValueError("src, label and dst must have the same length")
    _check(ctx, load_library().cflr_load_graph(ctx, int(n_vertices), s.shape[0],
                                               s.ctypes.data, l.ctypes.data, d.ctypes.data))


def cflr_solve(ctx) -> dict:
    st = cflr_stats()
    _check(ctx, load_library().cflr_solve(ctx, ctypes.byref(st)))
    return st.to_dict()


def cflr_solve_batch(ctxs, allow_limit: bool = False) -> list:
    """Solve contexts together; with allow_limit, CFLR_ELIMIT is not an error
    (each stats dict then says whether its context converged)."""
    arr = (ctypes.c_void_p * len(ctxs))(*[c.value for c in ctxs])
    stats = (cflr_stats * len(ctxs))()
    rc = load_library().cflr_solve_batch(arr, len(ctxs), stats)
    if not (allow_limit and rc == CFLR_ELIMIT):
        _check(ctxs[0] if ctxs else None, rc)
    return [s.to_dict() for s in stats]


def cflr_get_pairs(ctx, nonterminal: int, count_only: bool = False):
    """Pairs of one non-terminal as (src, dst) uint32 arrays sorted by (src, dst)."""
    lib = load_library()
    n = ctypes.c_uint64()
    _check(ctx, lib.cflr_get_pairs(ctx, int(nonterminal), None, None, 0, ctypes.byref(n)))
    if count_only:
        return int(n.value)
    src = np.empty(n.value, dtype=np.uint32)
    dst = np.empty(n.value, dtype=np.uint32)
    if n.value:
        _check(ctx, lib.cflr_get_pairs(ctx, int(nonterminal), src.ctypes.data, dst.ctypes.data,
                                       n.value, ctypes.byref(n)))
    return src, dst


def cflr_get_pairs_device(ctx, nonterminal: int, d_src: int, d_dst: int, capacity: int) -> int:
    """Write the sorted pairs to caller-owned device buffers (raw pointers);
    returns the pair count."""
    n = ctypes.c_uint64()
    _check(ctx, load_library().cflr_get_pairs_device(ctx, int(nonterminal), ctypes.c_void_p(d_src),
                                                     ctypes.c_void_p(d_dst), int(capacity),
                                                     ctypes.byref(n)))
    return int(n.value)


def cflr_get_pairs_many(ctx, nonterminals, count_only: bool = False, out=None):
    """Pairs of several non-terminals in one call: (src, dst, offsets), the
    pairs of nonterminals[i] being src[offsets[i]:offsets[i + 1]] (and dst
    alike), each sorted by (src, dst).  With count_only, only the offsets.
    `out` may give (src, dst) host arrays (uint32, C-contiguous) to write
    into, e.g. views of pinned memory; they must hold the total."""
    lib = load_library()
    ids = np.ascontiguousarray(nonterminals, dtype=np.uint32)
    off = np.empty(ids.size + 1, dtype=np.uint64)
    _check(ctx, lib.cflr_get_pairs_many(ctx, ids.size, ids.ctypes.data, None, None, 0,
                                        off.ctypes.data))
    if count_only:
        return off
    total = int(off[-1])
    if out is None:
        src = np.empty(total, dtype=np.uint32)
        dst = np.empty(total, dtype=np.uint32)
    else:
        src, dst = out
        if src.dtype != np.uint32 or dst.dtype != np.uint32 or not (
                src.flags.c_contiguous and dst.flags.c_contiguous):
            raise ValueError("out arrays must be C-contiguous uint32")
        if min(src.size, dst.size) < total:
            raise ValueError(f"out arrays hold {min(src.size, dst.size)} pairs, need {total}")
    if total:
        _check(ctx, lib.cflr_get_pairs_many(ctx, ids.size, ids.ctypes.data, src.ctypes.data,
                                            dst.ctypes.data, min(src.size, dst.size),
                                            off.ctypes.data))
    return src[:total], dst[:total], off


def cflr_get_pairs_device_many(ctx, nonterminals, d_src: int, d_dst: int,
                               capacity: int) -> np.ndarray:
    """Write the pairs of several non-terminals one after another to
    caller-owned device buffers (raw pointers); returns the offsets (uint64,
    one more than the non-terminals)."""
    ids = np.ascontiguousarray(nonterminals, dtype=np.uint32)
    off = np.empty(ids.size + 1, dtype=np.uint64)
    _check(ctx, load_library().cflr_get_pairs_device_many(
        ctx, ids.size, ids.ctypes.data, ctypes.c_void_p(d_src), ctypes.c_void_p(d_dst),
        int(capacity), off.ctypes.data))
    return off


def cflr_get_witness(ctx, nonterminal: int, src: int, dst: int):
    """The derivation step recorded for (src, dst) in `nonterminal` (the
    context must have been created with witness=1): (kind, id, id2, mid)."""
    k = ctypes.c_int()
    a, b, m = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    _check(ctx, load_library().cflr_get_witness(ctx, int(nonterminal), int(src), int(dst),
                                                ctypes.byref(k), ctypes.byref(a),
                                                ctypes.byref(b), ctypes.byref(m)))
    return k.value, a.value, b.value, m.value


def cflr_get_pairs_device_noalloc(ctx, nonterminal: int, d_src: int, d_dst: int,
                                  capacity: int) -> int:
    """As cflr_get_pairs_device, for callers that may not allocate device
    memory: the scratch lives in a static device array inside the library, so
    the graph may have at most CFLR_NOALLOC_MAX_VERTICES vertices and calls
    that overlap on the GPU must not be issued.  Returns the pair count."""
    n = ctypes.c_uint64()
    _check(ctx, load_library().cflr_get_pairs_device_noalloc(
        ctx, int(nonterminal), ctypes.c_void_p(d_src), ctypes.c_void_p(d_dst), int(capacity),
        ctypes.byref(n)))
    return int(n.value)


def cflr_get_vertex_order(ctx, n_vertices: int) -> np.ndarray:
    """The caller's id of the vertex stored as each row (uint32, n_vertices)."""
    out = np.empty(max(int(n_vertices), 1), dtype=np.uint32)
    _check(ctx, load_library().cflr_get_vertex_order(ctx, out.ctypes.data, out.size))
    return out[:int(n_vertices)]


def cflr_reset(ctx):
    _check(ctx, load_library().cflr_reset(ctx))


def cflr_kernel_stats(ctx) -> list:
    lib = load_library()
    cnt = ctypes.c_uint64()
    _check(ctx, lib.cflr_kernel_stats(ctx, -1, None, ctypes.byref(cnt), None, None))
    out = []
    for k in range(cnt.value):
        name = ctypes.c_char_p()
        launches, ms, by = ctypes.c_uint64(), ctypes.c_double(), ctypes.c_uint64()
        _check(ctx, lib.cflr_kernel_stats(ctx, k, ctypes.byref(name), ctypes.byref(launches),
                                          ctypes.byref(ms), ctypes.byref(by)))
        out.append({"name": name.value.decode(), "launches": int(launches.value),
                    "ms": float(ms.value), "alg_bytes": int(by.value)})
    return out


def cflr_get_tuning(ctx) -> dict:
    t = cflr_tuning()
    _check(ctx, load_library().cflr_get_tuning(ctx, ctypes.byref(t)))
    return t.to_dict()


def cflr_set_tuning(ctx, probe_ratio: int, bin_limit, ctas_per_sm):
    t = cflr_tuning(probe_ratio, (ctypes.c_uint32 * 3)(*bin_limit),
                    (ctypes.c_uint32 * 4)(*ctas_per_sm))
    _check(ctx, load_library().cflr_set_tuning(ctx, ctypes.byref(t)))


def cflr_autotune(ctx, max_trials: int = 0) -> dict:
    """Measure and set the product-kernel schedule for the loaded graph;
    returns it.  The matrices are left at the terminal initialisation."""
    t = cflr_tuning()
    _check(ctx, load_library().cflr_autotune(ctx, int(max_trials), ctypes.byref(t)))
    return t.to_dict()


def cflr_last_error(ctx) -> str:
    return load_library().cflr_last_error(ctx).decode()


def cflr_destroy(ctx):
    if ctx is not None and ctx.value:
        load_library().cflr_destroy(ctx)


# ---------------------------------------------------------------------------
# Convenience wrapper (still only marshalling)
# ---------------------------------------------------------------------------

class Solver:
    """One context with a grammar; ``load(graph)`` maps label names to ids."""

    def __init__(self, grammar_text: str, **config):
        self.ctx = cflr_create(**config)
        try:
            cflr_load_grammar(self.ctx, grammar_text)
            self.n_nt, self.n_named, self.n_terms = cflr_grammar_sizes(self.ctx)
        except Exception:
            cflr_destroy(self.ctx)
            raise
        self.stats = None

    def close(self):
        cflr_destroy(self.ctx)
        self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def label_ids(self, labels) -> np.ndarray:
        """Terminal id of each label name, 0xFFFFFFFF for names the grammar lacks."""
        out = []
        for name in labels:
            try:
                i, term = cflr_symbol_id(self.ctx, name)
                out.append(i if term else 0xFFFFFFFF)
            except CflrError:
                out.append(0xFFFFFFFF)
        return np.asarray(out, dtype=np.uint32)

    def load(self, graph):
        ids = self.label_ids(graph.labels)
        cflr_load_graph(self.ctx, graph.n, graph.src, ids[graph.lab], graph.dst)

    def solve(self) -> dict:
        self.stats = cflr_solve(self.ctx)
        return self.stats

    def nt_id(self, name: str) -> int:
        i, term = cflr_symbol_id(self.ctx, name)
        if term:
            raise CflrError(CFLR_EINVAL, f"{name!r} is a terminal")
        return i

    def pairs(self, name: str) -> np.ndarray:
        """Sorted uint64 keys src << 32 | dst of one non-terminal."""
        s, d = cflr_get_pairs(self.ctx, self.nt_id(name))
        return (s.astype(np.uint64) << np.uint64(32)) | d.astype(np.uint64)

    def pairs_many(self, names) -> dict:
        """Sorted uint64 keys of several non-terminals, read out in one call
        (cflr_get_pairs_many): name -> keys."""
        names = list(names)
        s, d, off = cflr_get_pairs_many(self.ctx, [self.nt_id(x) for x in names])
        keys = (s.astype(np.uint64) << np.uint64(32)) | d.astype(np.uint64)
        return {x: keys[int(off[i]):int(off[i + 1])] for i, x in enumerate(names)}

    def count(self, name: str) -> int:
        return cflr_get_pairs(self.ctx, self.nt_id(name), count_only=True)

    def path(self, name: str, src: int, dst: int, labels: list) -> list:
        """A path src -> dst whose label word `name` derives, rebuilt from
        the recorded derivation steps (needs witness=1): a list of edges
        (u, label name, v).  `labels` maps terminal ids to names."""
        out = []
        stack = [(self.nt_id(name), src, dst)]
        while stack:                   # depth first, left operand first
            x, u, v = stack.pop()
            kind, a, b, m = cflr_get_witness(self.ctx, x, u, v)
            if kind == CFLR_WIT_EDGE:
                out.append((u, labels[a], v))
            elif kind == CFLR_WIT_UNIT:
                stack.append((a, u, v))
            elif kind == CFLR_WIT_BINARY:
                stack.append((b, m, v))
                stack.append((a, u, m))
        return out
