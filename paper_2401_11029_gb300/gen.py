"""Seeded synthetic inputs: grammar texts and edge-labelled graphs.

This module is shared by the CUDA path, the oracle and the tests.  It holds no
part of the CFL-reachability computation: it only produces inputs (a grammar
text and a list of labelled edges), so that both sides read identical data.

All sampling is integer-only (numpy PCG64 integer draws, integer CDF tables and
``searchsorted``), so the same seed yields the same graph on x86-64 and
aarch64.  The few floating-point values (Zipf weight tables, log-uniform sizes)
are computed in scalar Python and rounded to integers before use.

Workload shapes follow the evaluation of the paper (Sec. 4, Table "graph"):
program-analysis graphs with |E|/|V| around 2-3, few labels (alias analysis)
or thousands of indexed labels (field-sensitive points-to), and cycle-free
forward edges (cycle elimination precedes CFL-r, Sec. 4 footnote on CPU17).
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field

import numpy as np

_GRAMMAR_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "grammars")

# Locality parameters of the program-shaped generator (frozen after calibration
# against the oracle; the values and the resulting closure sizes are recorded
# with the workload recipe in the design notes).
DEFAULT_WINDOW = 64
DEFAULT_P_LONG = 0.002
DEFAULT_K_MAX = 1024
ZIPF_S = 2.1


def grammar_text(name: str, index_hi: int | None = None) -> str:
    """Return the text of grammar ``name`` (a file under ``grammars/``).

    ``index_hi`` replaces the upper bound of every ``%index`` line, which lets
    tests use the indexed grammars with fewer fields.
    """
    with open(os.path.join(_GRAMMAR_DIR, name + ".wcnf")) as f:
        text = f.read()
    if index_hi is not None:
        out = []
        for line in text.splitlines():
            parts = line.split()
            if parts and parts[0] == "%index":
                line = f"%index {parts[1]} {parts[2]} {index_hi}"
            out.append(line)
        text = "\n".join(out) + "\n"
    return text


@dataclass
class Graph:
    """An edge-labelled graph: edge e goes ``src[e] --labels[lab[e]]--> dst[e]``."""

    n: int
    labels: list
    src: np.ndarray
    lab: np.ndarray
    dst: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def n_edges(self) -> int:
        return int(self.src.shape[0])

    def label_counts(self) -> dict:
        cnt = np.bincount(self.lab, minlength=len(self.labels))
        return {name: int(c) for name, c in zip(self.labels, cnt)}

    def edge_digest(self) -> str:
        """A short hex digest of the edge list (order-independent)."""
        keys = (self.src.astype(np.uint64) << np.uint64(40)) ^ (
            self.lab.astype(np.uint64) << np.uint64(20)) ^ self.dst.astype(np.uint64)
        h = _mix64(keys ^ np.uint64(self.n))
        return "%016x" % int(np.bitwise_xor.reduce(h) if h.size else 0) + "%016x" % int(
            np.sum(h, dtype=np.uint64) if h.size else 0)


def pair_keys(src, dst) -> np.ndarray:
    """Pairs (src[i], dst[i]) as 64-bit keys src << 32 | dst."""
    return (np.asarray(src).astype(np.uint32).astype(np.uint64) << np.uint64(32)) | \
        np.asarray(dst).astype(np.uint32).astype(np.uint64)


def pair_fingerprint(keys: np.ndarray) -> str:
    """Order-independent digest of a set of 64-bit pair keys: the count, and
    the xor and the sum of a 64-bit mix of every key.  Stored fingerprints of
    the oracle's full-size results are compared against it."""
    x = np.asarray(keys).astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        x ^= x >> np.uint64(31)
        x *= np.uint64(0x7FB5D329728EA185)
        x ^= x >> np.uint64(27)
        x *= np.uint64(0x81DADEF4BC2DD44D)
        x ^= x >> np.uint64(33)
    xr = int(np.bitwise_xor.reduce(x)) if x.size else 0
    sm = int(np.sum(x, dtype=np.uint64)) if x.size else 0
    return "%d:%016x:%016x" % (x.size, xr, sm)


def _mix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser on a uint64 array (wrapping arithmetic)."""
    x = x.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        x ^= x >> np.uint64(30)
        x *= np.uint64(0xBF58476D1CE4E5B9)
        x ^= x >> np.uint64(27)
        x *= np.uint64(0x94D049BB133111EB)
        x ^= x >> np.uint64(31)
    return x


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def zipf_cdf(s: float, k_max: int) -> np.ndarray:
    """Integer CDF of a Zipf law P(k) ~ k^-s on k = 1..k_max (weights scaled to 2^40)."""
    w = [int(round(math.ldexp(1.0, 40) * math.pow(k, -s))) for k in range(1, k_max + 1)]
    w = [max(1, x) for x in w]
    return np.cumsum(np.asarray(w, dtype=np.int64))


def sample_cdf(rng: np.random.Generator, cdf: np.ndarray, size: int) -> np.ndarray:
    """Draw ``size`` indices i (0-based) with probability (cdf[i]-cdf[i-1])/cdf[-1]."""
    u = rng.integers(0, int(cdf[-1]), size=size, dtype=np.int64)
    return np.searchsorted(cdf, u, side="right").astype(np.int64)


def _take_distinct(keys_chunks: list, want: int) -> np.ndarray:
    """First ``want`` distinct keys in generation order, or all if fewer."""
    keys = np.concatenate(keys_chunks)
    _, first = np.unique(keys, return_index=True)
    first.sort()
    return keys[first[:want]]


class _Locality:
    """Program-shaped edge sampler over one vertex population.

    The population is put in a seeded random order and cut into consecutive
    blocks of ``window`` vertices ("procedures").  Sources are drawn Chung-Lu
    style from Zipf(``s``) vertex weights truncated at ``k_max``.  A target is
    uniform over the later positions of the source's own block; with
    probability ``p_long`` it is uniform over the next ``LONG_BLOCKS`` blocks
    instead (an inter-procedural edge).  These edges therefore form a DAG,
    like the cycle-eliminated graphs the paper evaluates on, and reachability
    stays mostly inside a procedure and its few callees at every graph size.
    """

    LONG_BLOCKS = 64

    def __init__(self, rng, verts: np.ndarray, window: int, p_long: float, k_max: int,
                 s: float = ZIPF_S):
        self.rng = rng
        self.verts = verts.astype(np.int64)
        m = self.verts.shape[0]
        self.order = rng.permutation(m)             # position -> index into verts
        self.pos = np.empty(m, dtype=np.int64)      # index into verts -> position
        self.pos[self.order] = np.arange(m, dtype=np.int64)
        wk = sample_cdf(rng, zipf_cdf(s, k_max), m) + 1
        self.cw = np.cumsum(wk)
        self.window = max(1, int(window))
        self.thr = int(round(p_long * (1 << 32)))

    def sample(self, size: int):
        """``size`` draws of (src, dst); a draw is dropped when its source has
        no later vertex in its block (a block-local draw) or no block after
        its own (a long draw), so fewer may come back."""
        rng, m, W = self.rng, self.verts.shape[0], self.window
        si = np.searchsorted(self.cw, rng.integers(0, int(self.cw[-1]), size=size,
                                                   dtype=np.int64), side="right")
        longp = rng.integers(0, 1 << 32, size=size, dtype=np.int64) < self.thr
        r = rng.integers(0, 1 << 62, size=size, dtype=np.int64)
        p = self.pos[si]
        block_end = np.minimum((p // W + 1) * W, m)    # first position after the block
        in_block = block_end - 1 - p                   # later positions in the block
        far_end = np.minimum(block_end + self.LONG_BLOCKS * W, m)
        later = far_end - block_end                    # positions in the next blocks
        ok = np.where(longp, later > 0, in_block > 0)
        near = p + 1 + r % np.maximum(in_block, 1)
        far = block_end + r % np.maximum(later, 1)
        tpos = np.minimum(np.where(longp, far, near), m - 1)
        ti = self.order[tpos]
        return self.verts[si[ok]], self.verts[ti[ok]]


def _distinct_edges(sampler_fn, want: int, n: int, n_labels: int, label: int):
    """Sample edges with ``sampler_fn(size) -> (src, dst)`` until ``want`` distinct."""
    chunks = []
    have = 0
    rounds = 0
    while have < want:
        ask = max(1024, int((want - have) * 1.25) + 16)
        s, d = sampler_fn(ask)
        chunks.append((s * n_labels + label) * n + d)
        have = np.unique(np.concatenate(chunks)).shape[0]
        rounds += 1
        if rounds > 64:
            raise RuntimeError("edge sampler cannot reach the requested distinct count")
    return _take_distinct(chunks, want)


def _keys_to_graph(n, labels, keys: np.ndarray, meta) -> Graph:
    L = len(labels)
    keys = keys.astype(np.int64)
    dst = keys % n
    rest = keys // n
    lab = rest % L
    src = rest // L
    return Graph(n=n, labels=list(labels), src=src.astype(np.uint32),
                 lab=lab.astype(np.uint32), dst=dst.astype(np.uint32), meta=meta)


def _with_reverses(g: Graph, pairs: dict) -> Graph:
    """Append, for each forward label x in ``pairs``, the reversed edge labelled pairs[x]."""
    labels = list(g.labels)
    for rev in pairs.values():
        if rev not in labels:
            labels.append(rev)
    src, lab, dst = [g.src], [g.lab], [g.dst]
    for fwd, rev in pairs.items():
        fi = g.labels.index(fwd)
        sel = g.lab == fi
        src.append(g.dst[sel])
        dst.append(g.src[sel])
        lab.append(np.full(int(sel.sum()), labels.index(rev), dtype=np.uint32))
    return Graph(n=g.n, labels=labels, src=np.concatenate(src), lab=np.concatenate(lab),
                 dst=np.concatenate(dst), meta=dict(g.meta))


# ---------------------------------------------------------------------------
# The five workloads
# ---------------------------------------------------------------------------

def dyck1_er(n: int = 1000, n_a: int = 1500, n_b: int = 1500, seed: int = 1) -> Graph:
    """Dyck-1 workload: Erdos-Renyi digraph, ``n_a`` 'a' and ``n_b`` 'b' edges.

    Endpoints are uniform (self-loops allowed); each (src, label, dst) triple is
    distinct.
    """
    rng = _rng(seed)
    labels = ["a", "b"]
    keys = []
    for li, want in enumerate((n_a, n_b)):
        def fn(size):
            return (rng.integers(0, n, size=size, dtype=np.int64),
                    rng.integers(0, n, size=size, dtype=np.int64))
        keys.append(_distinct_edges(fn, want, n, 2, li))
    return _keys_to_graph(n, labels, np.concatenate(keys),
                          {"workload": "dyck1_er", "seed": seed})


def fica_like(n: int = 200_000, n_a: int = 400_000, n_d: int = 150_000, seed: int = 2,
              window: int = DEFAULT_WINDOW, p_long: float = DEFAULT_P_LONG,
              k_max: int = DEFAULT_K_MAX) -> Graph:
    """Memory-alias workload: 'a' (assignment) and 'd' (dereference) edges plus
    their reverses 'a_r' and 'd_r' (the barred labels of Fig. "wcnf:fica").
    """
    rng = _rng(seed)
    loc = _Locality(rng, np.arange(n), window, p_long, k_max)
    labels = ["a", "d"]
    keys = [_distinct_edges(loc.sample, n_a, n, 2, 0),
            _distinct_edges(loc.sample, n_d, n, 2, 1)]
    g = _keys_to_graph(n, labels, np.concatenate(keys),
                       {"workload": "fica_like", "seed": seed, "window": window,
                        "p_long": p_long, "k_max": k_max})
    return _with_reverses(g, {"a": "a_r", "d": "d_r"})


def fsjpt_like(n: int = 500_000, n_edges: int = 2_000_000, fields: int = 64, seed: int = 3,
               window: int = DEFAULT_WINDOW, p_long: float = DEFAULT_P_LONG,
               k_max: int = DEFAULT_K_MAX, field_s: float = 1.0) -> Graph:
    """Field-sensitive points-to workload (Fig. "wcnf:fsjpt" labels).

    10 % of vertices are objects, the rest variables; variables fall into
    procedures of ``window`` variables, each owning ``window``/9 objects.
    Forward edges: 40 % assign (variable -> variable), 10 % alloc (variable
    -> an object of its procedure, or any object with probability p_long), 50 %
    load_i / store_i split evenly (variable -> variable) with the field index i
    drawn Zipf(``field_s``) over ``fields`` fields.  Every edge also gets its
    reverse (alloc_r, assign_r, load_r_i, store_r_i).
    """
    rng = _rng(seed)
    perm = rng.permutation(n)
    n_obj = n // 10
    objs, vars_ = np.sort(perm[:n_obj]), np.sort(perm[n_obj:])
    loc = _Locality(rng, vars_, window, p_long, k_max)
    labels = ["assign", "alloc"] + [f"load_{i}" for i in range(fields)] + \
             [f"store_{i}" for i in range(fields)]
    L = len(labels)
    n_assign = n_edges * 4 // 10
    n_alloc = n_edges // 10
    n_ls = n_edges - n_assign - n_alloc
    n_load = n_ls // 2
    n_store = n_ls - n_load
    keys = [_distinct_edges(loc.sample, n_assign, n, L, 0)]

    obj_rank = rng.permutation(n_obj)
    per_block = max(1, n_obj * window // max(1, vars_.shape[0]))   # objects per procedure
    thr = int(round(p_long * (1 << 32)))

    def alloc_fn(size):
        # a variable allocates one of its own procedure's objects; with
        # probability p_long any object (a factory or global)
        s, _ = loc.sample(size)
        blk = loc.pos[np.searchsorted(vars_, s)] // window
        near = (blk * per_block + rng.integers(0, per_block, size=s.shape[0],
                                               dtype=np.int64)) % n_obj
        far = rng.integers(0, n_obj, size=s.shape[0], dtype=np.int64)
        longp = rng.integers(0, 1 << 32, size=s.shape[0], dtype=np.int64) < thr
        return s, objs[obj_rank[np.where(longp, far, near)]]
    keys.append(_distinct_edges(alloc_fn, n_alloc, n, L, 1))

    fcdf = zipf_cdf(field_s, fields)
    for kind, count in (("load", n_load), ("store", n_store)):
        base_label = 2 if kind == "load" else 2 + fields
        fidx = sample_cdf(rng, fcdf, count)
        per_field = np.bincount(fidx, minlength=fields)
        for i in range(fields):
            if per_field[i]:
                keys.append(_distinct_edges(loc.sample, int(per_field[i]), n, L,
                                            base_label + i))
    g = _keys_to_graph(n, labels, np.concatenate(keys),
                       {"workload": "fsjpt_like", "seed": seed, "fields": fields,
                        "window": window, "p_long": p_long, "k_max": k_max})
    rev = {"assign": "assign_r", "alloc": "alloc_r"}
    rev.update({f"load_{i}": f"load_r_{i}" for i in range(fields)})
    rev.update({f"store_{i}": f"store_r_{i}" for i in range(fields)})
    return _with_reverses(g, rev)


def fsca_like(n: int = 41_652, n_edges: int = 55_775, fields: int = 142, seed: int = 6,
              window: int = DEFAULT_WINDOW, p_long: float = DEFAULT_P_LONG,
              k_max: int = DEFAULT_K_MAX, field_s: float = 1.0) -> Graph:
    """Field-sensitive C/C++ alias workload (Fig. "wcnf:fsca" labels).

    Forward edges from the program-shaped sampler: 45 % 'a' (assignment),
    25 % 'd' (dereference) and 30 % 'f_i' (access of field i, i drawn
    Zipf(``field_s``) over ``fields`` fields); every edge also gets its
    reverse (a_r, d_r, f_r_i).  The defaults take the shape of the paper's
    imagick graph (41,652 vertices, 111,550 edges with reverses, 288 labels:
    142 fields).
    """
    rng = _rng(seed)
    loc = _Locality(rng, np.arange(n), window, p_long, k_max)
    labels = ["a", "d"] + [f"f_{i}" for i in range(fields)]
    L = len(labels)
    n_a = n_edges * 45 // 100
    n_d = n_edges * 25 // 100
    n_f = n_edges - n_a - n_d
    keys = [_distinct_edges(loc.sample, n_a, n, L, 0), _distinct_edges(loc.sample, n_d, n, L, 1)]
    per_field = np.bincount(sample_cdf(rng, zipf_cdf(field_s, fields), n_f), minlength=fields)
    for i in range(fields):
        if per_field[i]:
            keys.append(_distinct_edges(loc.sample, int(per_field[i]), n, L, 2 + i))
    g = _keys_to_graph(n, labels, np.concatenate(keys),
                       {"workload": "fsca_like", "seed": seed, "fields": fields,
                        "window": window, "p_long": p_long, "k_max": k_max})
    rev = {"a": "a_r", "d": "d_r"}
    rev.update({f"f_{i}": f"f_r_{i}" for i in range(fields)})
    return _with_reverses(g, rev)


def cscvf_like(n: int = 346_034, n_edges: int = 581_210, calls: int = 5_655, seed: int = 7,
               window: int = DEFAULT_WINDOW, p_long: float = DEFAULT_P_LONG,
               k_max: int = DEFAULT_K_MAX, callee_s: float = 1.0) -> Graph:
    """Context-sensitive C/C++ value-flow workload (Fig. "wcnf:cscvf" labels).

    The vertices fall into procedures (the blocks of the program-shaped
    sampler).  Intraprocedural flow is ``n_edges - 2 calls`` 'a' edges from the
    sampler.  Call site i joins a caller procedure (uniform) and a callee
    (Zipf(``callee_s``) over procedures, so a few functions are called from
    many sites): 'call_i' from a vertex of the caller to the callee's first
    vertex, and 'ret_i' from the callee's last vertex to a later vertex of the
    caller (the call's result).  The defaults take the shape of the paper's
    povray graph (346,034 vertices, 581,210 edges, 11,311 labels: 5,655 call
    sites).
    """
    rng = _rng(seed)
    loc = _Locality(rng, np.arange(n), window, p_long, k_max)
    labels = ["a"] + [f"call_{i}" for i in range(calls)] + [f"ret_{i}" for i in range(calls)]
    L = len(labels)
    keys = [_distinct_edges(loc.sample, n_edges - 2 * calls, n, L, 0)]
    W = max(1, int(window))
    n_blocks = (n + W - 1) // W
    caller = rng.integers(0, n_blocks, size=calls, dtype=np.int64)
    callee = (sample_cdf(rng, zipf_cdf(callee_s, n_blocks), calls) +
              rng.integers(0, n_blocks, size=calls, dtype=np.int64)) % n_blocks
    b_lo = caller * W
    b_len = np.minimum(b_lo + W, n) - b_lo
    at = b_lo + rng.integers(0, 1 << 62, size=calls, dtype=np.int64) % b_len
    back = at + rng.integers(0, 1 << 62, size=calls, dtype=np.int64) % (b_lo + b_len - at)
    entry = callee * W
    exit_ = np.minimum(entry + W, n) - 1
    ci = np.arange(calls, dtype=np.int64)
    keys.append((loc.order[at] * L + 1 + ci) * n + loc.order[entry])
    keys.append((loc.order[exit_] * L + 1 + calls + ci) * n + loc.order[back])
    return _keys_to_graph(n, labels, np.concatenate(keys),
                          {"workload": "cscvf_like", "seed": seed, "calls": calls,
                           "window": window, "p_long": p_long, "k_max": k_max})


def log_uniform_int(rng: np.random.Generator, lo: int, hi: int) -> int:
    """An integer log-uniform in [lo, hi] (scalar math, rounded down)."""
    u = int(rng.integers(0, 1 << 53)) / float(1 << 53)
    return min(hi, int(lo * math.exp(u * math.log(hi / lo))))


def dyck3_instance(seed: int, n_lo: int = 1000, n_hi: int = 50_000,
                   window: int = DEFAULT_WINDOW, p_long: float = DEFAULT_P_LONG,
                   k_max: int = DEFAULT_K_MAX) -> Graph:
    """One batched Dyck-3 instance: n log-uniform in [n_lo, n_hi], 3n edges with
    labels uniform over a_1, b_1, a_2, b_2, a_3, b_3."""
    rng = _rng(seed)
    n = log_uniform_int(rng, n_lo, n_hi)
    loc = _Locality(rng, np.arange(n), window, p_long, k_max)
    labels = ["a_1", "b_1", "a_2", "b_2", "a_3", "b_3"]
    per = np.bincount(rng.integers(0, 6, size=3 * n, dtype=np.int64), minlength=6)
    keys = [_distinct_edges(loc.sample, int(per[li]), n, 6, li) for li in range(6) if per[li]]
    return _keys_to_graph(n, labels, np.concatenate(keys),
                          {"workload": "dyck3", "seed": seed})


def dyck3_batch(count: int = 256, seed0: int = 4000, **kw) -> list:
    """``count`` independent Dyck-3 instances with seeds seed0 .. seed0+count-1."""
    return [dyck3_instance(seed0 + k, **kw) for k in range(count)]


@dataclass
class Request:
    """One serving request: arrival time (s) and its alias-analysis graph size."""

    rid: int
    arrival_s: float
    n: int
    seed: int

    def graph(self) -> Graph:
        return fica_like(n=self.n, n_a=2 * self.n, n_d=(3 * self.n) // 4, seed=self.seed)


def serving_stream(n_req: int = 1000, rate: float = 50.0, seed: int = 5,
                   n_lo: int = 5000, n_hi: int = 300_000) -> list:
    """Poisson arrivals (mean ``rate`` per second) of alias-analysis solves whose
    vertex counts are log-uniform in [n_lo, n_hi]."""
    rng = _rng(seed)
    t = 0.0
    out = []
    for r in range(n_req):
        u = (int(rng.integers(1, 1 << 53)) / float(1 << 53))
        t += -math.log(u) / rate
        n = log_uniform_int(rng, n_lo, n_hi)
        out.append(Request(rid=r, arrival_s=t, n=n, seed=seed * 1_000_003 + r))
    return out


def random_graph(n: int, n_edges: int, labels: list, seed: int, self_loops: bool = True) -> Graph:
    """Small uniform random multi-label graph (distinct triples) for tests."""
    rng = _rng(seed)
    L = len(labels)
    cap = n * n * L if self_loops else n * (n - 1) * L
    n_edges = min(n_edges, cap)

    def fn(size):
        s = rng.integers(0, n, size=size, dtype=np.int64)
        d = rng.integers(0, n, size=size, dtype=np.int64)
        if not self_loops:
            d = np.where(d == s, (d + 1) % n, d)
        return s, d
    chunks, have = [], 0
    while have < n_edges:
        s, d = fn(max(64, 2 * n_edges))
        lab = rng.integers(0, L, size=s.shape[0], dtype=np.int64)
        chunks.append((s * L + lab) * n + d)
        have = np.unique(np.concatenate(chunks)).shape[0]
    return _keys_to_graph(n, labels, _take_distinct(chunks, n_edges),
                          {"workload": "random", "seed": seed})


def path_graph(word: list, labels: list | None = None) -> Graph:
    """A path 0 -> 1 -> ... -> len(word) whose edge labels spell ``word``."""
    labels = labels or sorted(set(word))
    n = len(word) + 1
    src = np.arange(len(word), dtype=np.uint32)
    dst = src + 1
    lab = np.asarray([labels.index(x) for x in word], dtype=np.uint32)
    return Graph(n=n, labels=list(labels), src=src, lab=lab, dst=dst.astype(np.uint32),
                 meta={"workload": "path"})


def layered_graph(n: int, n_edges: int, seed: int, heights: int = 8,
                  pairs=(("a", "b"),)) -> Graph:
    """Height-layered graph: every open label goes from height h to h+1 and the
    matching close label from h+1 to h.  Any balanced path therefore joins two
    vertices of equal height."""
    rng = _rng(seed)
    h = rng.integers(0, heights, size=n, dtype=np.int64)
    labels = [x for p in pairs for x in p]
    L = len(labels)
    by_h = [np.flatnonzero(h == k) for k in range(heights)]
    src, lab, dst = [], [], []
    while len(src) < n_edges:
        u = int(rng.integers(0, n))
        p = int(rng.integers(0, len(pairs)))
        up = bool(rng.integers(0, 2))
        th = h[u] + 1 if up else h[u] - 1
        if th < 0 or th >= heights or by_h[th].size == 0:
            continue
        v = int(by_h[th][int(rng.integers(0, by_h[th].size))])
        src.append(u)
        dst.append(v)
        lab.append(labels.index(pairs[p][0] if up else pairs[p][1]))
    keys = (np.asarray(src) * L + np.asarray(lab)) * n + np.asarray(dst)
    keys = np.unique(keys)
    g = _keys_to_graph(n, labels, keys, {"workload": "layered", "seed": seed})
    g.meta["height"] = h
    return g
