"""CFL-reachability oracle (TEST INFRASTRUCTURE ONLY).

A plain, slow, obviously correct CPU implementation of what the CUDA library
computes: for every non-terminal X of a WCNF grammar, the set of vertex pairs
(i, j) joined by a path whose label word X derives (the paper's problem
statement, Algorithm 1 "Result").  The core is the single-threaded worklist in
``worklist.c``; the grammar reader is ``grammar.py``.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path;
both sides read the same inputs from the seeded generators only.

Parity status: pinned.  The tests check this oracle against Algorithm 1 run
as written (dense boolean fixpoint), against brute-force path enumeration with
CYK parsing, against breadth-first search for the transitive-closure grammar,
against the balanced-word closed form of Dyck languages on path graphs, and
against the paper's grammar equivalences and structural invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import time

import numpy as np

from .grammar import OracleGrammar, parse, GrammarError  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "worklist.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``worklist.c`` into ``liboracle.so`` (gcc, portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        lib.oracle_solve.restype = ctypes.c_void_p
        lib.oracle_solve.argtypes = [ctypes.c_uint32, ctypes.c_uint32,
                                     ctypes.c_uint32, u32p, ctypes.c_uint32, u32p,
                                     ctypes.c_uint32, u32p, ctypes.c_uint64, u32p]
        lib.oracle_count.restype = ctypes.c_uint64
        lib.oracle_count.argtypes = [ctypes.c_void_p, ctypes.c_uint32]
        lib.oracle_keys.restype = ctypes.c_uint64
        lib.oracle_keys.argtypes = [ctypes.c_void_p, ctypes.c_uint32,
                                    ctypes.POINTER(ctypes.c_uint64)]
        lib.oracle_pops.restype = ctypes.c_uint64
        lib.oracle_pops.argtypes = [ctypes.c_void_p]
        lib.oracle_joins.restype = ctypes.c_uint64
        lib.oracle_joins.argtypes = [ctypes.c_void_p]
        lib.oracle_free.restype = None
        lib.oracle_free.argtypes = [ctypes.c_void_p]
        _lib = lib
    return _lib


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint32).reshape(-1))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def terminal_init(g: OracleGrammar, graph) -> np.ndarray:
    """Algorithm 1, terminal initialisation: the triples (u, A, v) for every
    edge (u, x, v) and every production A -> x, as an (m, 3) uint32 array.
    Edges whose label has no production contribute nothing."""
    rows = []
    for li, name in enumerate(graph.labels):
        for A in g.term.get(name, []):
            sel = graph.lab == li
            m = int(sel.sum())
            if m:
                rows.append(np.stack([graph.src[sel], np.full(m, A, np.uint32),
                                      graph.dst[sel]], axis=1))
    if not rows:
        return np.zeros((0, 3), np.uint32)
    return np.concatenate(rows).astype(np.uint32)


class OracleResult:
    """Per-non-terminal pair sets, each a sorted uint64 array of src<<32|dst."""

    def __init__(self, grammar: OracleGrammar, pairs: dict, seconds: float, pops: int,
                 joins: int):
        self.grammar = grammar
        self.pairs = pairs
        self.seconds = seconds
        self.pops = pops
        self.joins = joins

    def total(self, include_wrappers: bool = False) -> int:
        names = self.grammar.nts if include_wrappers else self.grammar.nts[:self.grammar.n_user]
        return int(sum(self.pairs[x].shape[0] for x in names))

    def dense(self, name: str, n: int) -> np.ndarray:
        m = np.zeros((n, n), dtype=bool)
        k = self.pairs[name]
        m[(k >> np.uint64(32)).astype(np.int64), (k & np.uint64(0xFFFFFFFF)).astype(np.int64)] = True
        return m


def solve(grammar_text_or_parsed, graph) -> OracleResult:
    """Solve CFL-reachability for ``graph`` (a ``gen.Graph``) under the grammar.

    Returns every non-terminal's pairs, terminal wrappers included (their
    names are ``<x>``).  ``seconds`` covers the worklist solve only, the same
    scope the paper times (Sec. 4: graph construction excluded).
    """
    g = grammar_text_or_parsed
    if isinstance(g, str):
        g = parse(g)
    lib = _load()
    init = _u32(terminal_init(g, graph))
    binary = _u32(g.binary if g.binary else np.zeros(0))
    unit = _u32(g.unit if g.unit else np.zeros(0))
    eps = _u32(g.eps if g.eps else np.zeros(0))
    n_nt = len(g.nts)
    t0 = time.perf_counter()
    st = lib.oracle_solve(int(graph.n), n_nt, len(g.binary), _ptr(binary), len(g.unit),
                          _ptr(unit), len(g.eps), _ptr(eps), init.shape[0] // 3, _ptr(init))
    dt = time.perf_counter() - t0
    if not st:
        raise MemoryError("oracle ran out of host memory")
    try:
        pairs = {}
        for X, name in enumerate(g.nts):
            cnt = lib.oracle_count(st, X)
            buf = np.empty(cnt, dtype=np.uint64)
            lib.oracle_keys(st, X, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
            buf.sort()
            pairs[name] = buf
        pops, joins = lib.oracle_pops(st), lib.oracle_joins(st)
    finally:
        lib.oracle_free(st)
    return OracleResult(g, pairs, dt, pops, joins)
