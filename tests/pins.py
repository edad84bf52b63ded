"""Independent references that pin the oracle (used by the CPU tests only).

Nothing here imports the oracle or the CUDA library.  Each function restates
a definition from the paper or from textbook mathematics in the plainest form
that small inputs allow:

* ``naive_alg1``   - Algorithm 1 as printed (Sec. 2): |N| dense boolean
  matrices, terminal initialisation, then ``M <- M u (M . M)`` over the
  reachability semiring until M stops changing.
* ``brute_force``  - the definition of the result (Algorithm 1, "Result"):
  enumerate every path up to a length bound and parse its label word with a
  CYK table that allows epsilon and unit productions.
* ``bfs_reach``    - breadth-first search, the textbook routine that the
  grammar ``S -> S S | a`` (transitive closure of a-edges) reduces to.
* ``dyck_balanced`` - the counter test for balanced bracket words.

Grammars are read by ``read_grammar`` below, written separately from the
oracle's reader so that a reader mistake cannot hide on both sides.
"""
from __future__ import annotations

import itertools
import re
from collections import defaultdict, deque

import numpy as np


def read_grammar(text: str):
    """Return (nonterminals, productions) with productions as tuples
    (lhs, rhs_tuple); rhs_tuple is () for epsilon."""
    ranges = {}
    lines = []
    for line in text.splitlines():
        line = line.split("#")[0].strip()
        if not line:
            continue
        if line.startswith("%index"):
            _, var, lo, hi = line.split()
            ranges[var] = range(int(lo), int(hi) + 1)
            continue
        lhs, rhs = line.split("->")
        for alt in rhs.split("|"):
            lines.append((lhs.strip(), alt.split()))
    prods = []
    for lhs, rhs in lines:
        toks = [lhs] + rhs
        used = sorted(set(v for t in toks for v in re.findall(r"_\{(\w+)\}", t)))
        for vals in itertools.product(*(ranges[v] for v in used)):
            def sub(t):
                for v, x in zip(used, vals):
                    t = t.replace("_{%s}" % v, "_%d" % x)
                return t
            l2 = sub(lhs)
            r2 = tuple(sub(t) for t in rhs)
            prods.append((l2, () if r2 == ("eps",) else r2))
    nts = []
    for l, _ in prods:
        if l not in nts:
            nts.append(l)
    return nts, sorted(set(prods))


def naive_alg1(text: str, graph) -> dict:
    """Algorithm 1 with dense boolean matrices; returns {NT: bool (n, n) array}."""
    nts, prods = read_grammar(text)
    n = graph.n
    M = {x: np.zeros((n, n), dtype=bool) for x in nts}
    T = {}
    for li, name in enumerate(graph.labels):
        t = np.zeros((n, n), dtype=bool)
        sel = graph.lab == li
        t[graph.src[sel].astype(int), graph.dst[sel].astype(int)] = True
        T[name] = t

    def mat(sym):
        if sym in M:
            return M[sym]
        return T.get(sym, np.zeros((n, n), dtype=bool))

    # terminal initialisation: M_ij u= {A | A -> x}; A -> eps gives the identity
    for lhs, rhs in prods:
        if len(rhs) == 1 and rhs[0] not in M:
            M[lhs] |= mat(rhs[0])
        elif len(rhs) == 0:
            M[lhs] |= np.eye(n, dtype=bool)
    changed = True
    while changed:                       # "while M is changing"
        changed = False
        for lhs, rhs in prods:           # M <- M u (M . M)
            if len(rhs) == 2:
                prod = (mat(rhs[0]).astype(np.int64) @ mat(rhs[1]).astype(np.int64)) > 0
            elif len(rhs) == 1 and rhs[0] in M:
                prod = M[rhs[0]]
            else:
                continue
            new = M[lhs] | prod
            if (new != M[lhs]).any():
                M[lhs] = new
                changed = True
    return M


class CYK:
    """Which non-terminals derive a word (epsilon and unit productions allowed)."""

    def __init__(self, text: str):
        self.nts, self.prods = read_grammar(text)
        self.cache = {}

    def _close(self, cell: set, empty: set, first_split=None):
        # add lhs of unit productions and of binary productions whose other
        # side is the empty word, until nothing changes
        changed = True
        while changed:
            changed = False
            for lhs, rhs in self.prods:
                if lhs in cell:
                    continue
                if len(rhs) == 1 and rhs[0] in cell:
                    cell.add(lhs); changed = True
                elif len(rhs) == 2 and ((rhs[0] in empty and rhs[1] in cell) or
                                        (rhs[0] in cell and rhs[1] in empty)):
                    cell.add(lhs); changed = True
        return cell

    def derives(self, word: tuple) -> set:
        if word in self.cache:
            return self.cache[word]
        L = len(word)
        empty = self._close(set(lhs for lhs, rhs in self.prods if rhs == ()), set())
        # with the empty set as "empty", _close above only used unit/eps forms;
        # binary productions with both sides nullable:
        changed = True
        while changed:
            changed = False
            for lhs, rhs in self.prods:
                if lhs not in empty and len(rhs) == 2 and rhs[0] in empty and rhs[1] in empty:
                    empty.add(lhs); changed = True
                elif lhs not in empty and len(rhs) == 1 and rhs[0] in empty:
                    empty.add(lhs); changed = True
        if L == 0:
            self.cache[word] = set(x for x in empty if x in self.nts)
            return self.cache[word]
        D = {}
        for length in range(1, L + 1):
            for i in range(0, L - length + 1):
                j = i + length
                cell = set()
                if length == 1:
                    cell.add(word[i])
                    for lhs, rhs in self.prods:
                        if rhs == (word[i],):
                            cell.add(lhs)
                for k in range(i + 1, j):
                    left, right = D[(i, k)], D[(k, j)]
                    for lhs, rhs in self.prods:
                        if len(rhs) == 2 and rhs[0] in left and rhs[1] in right:
                            cell.add(lhs)
                D[(i, j)] = self._close(cell, empty)
        out = set(x for x in D[(0, L)] if x in self.nts)
        self.cache[word] = out
        return out


def brute_force(text: str, graph, max_len: int) -> dict:
    """{NT: set of (i, j)} over every path of length <= max_len (length 0
    included, for epsilon), each label word parsed by CYK."""
    cyk = CYK(text)
    out = defaultdict(set)
    adj = defaultdict(list)
    for s, l, d in zip(graph.src.tolist(), graph.lab.tolist(), graph.dst.tolist()):
        adj[s].append((graph.labels[l], d))
    words = defaultdict(set)                # word -> set of (i, j)
    for start in range(graph.n):
        stack = [(start, ())]
        while stack:
            v, w = stack.pop()
            words[w].add((start, v))
            if len(w) < max_len:
                for lab, d in adj[v]:
                    stack.append((d, w + (lab,)))
    for w, ends in words.items():
        for X in cyk.derives(w):
            out[X] |= ends
    return out


def bfs_reach(graph, label: str) -> set:
    """Pairs (i, j) joined by a path of one or more ``label`` edges (BFS)."""
    li = graph.labels.index(label)
    adj = defaultdict(list)
    for s, l, d in zip(graph.src.tolist(), graph.lab.tolist(), graph.dst.tolist()):
        if l == li:
            adj[s].append(d)
    out = set()
    for s in range(graph.n):
        seen = set()
        q = deque(adj[s])
        while q:
            v = q.popleft()
            if v in seen:
                continue
            seen.add(v)
            q.extend(adj[v])
        out |= {(s, v) for v in seen}
    return out


def dyck_balanced(word, pairs) -> bool:
    """True iff ``word`` is a non-empty well-nested bracket word; ``pairs``
    maps each opening symbol to its closing symbol."""
    if not word:
        return False
    closing = {c: o for o, c in pairs.items()}
    stack = []
    for x in word:
        if x in pairs:
            stack.append(x)
        elif x in closing:
            if not stack or stack[-1] != closing[x]:
                return False
            stack.pop()
        else:
            return False
    return not stack
