"""Grammar-text reader of the oracle (test infrastructure only).

Reads the WCNF grammar format shared by the library and the oracle, with its
own code (the CUDA library has an independent C++ reader):

* one production per line, ``LHS -> X Y``, ``LHS -> x`` or ``LHS -> eps``,
  ``|`` separating alternatives and ``#`` starting a comment;
* a symbol is a non-terminal iff it is the left-hand side of some production,
  every other symbol is a terminal (an edge label);
* ``%index v lo hi`` makes every production that mentions ``_{v}`` stand for
  one copy per value of v in lo..hi (the "indexed" non-terminals of the
  field-sensitive grammars, paper appendix B).

Productions are those of weak Chomsky normal form (Sec. 2, WCNF definition),
plus two forms that the paper's figures use but the definition leaves out,
read as follows:

* a terminal x inside a binary production (e.g. ``N1 -> N1 a_r`` of Fig.
  "wcnf:fica") is replaced by a fresh non-terminal ``<x>`` with the single
  production ``<x> -> x``; this derives exactly the same words;
* a unit production ``C -> A`` (Fig. "wcnf:fsca") means R_C includes R_A.
"""
from __future__ import annotations

import itertools
import re
from dataclasses import dataclass, field


class GrammarError(ValueError):
    pass


@dataclass
class OracleGrammar:
    nts: list                      # non-terminal names; wrappers "<x>" come last
    n_user: int                    # number of non-terminals named in the text
    binary: list                   # (c, a, b) ids, c -> a b
    unit: list                     # (c, a) ids, c -> a
    eps: list                      # ids A with A -> eps
    term: dict = field(default_factory=dict)   # terminal name -> [A ids with A -> x]

    def nt_id(self, name: str) -> int:
        return self.nts.index(name)


_IDX = re.compile(r"_\{([A-Za-z][A-Za-z0-9]*)\}")


def _expand(tokens: list, ranges: dict) -> list:
    """All copies of a token list, one per assignment of its index variables."""
    names = sorted({m for t in tokens for m in _IDX.findall(t)})
    for v in names:
        if v not in ranges:
            raise GrammarError(f"index variable {v!r} has no %index line")
    if not names:
        return [tokens]
    out = []
    for vals in itertools.product(*(range(ranges[v][0], ranges[v][1] + 1) for v in names)):
        sub = dict(zip(names, vals))
        out.append([_IDX.sub(lambda m: "_" + str(sub[m.group(1)]), t) for t in tokens])
    return out


def parse(text: str) -> OracleGrammar:
    ranges = {}
    raw = []                          # (lhs, [rhs symbols])
    for ln, line in enumerate(text.splitlines(), 1):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        if line.startswith("%"):
            parts = line.split()
            if parts[0] != "%index" or len(parts) != 4:
                raise GrammarError(f"line {ln}: bad directive")
            lo, hi = int(parts[2]), int(parts[3])
            if hi < lo:
                raise GrammarError(f"line {ln}: empty index range")
            ranges[parts[1]] = (lo, hi)
            continue
        if "->" not in line:
            raise GrammarError(f"line {ln}: missing '->'")
        lhs, rhs = line.split("->", 1)
        lhs = lhs.split()
        if len(lhs) != 1:
            raise GrammarError(f"line {ln}: left-hand side must be one symbol")
        for alt in rhs.split("|"):
            syms = alt.split()
            if not syms:
                raise GrammarError(f"line {ln}: empty alternative (write eps)")
            raw.append((ln, [lhs[0]] + syms))

    prods = []
    for ln, toks in raw:
        for t in _expand(toks, ranges):
            prods.append((ln, t[0], t[1:]))

    nts = []
    seen = set()
    for _, lhs, _ in prods:
        if lhs == "eps":
            raise GrammarError("eps cannot be a left-hand side")
        if lhs not in seen:
            seen.add(lhs)
            nts.append(lhs)
    n_user = len(nts)
    ids = {x: i for i, x in enumerate(nts)}
    wrappers = {}

    def operand(sym):
        if sym in ids:
            return ids[sym]
        if sym not in wrappers:
            wrappers[sym] = len(nts)
            nts.append("<" + sym + ">")
        return wrappers[sym]

    binary, unit, eps, term = [], [], [], {}
    for ln, lhs, rhs in prods:
        c = ids[lhs]
        if rhs == ["eps"]:
            eps.append(c)
        elif len(rhs) == 1:
            if rhs[0] in ids:
                unit.append((c, ids[rhs[0]]))
            else:
                term.setdefault(rhs[0], []).append(c)
        elif len(rhs) == 2:
            if "eps" in rhs:
                raise GrammarError(f"line {ln}: eps inside a binary production")
            binary.append((c, operand(rhs[0]), operand(rhs[1])))
        else:
            raise GrammarError(f"line {ln}: more than two right-hand symbols (not WCNF)")
    for sym, w in wrappers.items():
        term.setdefault(sym, []).append(w)
    # set semantics: drop repeated productions
    binary = sorted(set(binary))
    unit = sorted(set(unit))
    eps = sorted(set(eps))
    term = {k: sorted(set(v)) for k, v in term.items()}
    return OracleGrammar(nts=nts, n_user=n_user, binary=binary, unit=unit, eps=eps, term=term)
