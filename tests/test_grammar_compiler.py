"""The library's grammar compiler (host C++, hot-path step a1) against the
oracle's independent reader: for every grammar the tests use, the same
non-terminals and wrappers, binary, unit and epsilon productions and terminal
tables, compared by name.  Runs on the CPU: a small helper program links the
library's grammar.cpp and prints its tables."""
import json
import os
import shutil
import subprocess

import pytest

import oracle
from common import GRAMMARS, RANDOM_GRAMMARS
from paper_2401_11029_gb300 import gen

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2401_11029_gb300", "csrc")


@pytest.fixture(scope="module")
def compile_grammar(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("grammar_dump") / "grammar_dump")
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", CSRC, os.path.join(HERE, "grammar_dump.cpp"),
                    os.path.join(CSRC, "grammar.cpp"), "-o", exe], check=True)

    def run(text: str) -> dict:
        out = subprocess.run([exe], input=text.encode(), capture_output=True, check=True)
        return json.loads(out.stdout)
    return run


CASES = {name: text for name, (text, _) in GRAMMARS.items()}
CASES.update({f"random{i}": t for i, t in enumerate(RANDOM_GRAMMARS)})
CASES["fsjpt64"] = gen.grammar_text("fsjpt")
CASES["fsca"] = gen.grammar_text("fsca")
CASES["cscvf"] = gen.grammar_text("cscvf")


@pytest.mark.parametrize("name", sorted(CASES))
def test_tables_match_the_oracle_reader(compile_grammar, name):
    text = CASES[name]
    lib = compile_grammar(text)
    og = oracle.parse(text)
    nm = og.nts
    assert lib["n_named"] == og.n_user
    assert set(lib["nts"][:og.n_user]) == set(nm[:og.n_user])     # named first
    assert set(lib["nts"]) == set(nm)                             # then the wrappers
    assert {tuple(p[:3]) for p in lib["binary"]} == {(nm[c], nm[a], nm[b]) for c, a, b in og.binary}
    assert {tuple(p) for p in lib["unit"]} == {(nm[c], nm[a]) for c, a in og.unit}
    assert set(lib["eps"]) == {nm[a] for a in og.eps}
    lib_term = {t: set(v) for t, v in lib["term"].items() if v}
    or_term = {t: {nm[a] for a in v} for t, v in og.term.items() if v}
    assert lib_term == or_term


def test_indexed_families_cover_every_member(compile_grammar):
    """With 64 fields every family of the field-sensitive grammar has the 64
    copies of one production, one per field (optimisation 4)."""
    lib = compile_grammar(CASES["fsjpt64"])
    members = {}
    for c, a, b, fam, member in lib["binary"]:
        if fam >= 0:
            members.setdefault(fam, []).append(member)
    assert members and all(lib["fam_size"][f] == 64 for f in members)
    assert all(sorted(m) == list(range(64)) for m in members.values())


@pytest.mark.parametrize("text", ["A -> \n", "-> a\n", "A -> B C D\n", "A B -> c\n",
                                  "%index i 3 1\nA_{i} -> a\n", "A -> B_{j} c\n"])
def test_malformed_grammars_are_rejected_by_both(compile_grammar, text):
    assert "error" in compile_grammar(text)
    with pytest.raises(oracle.GrammarError):
        oracle.parse(text)
