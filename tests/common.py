"""Shared test inputs and helpers (no oracle arithmetic, no CUDA calls)."""
import numpy as np

from paper_2401_11029_gb300 import gen

FSJPT2_LABELS = ["alloc", "assign", "alloc_r", "assign_r", "load_0", "load_1", "store_0",
                 "store_1", "load_r_0", "load_r_1", "store_r_0", "store_r_1"]

GRAMMARS = {
    "dyck1": (gen.grammar_text("dyck1"), ["a", "b"]),
    "dyck3": (gen.grammar_text("dyck3"), ["a_1", "b_1", "a_2", "b_2", "a_3", "b_3"]),
    "fica": (gen.grammar_text("fica"), ["a", "d", "a_r", "d_r"]),
    "fica_cfg": (gen.grammar_text("fica_cfg"), ["a", "d", "a_r", "d_r"]),
    "fsjpt2": (gen.grammar_text("fsjpt", index_hi=1), FSJPT2_LABELS),
    "fsjpt2_cfg": (gen.grammar_text("fsjpt_cfg", index_hi=1), FSJPT2_LABELS),
    # the grammars of Figs. wcnf:fsca and wcnf:cscvf (epsilon, unit
    # productions, indexed families), two indices each
    "fsca2": (gen.grammar_text("fsca", index_hi=1),
              ["d", "d_r", "a", "a_r", "f_0", "f_1", "f_r_0", "f_r_1"]),
    "cscvf2": (gen.grammar_text("cscvf", index_hi=1),
               ["a", "call_0", "call_1", "ret_0", "ret_1"]),
}

# WCNF grammars with epsilon, unit and terminal-in-binary productions.
RANDOM_GRAMMARS = [
    "S -> S S | a | A b\nA -> eps | a A\n",
    "X -> Y Z | b\nY -> X a | eps\nZ -> Y | c\n",
    "P -> Q P | a\nQ -> P b | c Q | eps\nR -> P | Q Q\n",
    "A -> B C | a\nB -> C A | b\nC -> A B | c | A\n",
]


def keys_of(src, dst) -> np.ndarray:
    return gen.pair_keys(src, dst)


# order-independent digest of a set of uint64 keys (count, xor and sum of a
# 64-bit mix of every key)
fingerprint = gen.pair_fingerprint
