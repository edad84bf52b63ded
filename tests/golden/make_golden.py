"""Write the oracle's fingerprints of the full-size workloads (tests/golden).

Run from the repository root:  python tests/golden/make_golden.py [name ...]

Every stored value comes from the CPU oracle (package ``oracle``) on inputs
from the seeded generators; nothing here runs the CUDA library.  For each
workload the file records the generator call, a digest of its edge list (so
a test can tell whether the generator still produces the same graph on its
machine) and, per non-terminal named in the grammar, the pair count and an
order-independent fingerprint of the pair set.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
from common import fingerprint  # noqa: E402
from paper_2401_11029_gb300 import gen  # noqa: E402

WORKLOADS = {
    "dyck1_er_1000": ("dyck1", lambda: gen.dyck1_er()),
    "fica_like_200k": ("fica", lambda: gen.fica_like()),
    "fsjpt_like_500k": ("fsjpt", lambda: gen.fsjpt_like()),
    # the imagick-shaped field-sensitive alias graph (142 fields)
    "fsca_like_41k": (("fsca", 141), lambda: gen.fsca_like()),
    # context-sensitive value flow, 100k vertices (povray's edge ratio), 512
    # call sites
    "cscvf_like_100k": (("cscvf", 511),
                        lambda: gen.cscvf_like(n=100_000, n_edges=168_000, calls=512)),
}


def one(name, grammar, make):
    g = make()
    # a grammar name, or (name, last index) for the indexed grammars
    text = gen.grammar_text(*grammar) if isinstance(grammar, tuple) else gen.grammar_text(grammar)
    t0 = time.time()
    res = oracle.solve(text, g)
    pg = res.grammar
    out = {"workload": name, "grammar": list(grammar) if isinstance(grammar, tuple) else grammar,
           "n": g.n, "edges": g.n_edges,
           "edge_digest": g.edge_digest(), "meta": {k: v for k, v in g.meta.items()
                                                    if isinstance(v, (int, float, str))},
           "oracle_seconds": round(res.seconds, 2), "total_pairs": res.total(),
           "pairs": {x: fingerprint(res.pairs[x]) for x in pg.nts[:pg.n_user]}}
    path = os.path.join(HERE, name + ".json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
    print(f"{name}: {res.total()} pairs, oracle {res.seconds:.1f} s "
          f"({time.time() - t0:.1f} s with extraction) -> {path}", flush=True)


def dyck3_batch_golden():
    """Per-instance fingerprints of the 256 batched Dyck-3 instances."""
    text = gen.grammar_text("dyck3")
    inst = []
    t0 = time.time()
    for k in range(256):
        g = gen.dyck3_instance(4000 + k)
        res = oracle.solve(text, g)
        pg = res.grammar
        inst.append({"seed": 4000 + k, "n": g.n, "edges": g.n_edges,
                     "edge_digest": g.edge_digest(), "total_pairs": res.total(),
                     "pairs": {x: fingerprint(res.pairs[x]) for x in pg.nts[:pg.n_user]}})
    out = {"workload": "dyck3_batch_256", "grammar": "dyck3", "instances": inst,
           "oracle_seconds": round(time.time() - t0, 2)}
    path = os.path.join(HERE, "dyck3_batch_256.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
    print(f"dyck3_batch_256: {sum(i['total_pairs'] for i in inst)} pairs -> {path}", flush=True)


if __name__ == "__main__":
    names = sys.argv[1:] or list(WORKLOADS) + ["dyck3_batch_256"]
    for nm in names:
        if nm == "dyck3_batch_256":
            dyck3_batch_golden()
        else:
            grammar, make = WORKLOADS[nm]
            one(nm, grammar, make)
