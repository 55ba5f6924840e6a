"""Readers for the fixtures under tests/golden/ (no method arithmetic)."""
import json
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _lit(tok: str) -> int:
    tok = tok.strip()
    neg = tok.startswith("-")
    v = int(tok.lstrip("+-"))
    return -(v + 1) if neg else (v + 1)


def paper_instances():
    with open(os.path.join(GOLDEN, "paper_instances.json")) as fh:
        doc = json.load(fh)
    out = []
    for inst in doc["instances"]:
        lits = np.array([[_lit(t) for t in cl] for cl in inst["clauses"]], dtype=np.int32)
        out.append(dict(name=inst["name"], n=inst["n"], lits=lits,
                        table1=inst["table1_noiseless_solution_percent"]))
    return out
