"""Hand-off of a partial assignment to a CDCL solver (Sec. IV-B).

The GPU phase ends with the best sample and the top-k most confident
variables of it (`tsat_best`: 1-based variables and their values).  The CDCL
phase of the paper fixes those variables and lets a CDCL solver complete the
rest; no CDCL solver ships here, so this module only produces its input:

* `partial_units`: the fixed variables as DIMACS unit literals (+v true, -v false);
* `to_dimacs`: a CNF in DIMACS text, optionally with the unit clauses appended
  (the form every DIMACS-reading CDCL solver accepts; an incremental solver can
  take the same literals as assumptions instead);
* `parse_dimacs`: the inverse, for checking.
"""
from __future__ import annotations

import numpy as np


def partial_units(part_var, part_val) -> np.ndarray:
    """DIMACS literals of the partial assignment (1-based variables)."""
    v = np.asarray(part_var, np.int64)
    x = np.asarray(part_val, np.uint8)
    if v.shape != x.shape:
        raise ValueError("part_var and part_val differ in length")
    if v.size and v.min() < 1:
        raise ValueError("variables are 1-based")
    return np.where(x != 0, v, -v).astype(np.int32)


def to_dimacs(n_vars: int, clause_ptr, lits, units=None) -> str:
    """DIMACS CNF text of the clauses (clause_ptr [C+1] offsets into DIMACS-signed
    lits), followed by one unit clause per literal of `units`."""
    cp = np.asarray(clause_ptr, np.int64)
    li = np.asarray(lits, np.int64)
    u = np.zeros(0, np.int64) if units is None else np.asarray(units, np.int64)
    if u.size and np.abs(u).max() > n_vars:
        raise ValueError("unit literal out of range")
    out = [f"p cnf {n_vars} {cp.shape[0] - 1 + u.size}"]
    for c in range(cp.shape[0] - 1):
        out.append(" ".join(str(int(x)) for x in li[cp[c]:cp[c + 1]]) + " 0")
    out.extend(f"{int(x)} 0" for x in u)
    return "\n".join(out) + "\n"


def parse_dimacs(text: str):
    """(n_vars, clause_ptr int64 [C+1], lits int32) from DIMACS CNF text."""
    n_vars, clauses, cur = 0, [], []
    for line in text.splitlines():
        line = line.strip()
        if not line or line[0] in "c%":
            continue
        if line[0] == "p":
            parts = line.split()
            n_vars = int(parts[2])
            continue
        for tok in line.split():
            x = int(tok)
            if x == 0:
                clauses.append(cur)
                cur = []
            else:
                cur.append(x)
    if cur:
        clauses.append(cur)
    cp = np.zeros(len(clauses) + 1, np.int64)
    cp[1:] = np.cumsum([len(c) for c in clauses])
    lits = np.array([x for c in clauses for x in c], np.int32)
    return n_vars, cp, lits
