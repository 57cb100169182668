"""2V independent literal rows: the paper's real-valued assignment matrix with
one row per literal (Sec. III-A: 2V rows), read without the tie between a
variable's two literals.

It is built as an exact transform of the CNF, so every kernel of the library
runs it unchanged.  Literal x_v becomes the positive literal of variable v+
(row v) and literal not x_v the positive literal of a separate variable v-
(row V + v).  Each literal row then has its own parameters, Eq. 5 normaliser,
bits and straight-through gradient, and R_ci counts the true literal rows of
clause c.  The library's own "found" test then judges the transformed formula,
which every all-true assignment of the literal rows satisfies; an assignment of
the original formula is decoded as x_v = bit of row v+ and judged separately.
The default model of the library keeps one row per variable, with x' = not x
(the O3 reading); this module exists to measure the alternative.
"""
from __future__ import annotations

import numpy as np
import torch

from paper_2511_07737_b300 import cnfgen
from paper_2511_07737_b300 import turbosat as ts


def split_literals(inst: cnfgen.Instance) -> cnfgen.Instance:
    """The transformed instance over 2V variables: literal +v -> +v and
    -v -> +(V + v), all literals positive.  Its planted assignment is the
    consistent lift of the original one (row v+ = x_v, row v- = not x_v)."""
    V = inst.n_vars
    lits = np.asarray(inst.lits, np.int64)
    out = np.where(lits > 0, lits, V - lits).astype(np.int32)
    planted = np.concatenate([inst.planted, 1 - inst.planted]).astype(np.uint8)
    meta = dict(inst.meta)
    meta["literal_rows"] = True
    return cnfgen.Instance(2 * V, np.asarray(inst.clause_ptr, np.int64).copy(), out, planted, meta)


def decoded_bits(st: ts.State, n_vars: int) -> torch.Tensor:
    """The current bits of rows v+ (v < n_vars) of a state of the transformed
    instance: the decoded assignments of the original formula, [V][N/32]."""
    return st.view("bits")[:n_vars].contiguous()


def decoded_unsat(orig: ts.Problem, st: ts.State, tau: float = 1.0) -> np.ndarray:
    """Unsatisfied clauses of the original formula under the decoded
    assignment of every sample (the library's exact check, no allocation)."""
    V = orig.info["n_vars"]
    bits = decoded_bits(st, V)
    unsat = torch.zeros(st.N, dtype=torch.int32, device=bits.device)
    sm = torch.zeros(st.N // 32, dtype=torch.int32, device=bits.device)
    ts.tsat_evaluate_bits_noalloc(orig.h, bits, st.N, tau, unsat, sm)
    torch.cuda.synchronize()
    return unsat.cpu().numpy()


def inconsistent_fraction(st: ts.State, n_vars: int) -> float:
    """Fraction of (variable, sample) pairs whose two literal rows agree
    (both true or both false), i.e. not a complete assignment."""
    b = st.view("bits").cpu().numpy().view(np.uint32)
    pos, neg = b[:n_vars], b[n_vars:2 * n_vars]
    same = np.unpackbits((~(pos ^ neg)).view(np.uint8), bitorder="little")
    return float(same.mean())
