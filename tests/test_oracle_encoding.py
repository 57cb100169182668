"""Pins of the oracle's encoding, R = P A and exact check (Sec. III-A).

Independent references: direct clause evaluation on the DIMACS text, a dense
integer matrix product of an independently built 0/1 problem matrix, brute
force over every assignment of tiny formulas, and the Fig. 2 fragments stated
in the text of Sec. III-A."""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from paper_2511_07737_b300 import cnfgen

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def all_assignments(n):
    """V x 2^n matrix whose columns are every assignment."""
    cols = np.arange(1 << n, dtype=np.int64)
    return ((cols[None, :] >> np.arange(n)[:, None]) & 1).astype(np.uint8)


def dense_P(n_vars, cptr, lits):
    """0/1 problem matrix C x 2V (column 2v = x_v, 2v+1 = x_v')."""
    C = len(cptr) - 1
    P = np.zeros((C, 2 * n_vars), np.int64)
    for c in range(C):
        for L in lits[cptr[c]:cptr[c + 1]]:
            v = abs(int(L)) - 1
            P[c, 2 * v + (1 if L < 0 else 0)] = 1
    return P


def dense_A(X):
    V, N = X.shape
    A = np.zeros((2 * V, N), np.int64)
    A[0::2] = X
    A[1::2] = 1 - X
    return A


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_tiny(seed):
    n = 6 + seed % 5
    inst = cnfgen.tiny_random(n, 3 * n, seed, kmin=1, kmax=4)
    cnf = oracle.CNF(n, inst.clause_ptr, inst.lits)
    X = all_assignments(n)
    unsat, satmask = oracle.check(cnf, X)
    # direct clause evaluation from the DIMACS literals
    ref = np.zeros(X.shape[1], np.int64)
    for c in range(inst.n_clauses):
        sat = np.zeros(X.shape[1], bool)
        for L in inst.lits[inst.clause_ptr[c]:inst.clause_ptr[c + 1]]:
            x = X[abs(int(L)) - 1].astype(bool)
            sat |= ~x if L < 0 else x
        ref += ~sat
    np.testing.assert_array_equal(unsat, ref)
    # Eq. 1 against a dense integer matmul of an independently built P and A
    R = oracle.result_matrix(cnf, X)
    np.testing.assert_array_equal(R, dense_P(n, inst.clause_ptr, inst.lits) @ dense_A(X))
    # an assignment is satisfying iff the column minimum of R is nonzero
    np.testing.assert_array_equal(unsat == 0, R.min(axis=0) > 0)
    np.testing.assert_array_equal(unsat, (R == 0).sum(axis=0))
    bits = np.unpackbits(satmask.view(np.uint8), bitorder="little")[: X.shape[1]]
    np.testing.assert_array_equal(bits.astype(bool), unsat == 0)
    # the STE objective reports the same unsatisfied counts at binary points
    _, _, _, u2 = oracle.objective(cnf, X=X, tau=1.0, grad=False)
    np.testing.assert_array_equal(u2, unsat)


def test_planted_model_satisfies():
    inst = cnfgen.planted_ksat(200, 852, 3, 7)
    cnf = oracle.CNF(inst.n_vars, inst.clause_ptr, inst.lits)
    unsat, _ = oracle.check(cnf, inst.planted[:, None])
    assert unsat[0] == 0


def test_duplicates_and_tautology():
    # clause 1: x1 x1 x2 (duplicate), clause 2: x1 x1' (tautology)
    ptr = np.array([0, 3, 5])
    lits = np.array([1, 1, 2, 1, -1])
    cnf = oracle.CNF(2, ptr, lits)
    assert cnf.nnz == 4
    X = all_assignments(2)
    R = oracle.result_matrix(cnf, X)
    np.testing.assert_array_equal(R[1], np.ones(4))          # tautology always 1
    np.testing.assert_array_equal(R[0], X[0] + X[1])         # duplicate counted once


@pytest.mark.parametrize("ptr,lits", [
    ([0, 2, 2], [1, 2]),          # empty clause
    ([0, 2], [1, 3]),             # variable out of range
    ([0, 2], [1, 0]),             # zero literal
])
def test_parse_errors(ptr, lits):
    with pytest.raises(ValueError):
        oracle.CNF(2, np.array(ptr), np.array(lits))


def test_fig2_fragments():
    g = json.load(open(os.path.join(GOLD, "fig2_fragments.json")))
    V = g["n_vars"]
    clauses = {1: [1, 2], 5: [2, -4]}          # unpinned: arbitrary
    for k, d in g["pinned_clauses"].items():
        clauses[int(k)] = d["lits"]
    lits = []
    ptr = [0]
    for c in range(1, g["n_clauses"] + 1):
        lits += clauses[c]
        ptr.append(len(lits))
    X = np.zeros((V, 3), np.uint8)
    fill = {1: {"x3": 0}, 3: {"x2": 1, "x4": 1}}   # unpinned: arbitrary
    for a in (1, 2, 3):
        vals = dict(fill.get(a, {}))
        vals.update({k: v for k, v in g["pinned_assignments"][str(a)].items() if k.startswith("x")})
        for name, val in vals.items():
            X[int(name[1:]) - 1, a - 1] = val
    R = oracle.result_matrix(oracle.CNF(V, np.array(ptr), np.array(lits)), X)
    for e in g["pinned_R"]:
        assert R[e["clause"] - 1, e["assignment"] - 1] == e["R"], e["cite"]


def test_brute_force_satisfying_set_matches_planted_family():
    # exhaustive: the set of satisfying assignments of a planted formula
    # contains the planted model and equals {x : min_c R_c(x) > 0}
    inst = cnfgen.planted_ksat(12, 40, 3, 3)
    cnf = oracle.CNF(12, inst.clause_ptr, inst.lits)
    X = all_assignments(12)
    unsat, _ = oracle.check(cnf, X)
    idx = int(sum(int(b) << j for j, b in enumerate(inst.planted)))
    assert unsat[idx] == 0
    R = oracle.result_matrix(cnf, X)
    assert set(np.nonzero(unsat == 0)[0]) == set(np.nonzero(R.min(axis=0) > 0)[0])
