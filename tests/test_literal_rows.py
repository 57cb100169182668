"""The 2V literal-row transform (paper_2511_07737_b300.literal_rows) against
its definition, on the CPU: with independent 0/1 literal rows X2 (row v for
x_v, row V + v for not x_v) the clause sums of the transformed formula are
R_c = the number of the clause's literals whose own row is 1 (duplicate
literals counted once, as the library removes them); the consistent lift of
a model satisfies the transformed formula and decodes to that model; and
every all-true row assignment satisfies it too (the degenerate model)."""
import numpy as np

import oracle
from paper_2511_07737_b300 import cnfgen
from paper_2511_07737_b300.literal_rows import split_literals


def test_transform_clause_sums_match_the_definition():
    for seed in range(5):
        inst = cnfgen.tiny_random(12, 40, seed, kmin=1, kmax=4)
        t = split_literals(inst)
        assert t.n_vars == 24 and (t.lits > 0).all() and t.n_clauses == inst.n_clauses
        X2 = np.random.default_rng(seed).integers(0, 2, (24, 32), dtype=np.uint8)
        R = oracle.result_matrix(oracle.CNF(t.n_vars, t.clause_ptr, t.lits), X2)
        ref = np.zeros_like(R)
        for c in range(inst.n_clauses):
            for lit in set(inst.lits[inst.clause_ptr[c]:inst.clause_ptr[c + 1]].tolist()):
                ref[c] += X2[lit - 1] if lit > 0 else X2[inst.n_vars - lit - 1]
        np.testing.assert_array_equal(R, ref)


def test_lift_and_all_true_satisfy_the_transformed_formula():
    inst = cnfgen.planted_ksat(60, 256, 3, 4)
    t = split_literals(inst)
    cnf2 = oracle.CNF(t.n_vars, t.clause_ptr, t.lits)
    X = np.stack([t.planted, np.ones(t.n_vars, np.uint8), np.zeros(t.n_vars, np.uint8)], axis=1)
    u, _ = oracle.check(cnf2, X)
    assert u[0] == 0 and u[1] == 0 and u[2] == inst.n_clauses
    assert (t.planted[:60] == inst.planted).all() and (t.planted[60:] == 1 - inst.planted).all()
    u0, _ = oracle.check(oracle.CNF(inst.n_vars, inst.clause_ptr, inst.lits), t.planted[:60, None])
    assert u0[0] == 0
