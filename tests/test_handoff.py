"""CDCL hand-off export: DIMACS round trip, unit literals of a partial
assignment, and (on the GPU) that the units taken from a satisfying sample
keep the formula satisfied by that sample."""
import numpy as np
import pytest

from paper_2511_07737_b300 import cnfgen
from paper_2511_07737_b300.handoff import parse_dimacs, partial_units, to_dimacs


def test_dimacs_round_trip_with_units():
    inst = cnfgen.tiny_random(30, 90, 4, kmin=1, kmax=5)
    units = partial_units([3, 7, 30], [1, 0, 1])
    assert list(units) == [3, -7, 30]
    n, cp, li = parse_dimacs(to_dimacs(inst.n_vars, inst.clause_ptr, inst.lits, units))
    assert n == inst.n_vars
    C = inst.n_clauses
    assert cp.shape[0] == C + 3 + 1
    np.testing.assert_array_equal(cp[:C + 1], inst.clause_ptr)
    np.testing.assert_array_equal(li[:inst.nnz], inst.lits)
    np.testing.assert_array_equal(li[inst.nnz:], [3, -7, 30])


def test_units_reject_bad_input():
    with pytest.raises(ValueError):
        partial_units([0, 1], [1, 1])
    with pytest.raises(ValueError):
        to_dimacs(3, [0, 1], [1], units=[4])


@pytest.mark.gpu
def test_gpu_partial_of_a_model_keeps_it_a_model():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import oracle
    from paper_2511_07737_b300 import turbosat as ts
    inst = cnfgen.planted_ksat(100, 400, 3, 4)
    prob = ts.Problem([(inst.n_vars, inst.clause_ptr, inst.lits)])
    st = ts.State(prob, 64)
    hp = ts.hparams(seed=2, norm=ts.NORM_ABSMEAN, tau=2.0, lr0=0.5)
    ts.tsat_init(st.h, hp)
    ts.tsat_step(st.h, hp, 500, stop_on_sat=True)
    best = ts.tsat_best(st.h, hp, 0, inst.n_vars, k=25)
    assert best["complete"]
    units = partial_units(best["part_var"], best["part_val"])
    n, cp, li = parse_dimacs(to_dimacs(inst.n_vars, inst.clause_ptr, inst.lits, units))
    X = best["assignment"].astype(np.uint8)[:, None]
    unsat, _ = oracle.check(oracle.CNF(n, cp, li), X)
    assert int(unsat[0]) == 0
