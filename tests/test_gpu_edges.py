"""Degenerate and extreme inputs through the C ABI, against the FP64 oracle:
the longest clauses the library takes (31 literals after de-duplication) and
the first length it rejects, variables that occur in no clause, rows whose
Eq. 5 mean is zero (the normaliser guard), a one-variable formula, formulas
every assignment satisfies (frozen at step 0), and hundreds of tiny instances
in one batch.  Each runs on the multi-kernel path and, where it applies, on
the persistent solver."""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_07737_b300 import cnfgen
from paper_2511_07737_b300 import turbosat as ts
from paper_2511_07737_b300.autograd import SatObjective
from tests.conftest import rel_err
from tests.gpu_util import TOL_F32, make, run_lockstep, snapshot

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    torch.cuda.set_device(0)


def _cnf(n_vars, clauses):
    ptr = np.concatenate([[0], np.cumsum([len(c) for c in clauses])]).astype(np.int64)
    lits = np.concatenate([np.asarray(c, np.int32) for c in clauses]).astype(np.int32)
    return cnfgen.Instance(n_vars, ptr, lits, np.zeros(n_vars, np.uint8))


def _long_clauses():
    """Clauses of 1..31 distinct literals over 40 variables (signs and
    variables from the seeded generator), plus a 45-literal clause whose
    duplicates reduce it to 31 distinct literals."""
    base = cnfgen.tiny_random(40, 120, 71, kmin=1, kmax=3)
    sgn = (cnfgen.u64(71, 5, 0, 2000) >> np.uint64(63)).astype(np.int64)
    perm = np.argsort(cnfgen.u64(71, 6, 0, 40))
    clauses, k = [], 0
    for L in list(range(1, 32)) * 2:
        vs = np.roll(perm, L)[:L] + 1
        clauses.append([int(v) if sgn[(k + i) % 2000] else -int(v) for i, v in enumerate(vs)])
        k += L
    dup = clauses[30] + clauses[30][:14]
    clauses.append(dup)
    for c in range(base.n_clauses):
        clauses.append(base.lits[base.clause_ptr[c]:base.clause_ptr[c + 1]].tolist())
    return _cnf(40, clauses)


def test_longest_clauses_match_the_oracle():
    inst = _long_clauses()
    cnf = oracle.CNF(inst.n_vars, inst.clause_ptr, inst.lits)
    assert cnf.lmax == 31
    hp = ts.hparams(seed=5, norm=ts.NORM_ABSMEAN, binarize=ts.BIN_PHILOX, tau=0.7)
    _, prob, st, _ = run_lockstep([inst], 64, hp, 3)
    assert prob.info["lmax"] == 31
    h = torch.zeros((1, 32, 64), dtype=torch.int32, device="cuda")
    ts.tsat_histogram(st.h, h)
    R = oracle.result_matrix(cnf, snapshot(st)["X"])
    ref = np.stack([(R == r).sum(axis=0) for r in range(32)])
    np.testing.assert_array_equal(h.cpu().numpy()[0], ref)


def test_clause_longer_than_the_limit_is_rejected():
    inst = _cnf(40, [list(range(1, 33)), [1, -2]])
    with pytest.raises(ts.TsatError) as e:
        ts.Problem([(inst.n_vars, inst.clause_ptr, inst.lits)])
    assert e.value.status == -8          # TSAT_ELEN


def _spread(inst, factor):
    """The same formula with variable v renamed factor * v: the variables in
    between occur in no clause (rows of degree 0 among the others)."""
    lits = np.sign(inst.lits) * (np.abs(inst.lits) * factor)
    return cnfgen.Instance(inst.n_vars * factor, inst.clause_ptr, lits.astype(np.int32),
                           np.zeros(inst.n_vars * factor, np.uint8))


@pytest.mark.parametrize("N,persistent", [(1024, False), (64, False), (64, True)])
def test_variables_in_no_clause(N, persistent):
    inst = _spread(cnfgen.planted_ksat(150, 639, 3, 72), 3)
    hp = ts.hparams(seed=6, norm=ts.NORM_SIGNED_MEAN, binarize=ts.BIN_PHILOX)
    fn = (lambda st: ts.tsat_step_persistent(st.h, hp, 1, stop_on_sat=False)) if persistent else None
    run_lockstep([inst], N, hp, 3, fn)


@pytest.mark.parametrize("norm", [0, 1])
def test_zero_mean_rows_take_the_normaliser_guard(norm):
    inst = cnfgen.planted_ksat(200, 852, 3, 73)
    prob, st, cnfs = make([inst], 64)
    hp = ts.hparams(seed=7, norm=norm, tau=1.1)
    g = torch.Generator(device="cuda").manual_seed(4)
    z = torch.randn(200, 64, device="cuda", generator=g)
    z[0] = 0.0                                   # mean and mean |z| both zero
    z[1, :32], z[1, 32:] = 0.75, -0.75           # signed mean zero, mean |z| 0.75
    z = z.requires_grad_(True)
    loss, S = SatObjective.apply(z, st, hp, 0)
    loss.backward()
    torch.cuda.synchronize()
    zc = z.detach().cpu().numpy()
    nu = st.view("nu").cpu().numpy()
    nu_ref = oracle.nu_f32(zc, norm)
    assert nu[0] == np.float32(nu_ref[0]) and abs(nu_ref[0] - 1e-12) < 1e-18
    if norm == 0:
        assert nu[1] == np.float32(nu_ref[1]) and abs(nu_ref[1] - 1e-12) < 1e-18
    bound = 2e-6 * np.abs(zc).mean(axis=1) + 2e-6 * np.abs(nu_ref)
    assert np.all(np.abs(nu[2:] - nu_ref[2:]) <= bound[2:])
    X = oracle.binarize_f32(zc, nu, 0)
    assert not X[0].any()                        # B(0) = 0
    S_ref, L_ref, G, _ = oracle.objective(cnfs[0], X=X, tau=hp.tau)
    gref = oracle.normalize_backward(zc.astype(np.float64), nu.astype(np.float64), G, norm)
    grad = z.grad.cpu().numpy()
    guarded = np.abs(nu) <= 1e-11
    assert guarded.sum() == (2 if norm == 0 else 1)
    assert rel_err(grad[guarded], gref[guarded]) < TOL_F32        # G / 1e-12: the guard's scale
    assert rel_err(grad[~guarded], gref[~guarded]) < TOL_F32
    assert abs(loss.item() - L_ref) < TOL_F32 * abs(L_ref)


@pytest.mark.parametrize("persistent", [False, True])
def test_one_variable_and_always_satisfied_formulas(persistent):
    one = _cnf(1, [[1], [1, -1]])                                   # satisfied iff x1
    taut = _cnf(5, [[1, -1], [2, -2, 3], [-4, 4], [5, -5, 1, 2]])   # every assignment satisfies it
    other = cnfgen.planted_ksat(60, 240, 3, 74)
    insts = [one, taut, other]
    hp = ts.hparams(seed=8, norm=ts.NORM_ABSMEAN, tau=2.0, lr0=0.5)
    fn = (lambda st: ts.tsat_step_persistent(st.h, hp, 1, stop_on_sat=False)) if persistent else None
    status, prob, st, cnfs = run_lockstep(insts, 32, hp, 4, fn)
    assert status["inst"][1]["found"] and status["inst"][1]["found_step"] == 0
    assert status["inst"][1]["min_unsat"] == 0
    if status["inst"][0]["found"]:
        X = snapshot(st)["X"]
        assert X[0, status["inst"][0]["found_sample"]] == 1


@pytest.mark.parametrize("persistent", [False, True])
def test_hundreds_of_tiny_instances(persistent):
    insts = [cnfgen.planted_ksat(8 + j % 5, 20 + j % 7, 3, 1000 + j) for j in range(300)]
    hp = ts.hparams(seed=9, norm=ts.NORM_NONE, binarize=ts.BIN_PHILOX, tau=2.0)
    fn = (lambda st: ts.tsat_step_persistent(st.h, hp, 1, stop_on_sat=False)) if persistent else None
    status, _, _, _ = run_lockstep(insts, 32, hp, 2, fn)
    assert len(status["inst"]) == 300


@pytest.mark.parametrize("n,m,N,persistent", [(40, 2400, 64, False), (40, 2400, 64, True), (60, 3600, 256, True),
                                              (40, 2400, 1024, True), (40, 2400, 1024, False)])
def test_variables_with_more_than_127_occurrences(n, m, N, persistent):
    """Clause length 3 with about 180 occurrences per variable: the fused
    updates count occurrences in signed byte counters of at most 127 per
    chunk, so every row takes several chunks (persistent solver: resident at
    N = 64 with 16 samples per thread, not resident at N = 256 with 8, 32 at
    N = 1024)."""
    inst = cnfgen.planted_ksat(n, m, 3, 75)
    deg = np.bincount(np.abs(inst.lits) - 1, minlength=n)
    assert deg.min() > 127
    hp = ts.hparams(seed=10, norm=ts.NORM_ABSMEAN, binarize=ts.BIN_PHILOX, tau=1.5)
    fn = (lambda st: ts.tsat_step_persistent(st.h, hp, 1, stop_on_sat=False)) if persistent else None
    run_lockstep([inst], N, hp, 3, fn)


def test_literal_rows_model_matches_the_oracle_and_decodes():
    """The 2V literal-row model (one independent row per literal, built as a
    CNF transform) runs the unchanged kernels: lock-step parity against the
    oracle on the transformed formula, and the unsatisfied counts of the
    decoded assignment (x_v = row v+) on the original formula equal the
    oracle's exact check."""
    from paper_2511_07737_b300 import literal_rows
    inst = cnfgen.planted_ksat(100, 426, 3, 3)
    t = literal_rows.split_literals(inst)
    hp = ts.hparams(seed=4, norm=ts.NORM_ABSMEAN, tau=2.0, lr0=0.5)
    _, _, st, _ = run_lockstep([t], 64, hp, 3)
    orig = ts.Problem([(inst.n_vars, inst.clause_ptr, inst.lits)])
    u = literal_rows.decoded_unsat(orig, st, hp.tau)
    X = snapshot(st)["X"][:inst.n_vars]
    ref, _ = oracle.check(oracle.CNF(inst.n_vars, inst.clause_ptr, inst.lits), X)
    np.testing.assert_array_equal(u, ref)
    frac = literal_rows.inconsistent_fraction(st, inst.n_vars)
    both = (X == snapshot(st)["X"][inst.n_vars:]).mean()
    assert abs(frac - both) < 1e-12
