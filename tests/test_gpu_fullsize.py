"""Parity at the workloads' full sizes, each in the launch configuration its
benchmark times: planted 3-SAT n = 1,000,000 with N = 1024 (the headline
step), the relaxed layer on structured mixed k-SAT n = 2,000,000 with N = 256,
and the 512-instance batch with N = 64 after autotuning (the last two are
described at their tests).

Planted 3-SAT n = 1,000,000, m = 4,200,000, N = 1024 samples, FP32 state,
signed-mean Eq. 5 and Philox binarisation, through tsat_step's graph replay
with the default launch shapes.

The FP64 oracle cannot hold the whole state at this size, so the outputs are
sampled:
  * the forward's per-sample histograms (Eq. 1), exact, on 64 of the 1024
    sample columns, and h[0] = the unsatisfied counts on all columns;
  * the loss of the step (Eqs. 3, 4) over all columns, 1e-5 relative;
  * one whole optimisation step on sampled variable rows: the oracle forms the
    STE gradient of those rows over all 1024 columns (the Eq. 5 chain rule
    couples a row's samples), then Eq. 5, AdamW and the bits of the next step
    (Philox rule, bit-exact on rows 0..511, whose counters the oracle indexes
    the same way) are compared with the GPU's state after the step."""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_07737_b300 import cnfgen
from paper_2511_07737_b300 import turbosat as ts
from tests.conftest import rel_err
from tests.gpu_util import TOL_BF16, TOL_F32, assert_adamw_z, oracle_hp, unpack_bits

pytestmark = pytest.mark.gpu

N = 1024
CHUNK = 32


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    torch.cuda.set_device(0)


def test_full_size_step_matches_oracle_on_samples():
    inst = cnfgen.planted_ksat(1_000_000, 4_200_000, 3, 1)
    prob = ts.Problem([(inst.n_vars, inst.clause_ptr, inst.lits)])
    st = ts.State(prob, N)
    hp = ts.hparams(seed=1, norm=ts.NORM_SIGNED_MEAN, binarize=ts.BIN_PHILOX, bin_temp=1.0, tau=1.0)
    ts.tsat_init(st.h, hp)
    t = 3
    ts.tsat_step(st.h, hp, t, stop_on_sat=False)
    rng = np.random.default_rng(7)
    rows = np.unique(np.concatenate([np.arange(512), rng.choice(inst.n_vars, 256, replace=False)]))
    rows_d = torch.from_numpy(rows).cuda()
    torch.cuda.synchronize()
    X = unpack_bits(st.view("bits").cpu().numpy().view(np.uint32), N)       # bits of step t, [V][N]
    nu0 = st.view("nu").cpu().numpy()[rows].astype(np.float64)
    z0, m0, v0 = (st.view(k)[rows_d].cpu().numpy() for k in ("z", "m", "v"))
    hist = torch.zeros((1, prob.info["lmax"] + 1, N), dtype=torch.int32, device="cuda")
    ts.tsat_histogram(st.h, hist)
    unsat = torch.zeros(N, dtype=torch.int32, device="cuda")
    sm = torch.zeros(N // 32, dtype=torch.int32, device="cuda")
    ts.tsat_evaluate(st.h, hp, unsat, sm)
    ts.tsat_step(st.h, hp, 1, stop_on_sat=False)                            # step t, as the benchmark runs it
    torch.cuda.synchronize()
    status = ts.tsat_status(st.h, 1)
    z1, m1, v1 = (st.view(k)[rows_d].cpu().numpy() for k in ("z", "m", "v"))
    nu1 = st.view("nu").cpu().numpy()[rows]
    X1 = unpack_bits(st.view("bits").cpu().numpy().view(np.uint32)[:512], N)
    hist = hist.cpu().numpy()[0]
    unsat = unsat.cpu().numpy()

    cnf = oracle.CNF(inst.n_vars, inst.clause_ptr, inst.lits)
    # forward: exact histograms on two chunks of columns (first and last word)
    for c0 in (0, N - CHUNK):
        R = oracle.result_matrix(cnf, np.ascontiguousarray(X[:, c0:c0 + CHUNK]))
        ref = np.stack([(R == r).sum(axis=0) for r in range(hist.shape[0])])
        np.testing.assert_array_equal(hist[:, c0:c0 + CHUNK], ref)
        del R
    assert (hist.sum(axis=0) == inst.n_clauses).all()
    # objective and STE gradient of the sampled rows over all columns
    G = np.zeros((rows.size, N))
    S = np.zeros(N)
    ref_unsat = np.zeros(N, np.int32)
    for c0 in range(0, N, CHUNK):
        Sc, _, Gc, uc = oracle.objective(cnf, X=np.ascontiguousarray(X[:, c0:c0 + CHUNK]), tau=hp.tau, grad=True)
        S[c0:c0 + CHUNK], ref_unsat[c0:c0 + CHUNK] = Sc, uc
        G[:, c0:c0 + CHUNK] = Gc[rows]
        del Gc
    np.testing.assert_array_equal(unsat, ref_unsat)
    np.testing.assert_array_equal(hist[0], ref_unsat)
    L = -S.sum()
    assert abs(status["inst"][0]["loss"] - L) <= TOL_F32 * abs(L)
    assert status["inst"][0]["min_unsat"] == int(ref_unsat.min())
    # Eq. 5 chain rule and AdamW on the sampled rows, from the GPU's FP32 state
    g = oracle.normalize_backward(z0.astype(np.float64), nu0, G, hp.norm)
    z, m, v = (np.ascontiguousarray(a, dtype=np.float64) for a in (z0, m0, v0))
    lr = oracle.lr_at(t, hp.lr0, hp.lr_factor, hp.decay_period, hp.restart_period, hp.lr_floor)
    oracle.adamw(z, m, v, g, t + 1, lr, hp.beta1, hp.beta2, hp.eps, hp.weight_decay)
    assert_adamw_z(z1, z, m1, m, v1, v, t, hp)
    # new normaliser and the Philox bits of step t + 1 (rows 0..511)
    nu_ref = oracle.nu_f32(z1, hp.norm)
    assert np.all(np.abs(nu1 - nu_ref) <= 2e-6 * np.abs(z1).mean(axis=1) + 2e-6 * np.abs(nu_ref))
    head = rows < 512
    Xr = oracle.binarize_f32(z1[head], nu1[head], hp.binarize, c=0.25 / hp.bin_temp, seed=hp.seed, t=t + 1)
    np.testing.assert_array_equal(X1, Xr)


COLS = np.array([0, 1, 31, 32, 97, 130, 224, 255])


def _bit_columns(words: np.ndarray, cols: np.ndarray) -> np.ndarray:
    """[V][N/32] words -> [V][len(cols)] 0/1 of the chosen sample columns."""
    w = words.view(np.uint32)
    return np.stack([(w[:, c // 32] >> np.uint32(c % 32)) & np.uint32(1) for c in cols], axis=1).astype(np.uint8)


@pytest.fixture(scope="module")
def structured():
    inst = cnfgen.structured_mixed(2_000_000, 8_000_000, 5)
    # loaded as the relaxed experiment loads it: clauses ordered by smallest variable
    prob = ts.Problem([(inst.n_vars, inst.clause_ptr, inst.lits)], locality=True)
    return inst, prob, oracle.CNF(inst.n_vars, inst.clause_ptr, inst.lits)


@pytest.mark.parametrize("dtype,tol", [(ts.DTYPE_F32, TOL_F32), (ts.DTYPE_BF16, TOL_BF16)], ids=["fp32", "bf16"])
def test_relaxed_full_size_matches_oracle_on_columns(structured, dtype, tol):
    """Structured mixed k-SAT n = 2,000,000, m = 8,000,000 (lengths 2-16,
    power-law occurrences in 64 communities), N = 256 samples, the relaxed
    (sigmoid) layer with FP32 or BF16 literal storage, through tsat_step's
    graph replay with the default launch shapes.

    Without the Eq. 5 scaling (norm none) the samples of a step are
    independent, so the oracle takes a whole step on 8 sampled columns over
    all 2,000,000 rows: z / m / v after AdamW, the Eq. 2 bits and the exact
    check's counts of those columns.  With absmean scaling (whose per-row
    normaliser the oracle forms from all 256 columns) it computes the relaxed
    S_i (Eq. 4) of the same columns.  The gradient is checked by a central
    difference of the FP64 oracle along sign(GPU gradient) on a 5,000-variable
    slice of the sampled columns."""
    inst, prob, cnf = structured
    N = 256
    st = ts.State(prob, N, ts.LAYER_RELAXED, dtype)
    hp = ts.hparams(seed=3, norm=ts.NORM_NONE, layer=ts.LAYER_RELAXED)
    ts.tsat_init(st.h, hp)
    t = 2
    ts.tsat_step(st.h, hp, t, stop_on_sat=False)
    cols_d = torch.from_numpy(COLS).cuda()
    torch.cuda.synchronize()
    z0, m0, v0 = (st.view(k)[:, cols_d].cpu().numpy() for k in ("z", "m", "v"))
    nu0 = st.view("nu").cpu().numpy().astype(np.float64)
    ts.tsat_step(st.h, hp, 1, stop_on_sat=False)
    unsat = torch.zeros(N, dtype=torch.int32, device="cuda")
    sm = torch.zeros(N // 32, dtype=torch.int32, device="cuda")
    ts.tsat_evaluate(st.h, hp, unsat, sm)
    torch.cuda.synchronize()
    z1, m1, v1 = (st.view(k)[:, cols_d].cpu().numpy() for k in ("z", "m", "v"))
    nu1 = st.view("nu").cpu().numpy()
    X1 = _bit_columns(st.view("bits").cpu().numpy(), COLS)

    z, m, v = (np.ascontiguousarray(a, dtype=np.float64) for a in (z0, m0, v0))
    oracle.step(cnf, oracle_hp(hp), t, z, m, v, nu_in=nu0)
    assert_adamw_z(z1, z, m1, m, v1, v, t, hp, tol=tol)
    np.testing.assert_array_equal(X1, oracle.binarize_f32(z1, nu1, hp.binarize))
    np.testing.assert_array_equal(unsat.cpu().numpy()[COLS], oracle.check(cnf, X1)[0])

    # relaxed S_i under absmean Eq. 5 on the sampled columns
    zf = st.view("z")
    hp1 = ts.hparams(seed=3, norm=ts.NORM_ABSMEAN, layer=ts.LAYER_RELAXED)
    S = torch.zeros(N, device="cuda")
    L = torch.zeros(1, device="cuda")
    ts.tsat_forward(st.h, hp1, zf, 0, S, L)
    torch.cuda.synchronize()
    nu_abs = oracle.nu_f32(zf.cpu().numpy(), ts.NORM_ABSMEAN)
    S_ref, _, _, _ = oracle.objective(cnf, zt=z1.astype(np.float64) / nu_abs[:, None], tau=hp1.tau, grad=False)
    assert rel_err(S.cpu().numpy()[COLS], S_ref) < tol
    # the backward reuses its forward's gamma table: forward again under norm none
    ts.tsat_forward(st.h, hp, zf, 0, S, L)
    grad = torch.zeros_like(zf)
    ts.tsat_backward(st.h, hp, zf, 1.0, grad)                     # norm none: columns independent

    # central difference of the oracle (FP64) along sign(gradient) on 5,000 rows
    gc = grad[:, cols_d].cpu().numpy().astype(np.float64)
    rows = np.random.default_rng(11).choice(inst.n_vars, 5000, replace=False)
    d = np.zeros_like(gc)
    d[rows] = np.sign(gc[rows])
    h = 1e-3
    zc = z1.astype(np.float64)
    Lp = oracle.objective(cnf, zt=zc + h * d, tau=hp.tau, grad=False)[1]
    Lm = oracle.objective(cnf, zt=zc - h * d, tau=hp.tau, grad=False)[1]
    fd = (Lp - Lm) / (2 * h)
    an = float((gc * d).sum())
    # FP64 evaluation error of L is ~1e-13 |L|; the O(h^2) term is below 1e-6 |an|
    assert abs(fd - an) <= max(1e-3, tol) * abs(an), (fd, an)
    del st, grad
    torch.cuda.empty_cache()


def test_batch_full_size_matches_oracle_per_instance():
    """The 512-instance batch at full size (planted k-SAT, k uniform 3..7,
    n log-uniform 200..50,000, 0.9 x threshold; N = 64 restarts each, absmean
    Eq. 5, tau 2, lr0 0.5), launch shapes chosen by tsat_autotune, steps by
    the graph replay.

    The forward, check and state of one instance depend on that instance
    alone, so the oracle checks whole instances one by one: the smallest and
    the largest (up to 2e6 literals) instance of each k and the first and
    last of the batch, one step from the GPU's FP32 state (status record,
    z / m / v after AdamW, the next bits and normaliser) and their exact
    histograms (Eq. 1).  Over all 512 instances every histogram sums to the
    instance's clause count and its r = 0 row equals the check's counts."""
    insts = cnfgen.batch_ksat(512, 3)
    prob = ts.Problem([(i.n_vars, i.clause_ptr, i.lits) for i in insts])
    N = 64
    st = ts.State(prob, N)
    hp = ts.hparams(seed=2, norm=ts.NORM_ABSMEAN, tau=2.0, lr0=0.5)
    ts.tsat_init(st.h, hp)
    ts.tsat_autotune(st.h, hp)
    t = 3
    ts.tsat_step(st.h, hp, t, stop_on_sat=False)

    ks = np.array([int(np.diff(i.clause_ptr).max()) for i in insts])
    nnz = np.array([i.nnz for i in insts])
    sel = {0, len(insts) - 1}
    for k in range(3, 8):
        idx = np.nonzero(ks == k)[0]
        sel.add(int(idx[np.argmin(nnz[idx])]))
        small = idx[nnz[idx] <= 2_000_000]
        sel.add(int(small[np.argmax(nnz[small])]))
    sel = sorted(sel)
    offs = prob.var_offsets
    lmax = prob.info["lmax"]

    def rows(name, j):
        return st.view(name)[offs[j]:offs[j + 1]].cpu().numpy().copy()

    torch.cuda.synchronize()
    s0 = {j: {k: rows(k, j) for k in ("z", "m", "v", "nu", "bits")} for j in sel}
    hist = torch.zeros((len(insts), lmax + 1, N), dtype=torch.int32, device="cuda")
    ts.tsat_histogram(st.h, hist)
    unsat = torch.zeros(len(insts) * N, dtype=torch.int32, device="cuda")
    sm = torch.zeros(len(insts) * N // 32, dtype=torch.int32, device="cuda")
    ts.tsat_evaluate(st.h, hp, unsat, sm)
    ts.tsat_step(st.h, hp, 1, stop_on_sat=False)
    torch.cuda.synchronize()
    status = ts.tsat_status(st.h, len(insts))
    s1 = {j: {k: rows(k, j) for k in ("z", "m", "v", "nu", "bits")} for j in sel}
    hist = hist.cpu().numpy()
    unsat = unsat.cpu().numpy().reshape(len(insts), N)

    np.testing.assert_array_equal(hist.sum(axis=1), np.array([i.n_clauses for i in insts])[:, None].repeat(N, 1))
    np.testing.assert_array_equal(hist[:, 0, :], unsat)
    ohp = oracle_hp(hp)
    for j in sel:
        cnf = oracle.CNF(insts[j].n_vars, insts[j].clause_ptr, insts[j].lits)
        X0 = unpack_bits(s0[j]["bits"], N)
        R = oracle.result_matrix(cnf, X0)
        np.testing.assert_array_equal(hist[j], np.stack([(R == r).sum(axis=0) for r in range(lmax + 1)]))
        x = status["inst"][j]
        if x["found"] and x["found_step"] < t:
            continue
        z, m, v = (s0[j][k].astype(np.float64) for k in ("z", "m", "v"))
        res = oracle.step(cnf, ohp, t, z, m, v, X=X0, nu_in=s0[j]["nu"].astype(np.float64))
        np.testing.assert_array_equal(unsat[j], res["unsat"])
        assert x["min_unsat"] == int(res["unsat"].min())
        assert abs(x["loss"] - res["L"]) <= TOL_F32 * abs(res["L"])
        X1 = unpack_bits(s1[j]["bits"], N)
        if x["found"]:                                   # frozen on the model it found at step t
            np.testing.assert_array_equal(X1, X0)
            continue
        assert x["best_sample"] == oracle.best_sample(res["unsat"])
        assert_adamw_z(s1[j]["z"], z, s1[j]["m"], m, s1[j]["v"], v, t, hp)
        np.testing.assert_array_equal(X1, oracle.binarize_f32(s1[j]["z"], s1[j]["nu"], hp.binarize))
        nu_ref = oracle.nu_f32(s1[j]["z"], hp.norm)
        assert np.all(np.abs(s1[j]["nu"] - nu_ref) <= 2e-6 * np.abs(s1[j]["z"]).mean(axis=1) + 2e-6 * np.abs(nu_ref))
