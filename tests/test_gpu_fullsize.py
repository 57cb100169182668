"""Parity at the benchmark's full size: planted 3-SAT n = 1,000,000,
m = 4,200,000, N = 1024 samples, FP32 state, signed-mean Eq. 5 and Philox
binarisation, through tsat_step's graph replay with the default launch shapes
(the kernels and grid bench.py times).

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
from tests.gpu_util import TOL_F32, assert_adamw_z, unpack_bits

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
