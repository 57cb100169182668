"""Forward product of Eq. 1 as per-sample histograms (tsat_histogram), exact
against the oracle's R = P A.

Covers both forward kernels: the word-per-lane kernel with carry-save vertical
counters (clause length <= 3, N >= 512) and the clause-per-lane transpose
kernel (everything else).  The item sizes 512..4096 give each warp one to
several counter flushes (one per <= 248 clauses), with ragged item tails;
short clauses, duplicate literals and tautologies exercise the masked path."""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_07737_b300 import cnfgen
from paper_2511_07737_b300 import turbosat as ts
from tests.gpu_util import make, snapshot

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    torch.cuda.set_device(0)


def reference_hist(cnfs, offsets, X, lm1):
    out = np.zeros((len(cnfs), lm1, X.shape[1]), np.int32)
    for j, cnf in enumerate(cnfs):
        R = oracle.result_matrix(cnf, X[offsets[j]:offsets[j + 1]])
        for r in range(lm1):
            out[j, r] = (R == r).sum(axis=0)
    return out


def gpu_hist(prob, st):
    lm1 = prob.info["lmax"] + 1
    h = torch.full((prob.info["n_inst"], lm1, st.N), -7, dtype=torch.int32, device="cuda")
    ts.tsat_histogram(st.h, h)
    torch.cuda.synchronize()
    return h.cpu().numpy(), lm1


def set_items(st, ic):
    tun = ts.tsat_get_tuning(st.h)
    tun[0] = ic
    ts.tsat_set_tuning(st.h, tun)


CASES = [
    # (name, instances, N, steps before the check)
    ("3sat-N1024", lambda: [cnfgen.planted_ksat(3000, 12780, 3, 41)], 1024, 0),
    ("3sat-N512", lambda: [cnfgen.planted_ksat(2500, 10650, 3, 42)], 512, 2),
    ("short-dup-N1024", lambda: [cnfgen.tiny_random(400, 5000, 43, kmin=1, kmax=3)], 1024, 0),
    ("short-dup-N512", lambda: [cnfgen.tiny_random(300, 3001, 44, kmin=1, kmax=3)], 512, 1),
    ("batch-k2k3-N1024", lambda: cnfgen.batch_ksat(5, 45, n_lo=50, n_hi=1500, k_lo=3, k_hi=3)
     + [cnfgen.planted_ksat(300, 570, 2, 46)], 1024, 1),
    ("3sat-N256", lambda: [cnfgen.planted_ksat(2000, 8520, 3, 47)], 256, 0),      # transpose kernel
    ("5sat-N1024", lambda: [cnfgen.planted_ksat(500, 8000, 5, 48)], 1024, 0),     # transpose kernel
    ("1sat-N1024", lambda: [cnfgen.tiny_random(200, 700, 49, kmin=1, kmax=1)], 1024, 0),
]


@pytest.mark.parametrize("name,gen,N,steps", CASES, ids=[c[0] for c in CASES])
def test_histogram_exact(name, gen, N, steps):
    insts = gen()
    prob, st, cnfs = make(insts, N)
    hp = ts.hparams(seed=91, norm=ts.NORM_ABSMEAN, binarize=ts.BIN_PHILOX, bin_temp=0.8)
    ts.tsat_init(st.h, hp)
    if steps:
        ts.tsat_step(st.h, hp, steps, stop_on_sat=False)
    s = snapshot(st)
    for ic in (512, 1024, 2048, 4096):
        set_items(st, ic)
        got, lm1 = gpu_hist(prob, st)
        ref = reference_hist(cnfs, prob.var_offsets, s["X"], lm1)
        np.testing.assert_array_equal(got, ref, err_msg=f"{name} items of {ic} clauses")
        # every clause is counted once per sample
        assert (got.sum(axis=1) == np.array([c.C for c in cnfs])[:, None]).all()


def test_histogram_zero_for_unsatisfied_equals_exact_check():
    """h[0] of the forward equals the bit-packed exact check's unsatisfied counts."""
    insts = [cnfgen.planted_ksat(4000, 17040, 3, 50)]
    prob, st, cnfs = make(insts, 1024)
    hp = ts.hparams(seed=5, norm=ts.NORM_SIGNED_MEAN, binarize=ts.BIN_PHILOX)
    ts.tsat_init(st.h, hp)
    ts.tsat_step(st.h, hp, 4, stop_on_sat=False)
    got, _ = gpu_hist(prob, st)
    unsat = torch.zeros(1024, dtype=torch.int32, device="cuda")
    sm = torch.zeros(32, dtype=torch.int32, device="cuda")
    ts.tsat_evaluate(st.h, hp, unsat, sm)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(got[0, 0], unsat.cpu().numpy())
