"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Integers (CSR, unsatisfied counts, SAT masks, sampled bits, selected
variables) must agree exactly; FP32 results within 1e-5 max-norm relative
error, BF16 literal storage within 1e-2."""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_07737_b300 import cnfgen
from paper_2511_07737_b300 import turbosat as ts
from tests.conftest import rel_err
from tests.gpu_util import (TOL_BF16, TOL_F32, assert_adamw_z, binarize_like_gpu, lockstep, make, snapshot,
                            unpack_bits)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("locality", [False, True])
def test_layout_matches_oracle_parse(locality):
    """The device CSR equals the oracle's parse; with the locality load the
    clauses are stored ordered by their smallest variable and exported in the
    caller's order."""
    inst = cnfgen.tiny_random(40, 300, 3, kmin=1, kmax=9)     # duplicates and tautologies
    prob = ts.Problem([(inst.n_vars, inst.clause_ptr, inst.lits)], locality=locality)
    cptr, clit = ts.tsat_problem_csr(prob.h)
    cnf = oracle.CNF(inst.n_vars, inst.clause_ptr, inst.lits)
    np.testing.assert_array_equal(cptr.astype(np.int64), cnf.cptr)
    for c in range(cnf.C):
        gpu = sorted(clit[cptr[c]:cptr[c + 1]].tolist())
        ref = sorted(((cnf.var[j] << 1) | cnf.neg[j]) for j in range(cnf.cptr[c], cnf.cptr[c + 1]))
        assert gpu == ref
    assert prob.info["lmax"] == cnf.lmax


def test_locality_load_keeps_results_and_numbering():
    """A batch loaded with its clauses ordered by smallest variable gives the
    same integer results and the same (up to FP32 summation order) state as the
    caller's order: unsatisfied counts exactly, the relaxed layer's m / v within
    1e-5 and z within its AdamW bound after a step; errors name the caller's
    clause index."""
    insts = [cnfgen.structured_mixed(3000, 12000, 21, communities=8), cnfgen.planted_ksat(500, 2100, 3, 4)]
    hp = ts.hparams(seed=5, norm=1, layer=ts.LAYER_RELAXED, tau=1.1)
    outs = []
    for loc in (False, True):
        prob = ts.Problem([(i.n_vars, i.clause_ptr, i.lits) for i in insts], locality=loc)
        st = ts.State(prob, 64, ts.LAYER_RELAXED)
        ts.tsat_init(st.h, hp)
        ts.tsat_step(st.h, hp, 1, stop_on_sat=False)
        u = torch.zeros(2 * 64, dtype=torch.int32, device="cuda")
        sm = torch.zeros(4, dtype=torch.int32, device="cuda")
        ts.tsat_evaluate(st.h, hp, u, sm)
        outs.append((snapshot(st), u.cpu().numpy()))
    (a, ua), (b, ub) = outs
    np.testing.assert_array_equal(ua, ub)
    # one step from the same init: m, v to 1e-5; z to the first-order AdamW
    # bound of its m / v differences (where |g| is near eps the update is
    # ill-conditioned, as in the oracle lock-step)
    assert_adamw_z(b["z"], a["z"].astype(np.float64), b["m"], a["m"].astype(np.float64), b["v"],
                   a["v"].astype(np.float64), 0, hp)
    bad_ptr = np.array([0, 2, 4, 4, 6], np.int64)
    bad_lits = np.array([3, -2, 1, 2, 2, 1], np.int32)       # clause 2 (caller's order) is empty
    with pytest.raises(ts.TsatError) as e:
        ts.Problem([(3, bad_ptr, bad_lits)], locality=True)
    assert e.value.status == -3 and "clause 2 " in str(e.value)


@pytest.mark.parametrize("bad,status", [
    (([0, 2, 2], [1, 2]), -3),
    (([0, 2], [1, 5]), -2),
    (([0, 2], [1, 0]), -2),
])
def test_load_errors(bad, status):
    ptr, lits = bad
    with pytest.raises(ts.TsatError) as e:
        ts.Problem([(3, np.array(ptr), np.array(lits))])
    assert e.value.status == status


@pytest.mark.parametrize("N,norm,binz", [(64, 0, 0), (32, 1, 1), (256, 2, 0), (1024, 1, 1)])
def test_init_bits_and_check(N, norm, binz):
    inst = cnfgen.planted_ksat(300, 1278, 3, 2)
    prob, st, cnfs = make([inst], N)
    hp = ts.hparams(seed=12345, norm=norm, binarize=binz, bin_temp=0.7)
    ts.tsat_init(st.h, hp)
    s = snapshot(st)
    np.testing.assert_array_equal(s["z"], oracle.init_normal(inst.n_vars, N, 12345))
    np.testing.assert_array_equal(s["m"], 0)
    nu_ref = oracle.nu_f32(s["z"], norm)
    bound = 1e-6 * np.abs(s["z"]).mean(axis=1) + 1e-6 * np.abs(nu_ref)
    assert np.all(np.abs(s["nu"] - nu_ref) <= bound)
    X = oracle.binarize_f32(s["z"], s["nu"], binz, c=0.25 / 0.7, seed=12345, t=0)
    np.testing.assert_array_equal(s["X"], X)
    unsat = torch.zeros(N, dtype=torch.int32, device="cuda")
    sm = torch.zeros(N // 32, dtype=torch.int32, device="cuda")
    ts.tsat_evaluate(st.h, hp, unsat, sm)
    ref_u, ref_sm = oracle.check(cnfs[0], s["X"])
    np.testing.assert_array_equal(unsat.cpu().numpy(), ref_u)
    np.testing.assert_array_equal(sm.cpu().numpy().view(np.uint32), ref_sm)


CASES = [
    # (instances, N, hp kwargs, steps)
    ("c0", lambda: [cnfgen.planted_ksat(100, 426, 3, 0)], 64, dict(norm=0, binarize=0), 6),
    ("c0-philox", lambda: [cnfgen.planted_ksat(100, 426, 3, 0)], 64, dict(norm=1, binarize=1, bin_temp=0.5), 6),
    ("ragged-items", lambda: [cnfgen.planted_ksat(3000, 12780, 3, 4)], 256, dict(norm=0, binarize=1), 3),
    ("wide-N", lambda: [cnfgen.planted_ksat(1500, 6390, 3, 5)], 1024, dict(norm=1, binarize=0), 3),
    ("N32-none", lambda: [cnfgen.planted_ksat(700, 2982, 3, 6)], 32, dict(norm=2, binarize=1), 3),
    ("mixed-k", lambda: [cnfgen.structured_mixed(2048, 8000, 7, communities=8)], 128, dict(norm=1, binarize=1), 3),
    ("k7", lambda: [cnfgen.planted_ksat(400, 14000, 7, 8)], 64, dict(norm=0, binarize=0), 2),
    ("batch", lambda: cnfgen.batch_ksat(5, 9, n_lo=60, n_hi=900), 64, dict(norm=1, binarize=1), 3),
    # clause length 4..7 (fixed 8-int records): gamma table in shared memory (N <= 128) or through L1
    ("k5-N256", lambda: [cnfgen.planted_ksat(600, 6000, 5, 31)], 256, dict(norm=2, binarize=1), 3),
    ("k4-N1024", lambda: [cnfgen.planted_ksat(300, 2400, 4, 32)], 1024, dict(norm=1, binarize=0), 2),
    ("k6-N128", lambda: [cnfgen.planted_ksat(500, 12000, 6, 35)], 128, dict(norm=0, binarize=1), 2),
    # many small instances per warp (row groups span several instances)
    ("batch-N32", lambda: cnfgen.batch_ksat(12, 33, n_lo=20, n_hi=80, k_lo=4, k_hi=6), 32, dict(norm=0, binarize=1), 3),
    ("batch-N128", lambda: cnfgen.batch_ksat(6, 34, n_lo=40, n_hi=300), 128, dict(norm=1, binarize=0), 3),
]


@pytest.mark.parametrize("name,gen,N,kw,steps", CASES, ids=[c[0] for c in CASES])
def test_lockstep_ste(name, gen, N, kw, steps):
    insts = gen()
    prob, st, cnfs = make(insts, N)
    hp = ts.hparams(seed=77, tau=1.3, **kw)
    ts.tsat_init(st.h, hp)
    offs = prob.var_offsets
    for t in range(steps):
        s0 = snapshot(st)
        ts.tsat_step(st.h, hp, 1, stop_on_sat=False)
        s1 = snapshot(st)
        z, m, v, res = lockstep(cnfs, offs, hp, t, s0)
        status = ts.tsat_status(st.h, len(insts))
        for j, r in enumerate(res):
            if status["inst"][j]["found"] and status["inst"][j]["found_step"] < t:
                continue
            assert status["inst"][j]["min_unsat"] == int(r["unsat"].min())
            assert abs(status["inst"][j]["loss"] - r["L"]) <= TOL_F32 * abs(r["L"])
        frozen = np.zeros(prob.info["n_vars"], bool)
        for j in range(len(insts)):
            if status["inst"][j]["found"]:
                frozen[offs[j]:offs[j + 1]] = True
        live = ~frozen
        assert_adamw_z(s1["z"][live], z[live], s1["m"][live], m[live], s1["v"][live], v[live], t, hp)
        # bits of step t+1: Eq. 2 / Philox rule on the GPU's own FP32 z and nu
        X = binarize_like_gpu(s1["z"], s1["nu"], hp, t + 1, offs)
        np.testing.assert_array_equal(s1["X"][live], X[live])
        np.testing.assert_array_equal(s1["X"][frozen], s0["X"][frozen])
        nu_ref = oracle.nu_f32(s1["z"], hp.norm)
        bound = 2e-6 * np.abs(s1["z"]).mean(axis=1) + 2e-6 * np.abs(nu_ref)
        assert np.all(np.abs(s1["nu"] - nu_ref) <= bound)
    assert ts.tsat_status(st.h, len(insts))["step"] == steps


def test_lockstep_assignment_mixing_at_restarts():
    # restart period 3: steps 3 and 6 mix assignments per instance (best sample
    # kept, the others averaged with it, moments zeroed), the AdamW step count
    # restarts after each; both layouts of instance rows in a warp (N = 64)
    insts = [cnfgen.planted_ksat(90, 380, 3, 41), cnfgen.planted_ksat(70, 290, 3, 42)]
    prob, st, cnfs = make(insts, 64)
    hp = ts.hparams(seed=5, tau=1.5, norm=1, binarize=1, restart_period=3, decay_period=1, mix_restart=1)
    ts.tsat_init(st.h, hp)
    offs = prob.var_offsets
    for t in range(8):
        s0 = snapshot(st)
        ts.tsat_step(st.h, hp, 1, stop_on_sat=False)
        s1 = snapshot(st)
        z, m, v, res = lockstep(cnfs, offs, hp, t, s0)
        status = ts.tsat_status(st.h, len(insts))
        for j, r in enumerate(res):
            assert status["inst"][j]["min_unsat"] == int(r["unsat"].min())
            assert status["inst"][j]["best_sample"] == int(np.argmin(r["unsat"]))
        if t > 0 and t % 3 == 0:
            assert rel_err(s1["z"], z) < 1e-6
            assert not s1["m"].any() and not s1["v"].any()
        else:
            cnt = t % 3 if t >= 3 else t + 1
            assert_adamw_z(s1["z"], z, s1["m"], m, s1["v"], v, t, hp, cnt=cnt)
        X = binarize_like_gpu(s1["z"], s1["nu"], hp, t + 1, offs)
        np.testing.assert_array_equal(s1["X"], X)
        nu_ref = oracle.nu_f32(s1["z"], hp.norm)
        assert np.all(np.abs(s1["nu"] - nu_ref) <= 2e-6 * np.abs(s1["z"]).mean(axis=1) + 2e-6 * np.abs(nu_ref))


@pytest.mark.parametrize("norm,k,N", [(0, 3, 128), (1, 3, 128), (2, 3, 128), (1, 5, 64), (0, 6, 256)])
def test_autograd_hooks_match_oracle_gradient(norm, k, N):
    m = 2130 if k == 3 else int(round(0.8 * cnfgen.KSAT_THRESHOLD[k] * 500))
    inst = cnfgen.planted_ksat(500, m, k, 3)
    prob, st, cnfs = make([inst], N)
    hp = ts.hparams(seed=3, norm=norm, tau=0.8)
    z = torch.randn(500, N, device="cuda", generator=torch.Generator(device="cuda").manual_seed(4)) + 0.5
    S = torch.zeros(N, device="cuda")
    L = torch.zeros(1, device="cuda")
    ts.tsat_forward(st.h, hp, z, 0, S, L)
    grad = torch.zeros_like(z)
    ts.tsat_backward(st.h, hp, z, 1.0, grad)
    torch.cuda.synchronize()
    zc = z.cpu().numpy()
    nu_gpu = st.view("nu").cpu().numpy()
    nu = oracle.nu_f32(zc, norm)
    assert np.all(np.abs(nu_gpu - nu) <= 2e-6 * np.abs(zc).mean(axis=1) + 2e-6 * np.abs(nu))
    nu = nu_gpu.astype(np.float64)      # FP32 statistic of the GPU, as in the lock-step tests
    X = oracle.binarize_f32(zc, nu_gpu, 0)
    S_ref, L_ref, G, _ = oracle.objective(cnfs[0], X=X, tau=0.8)
    g = oracle.normalize_backward(zc.astype(np.float64), nu, G, norm)
    assert rel_err(S.cpu().numpy(), S_ref) < TOL_F32
    assert abs(L.item() - L_ref) < TOL_F32 * abs(L_ref)
    assert rel_err(grad.cpu().numpy(), g) < TOL_F32


@pytest.mark.parametrize("dtype,tol,locality", [(ts.DTYPE_F32, TOL_F32, False), (ts.DTYPE_BF16, TOL_BF16, False),
                                                (ts.DTYPE_F32, TOL_F32, True), (ts.DTYPE_BF16, TOL_BF16, True)])
def test_lockstep_relaxed(dtype, tol, locality):
    inst = cnfgen.structured_mixed(1024, 4000, 5, communities=8)
    prob, st, cnfs = make([inst], 64, layer=ts.LAYER_RELAXED, dtype=dtype, locality=locality)
    hp = ts.hparams(seed=5, norm=1, layer=ts.LAYER_RELAXED, tau=1.1)
    ts.tsat_init(st.h, hp)
    for t in range(3):
        s0 = snapshot(st)
        ts.tsat_step(st.h, hp, 1, stop_on_sat=False)
        s1 = snapshot(st)
        z, m, v, res = lockstep(cnfs, prob.var_offsets, hp, t, s0)
        status = ts.tsat_status(st.h, 1)
        assert abs(status["inst"][0]["loss"] - res[0]["L"]) <= tol * abs(res[0]["L"])
        assert_adamw_z(s1["z"], z, s1["m"], m, s1["v"], v, t, hp, tol=tol)


def test_relaxed_autograd_fd():
    """Directional central difference of the GPU relaxed objective (FP32) on a
    5,000-variable slice, along sign(gradient) so that the signal dominates the
    FP32 evaluation noise of L."""
    inst = cnfgen.structured_mixed(8192, 32000, 11, communities=16)
    prob, st, cnfs = make([inst], 64, layer=ts.LAYER_RELAXED)
    hp = ts.hparams(seed=2, norm=1, layer=ts.LAYER_RELAXED)
    g = torch.Generator(device="cuda").manual_seed(0)
    z = torch.randn(8192, 64, device="cuda", generator=g) + 0.1
    S = torch.zeros(64, device="cuda")
    L = torch.zeros(1, device="cuda")
    ts.tsat_forward(st.h, hp, z, 0, S, L)
    grad = torch.zeros_like(z)
    ts.tsat_backward(st.h, hp, z, 1.0, grad)
    rows = torch.randperm(8192, generator=torch.Generator().manual_seed(1))[:5000].cuda()
    d = torch.zeros_like(z)
    d[rows] = torch.sign(grad[rows])
    h = 1e-2
    Lp, Lm = torch.zeros(1, device="cuda"), torch.zeros(1, device="cuda")
    ts.tsat_forward(st.h, hp, z + h * d, 0, S, Lp)
    Sabs = float(S.abs().sum().item())
    ts.tsat_forward(st.h, hp, z - h * d, 0, S, Lm)
    torch.cuda.synchronize()
    fd = (Lp.item() - Lm.item()) / (2 * h)
    an = float((grad * d).sum().item())
    # FP32 evaluation error of L: S_i = Y_i / Z_i with Y, Z blocked FP32 sums
    # over C clauses, relative error <= ~2e-6 each -> |dL| <= 4e-6 sum|S_i|;
    # central differences add 2 |dL| / (2 h), the O(h^2) term is below 1e-3 |an|.
    noise = 2 * 4e-6 * Sabs / (2 * h)
    assert abs(fd - an) <= 1e-3 * abs(an) + noise, (fd, an, noise)


def test_stop_on_sat_freezes_model():
    inst = cnfgen.planted_ksat(100, 426, 3, 0)
    prob, st, cnfs = make([inst], 64)
    hp = ts.hparams(seed=1, norm=ts.NORM_NONE, tau=2.0)
    ts.tsat_init(st.h, hp)
    ts.tsat_step(st.h, hp, 600, stop_on_sat=True)
    status = ts.tsat_status(st.h, 1)
    assert status["inst"][0]["found"] == 1
    i = status["inst"][0]["found_sample"]
    s = snapshot(st)
    u, _ = oracle.check(cnfs[0], s["X"][:, i:i + 1])
    assert u[0] == 0
    assert status["step"] == status["inst"][0]["found_step"]
    ts.tsat_step(st.h, hp, 5, stop_on_sat=True)
    s2 = snapshot(st)
    np.testing.assert_array_equal(s2["bits"], s["bits"])
    best = ts.tsat_best(st.h, hp, 0, inst.n_vars)
    assert best["complete"] and best["unsat"] == 0 and best["sample"] == i
    np.testing.assert_array_equal(best["assignment"], s["X"][:, i])


@pytest.mark.parametrize("N,k", [(64, None), (256, 37), (32, 1)])
def test_best_partial_assignment(N, k):
    inst = cnfgen.planted_ksat(2500, 10650, 3, 13)
    prob, st, cnfs = make([inst], N)
    hp = ts.hparams(seed=8, norm=1, tau=1.7)
    ts.tsat_init(st.h, hp)
    ts.tsat_step(st.h, hp, 7, stop_on_sat=False)
    s = snapshot(st)
    best = ts.tsat_best(st.h, hp, 0, inst.n_vars, k)
    kk = best["part_var"].shape[0]
    unsat, _ = oracle.check(cnfs[0], s["X"])
    i = oracle.best_sample(unsat)
    assert best["sample"] == i and best["unsat"] == unsat[i]
    np.testing.assert_array_equal(best["assignment"], s["X"][:, i])
    assert best["ready"] == ((cnfs[0].C - unsat[i]) / cnfs[0].C > 0.99)
    _, _, G, _ = oracle.objective(cnfs[0], X=s["X"][:, i:i + 1], tau=1.7)
    a = np.abs(G[:, 0])
    ref = oracle.topk_confident(a, kk)
    got = best["part_var"] - 1
    # unique part: the selection equals the oracle's up to FP32 near-ties at the cut
    kth = a[ref[-1]]
    assert np.all(a[got] <= kth * (1 + 1e-5) + 1e-12)
    assert len(set(got.tolist())) == kk
    assert np.all(np.diff(a[got]) >= -1e-5 * kth - 1e-12)
    np.testing.assert_array_equal(best["part_val"], s["X"][got, i])


def test_checkpoint_resume_is_bit_exact():
    inst = cnfgen.planted_ksat(800, 3400, 3, 17)
    prob, st, _ = make([inst], 128)
    hp = ts.hparams(seed=99, norm=1, binarize=1)
    ts.tsat_init(st.h, hp)
    ts.tsat_step(st.h, hp, 4, stop_on_sat=False)
    torch.cuda.synchronize()
    ckpt = st.buf.clone()
    ts.tsat_step(st.h, hp, 5, stop_on_sat=False)
    a = snapshot(st)
    st.buf.copy_(ckpt)
    ts.tsat_step(st.h, hp, 5, stop_on_sat=False)
    b = snapshot(st)
    for k in ("z", "m", "v", "nu", "bits"):
        np.testing.assert_array_equal(a[k], b[k])


def test_graph_replay_equals_single_steps():
    inst = cnfgen.planted_ksat(600, 2556, 3, 23)
    hp = ts.hparams(seed=5, norm=1, binarize=1)
    _, st1, _ = make([inst], 64)
    _, st2, _ = make([inst], 64)
    ts.tsat_init(st1.h, hp)
    ts.tsat_init(st2.h, hp)
    ts.tsat_step(st1.h, hp, 12, stop_on_sat=False)
    for _ in range(12):
        ts.tsat_step(st2.h, hp, 1, stop_on_sat=False)
    a, b = snapshot(st1), snapshot(st2)
    for k in ("z", "m", "v", "bits"):
        np.testing.assert_array_equal(a[k], b[k])


def test_autotune_keeps_results():
    inst = cnfgen.planted_ksat(5000, 21000, 3, 29)
    hp = ts.hparams(seed=5, norm=1)
    _, st1, _ = make([inst], 128)
    _, st2, _ = make([inst], 128)
    ts.tsat_init(st1.h, hp)
    tun = ts.tsat_autotune(st1.h, hp)
    assert tun[0] % 512 == 0 and tun[2] >= 1 and tun[3] >= 1
    ts.tsat_init(st2.h, hp)
    ts.tsat_step(st1.h, hp, 3, stop_on_sat=False)
    ts.tsat_step(st2.h, hp, 3, stop_on_sat=False)
    a, b = snapshot(st1), snapshot(st2)
    for k in ("z", "bits"):
        np.testing.assert_array_equal(a[k], b[k])


def _time_step(st, hp, saved, reps=3):
    """Device time of one tsat_step from the saved state buffer (min of reps)."""
    best = 1e30
    for _ in range(reps):
        st.buf.copy_(saved)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ts.tsat_step(st.h, hp, 1, stop_on_sat=False)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def test_autotune_times_the_step_update_and_leaves_the_state():
    """On a small batch of uneven k-SAT instances (k 3..7) past step 0, the
    tuned update shape is within 3 % of the fastest shape of an exhaustive
    tsat_set_tuning sweep of the same candidates, each timed on tsat_step
    itself; the call leaves the state bit for bit as it was, and a step with
    the tuned shape gives the same state as one with the default shape."""
    insts = cnfgen.batch_ksat(40, 77, n_lo=2000, n_hi=20000)
    hp = ts.hparams(seed=5, norm=1, binarize=1, tau=2.0, lr0=0.5)
    prob, st, _ = make(insts, 64)
    ts.tsat_init(st.h, hp)
    ts.tsat_step(st.h, hp, 3, stop_on_sat=False)
    torch.cuda.synchronize()
    before = st.buf.clone()
    tun = ts.tsat_autotune(st.h, hp)
    torch.cuda.synchronize()
    assert torch.equal(st.buf.view(torch.uint8)[:ts.tsat_autotune_bytes(st.h)],
                       before.view(torch.uint8)[:ts.tsat_autotune_bytes(st.h)])
    assert ts.tsat_status(st.h, len(insts))["step"] == 3
    space = ts.tsat_tuning_space(st.h)
    assert tun[2] in space["upd_blocks_per_sm"] and tun[3] in space["upd_rows_per_item"]
    times = {}
    for b in space["upd_blocks_per_sm"]:
        for r in space["upd_rows_per_item"]:
            ts.tsat_set_tuning(st.h, [tun[0], tun[1], b, r])
            ts.tsat_step_prepare(st.h, hp, 1, stop_on_sat=False)
            _time_step(st, hp, before, reps=1)            # warm-up
            times[(b, r)] = _time_step(st, hp, before)
    best = min(times.values())
    assert times[(tun[2], tun[3])] <= 1.03 * best, (tun, times)
    # the launch shape changes no result
    ts.tsat_set_tuning(st.h, tun)
    st.buf.copy_(before)
    ts.tsat_step(st.h, hp, 2, stop_on_sat=False)
    a = snapshot(st)
    ts.tsat_set_tuning(st.h, [tun[0], tun[1], 0, 1])
    st.buf.copy_(before)
    ts.tsat_step(st.h, hp, 2, stop_on_sat=False)
    b = snapshot(st)
    for k in ("z", "m", "v", "nu", "bits"):
        np.testing.assert_array_equal(a[k], b[k])


def test_step_graph_is_rebuilt_for_each_launch_shape():
    """The cached step graph has the forward's work-item count and the update
    grid baked in, so a new launch shape must give a new graph: forward items
    of 64 clauses, then of 16,448 (a shape whose item count once shared the
    64-clause shape's cache key byte), each step from the same saved state,
    equal a fresh state run with that shape, bit for bit, and the exact
    unsatisfied counts equal the oracle's."""
    inst = cnfgen.planted_ksat(100, 426, 3, 4)
    hp = ts.hparams(seed=9, norm=1, tau=2.0, lr0=0.5)
    prob, st, cnfs = make([inst], 64)
    ts.tsat_init(st.h, hp)
    before = st.buf.clone()
    tun = ts.tsat_get_tuning(st.h)
    outs = {}
    for items in (64, 16448):
        ts.tsat_set_tuning(st.h, [items, tun[1], tun[2], tun[3]])
        st.buf.copy_(before)
        ts.tsat_step(st.h, hp, 3, stop_on_sat=False)
        outs[items] = snapshot(st)
    for items in (64, 16448):
        prob2, st2, _ = make([inst], 64)
        ts.tsat_set_tuning(st2.h, [items, tun[1], tun[2], tun[3]])
        ts.tsat_init(st2.h, hp)
        ts.tsat_step(st2.h, hp, 3, stop_on_sat=False)
        fresh = snapshot(st2)
        for k in ("z", "m", "v", "nu", "bits"):
            np.testing.assert_array_equal(outs[items][k], fresh[k], err_msg=f"{k} items={items}")
        u, _ = oracle.check(cnfs[0], fresh["X"])
        unsat = torch.zeros(64, dtype=torch.int32, device="cuda")
        sm = torch.zeros(2, dtype=torch.int32, device="cuda")
        ts.tsat_evaluate(st2.h, hp, unsat, sm)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(unsat.cpu().numpy(), u)
