"""Persistent solver (tsat_step_persistent: one block per instance, many steps
per launch) against the FP64 oracle, one step at a time from the GPU's FP32
state, and its stopping semantics against the multi-kernel path."""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_07737_b300 import cnfgen
from paper_2511_07737_b300 import turbosat as ts
from tests.gpu_util import TOL_F32, assert_adamw_z, binarize_like_gpu, lockstep, make, snapshot, unpack_bits

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    torch.cuda.set_device(0)


CASES = [
    ("3sat-N64", lambda: [cnfgen.planted_ksat(100, 426, 3, 0)], 64, dict(norm=0, binarize=0)),
    ("3sat-N64-philox", lambda: [cnfgen.planted_ksat(100, 426, 3, 1)], 64, dict(norm=1, binarize=1, bin_temp=0.5)),
    ("3sat-N32-none", lambda: [cnfgen.planted_ksat(700, 2982, 3, 6)], 32, dict(norm=2, binarize=1)),
    ("3sat-N1024", lambda: [cnfgen.planted_ksat(300, 1278, 3, 5)], 1024, dict(norm=1, binarize=1)),
    ("k7-N128", lambda: [cnfgen.planted_ksat(300, 9000, 7, 8)], 128, dict(norm=0, binarize=0)),
    ("short-dup-N256", lambda: [cnfgen.tiny_random(200, 1500, 9, kmin=1, kmax=5)], 256, dict(norm=1, binarize=1)),
    ("batch-k3..7-N64", lambda: cnfgen.batch_ksat(9, 10, n_lo=40, n_hi=600), 64, dict(norm=1, binarize=1)),
    # clause pointers and literals (clauses longer than 3) with two sample words
    # per forward task: resident at N = 64 (16 samples per thread) and at N = 1024
    ("k5-N64-resident", lambda: [cnfgen.planted_ksat(60, 400, 5, 12)], 64, dict(norm=1, binarize=1)),
    ("short-dup-N64-resident", lambda: [cnfgen.tiny_random(50, 300, 14, kmin=1, kmax=5)], 64, dict(norm=0, binarize=0)),
    ("k5-N1024", lambda: [cnfgen.planted_ksat(60, 1200, 5, 13)], 1024, dict(norm=2, binarize=1)),
]


# one block per instance, and (N <= 256) a cluster of 4 blocks per instance
LOCK_CASES = [c + (b,) for c in CASES for b in ([1, 4] if c[2] <= 256 else [1])]


@pytest.mark.parametrize("name,gen,N,kw,blocks", LOCK_CASES, ids=[f"{c[0]}-x{c[4]}" for c in LOCK_CASES])
def test_persistent_lockstep(name, gen, N, kw, blocks):
    _persistent_lockstep(gen(), N, kw, blocks, 4)


def _persistent_lockstep(insts, N, kw, blocks, steps):
    """steps single-step launches (the third one on the multi-kernel path),
    each checked against one oracle step from the GPU's FP32 state."""
    prob, st, cnfs = make(insts, N)
    ts.tsat_set_persist_blocks(st.h, blocks)
    hp = ts.hparams(**{"seed": 33, "tau": 1.3, **kw})
    ts.tsat_init(st.h, hp)
    offs = prob.var_offsets
    for t in range(steps):
        s0 = snapshot(st)
        # alternate the persistent launch with the multi-kernel step: both leave the same state layout
        if t == 2:
            ts.tsat_step(st.h, hp, 1, stop_on_sat=False)
        else:
            ts.tsat_step_persistent(st.h, hp, 1, stop_on_sat=False)
        s1 = snapshot(st)
        z, m, v, res = lockstep(cnfs, offs, hp, t, s0)
        status = ts.tsat_status(st.h, len(insts))
        frozen = np.zeros(prob.info["n_vars"], bool)
        for j, r in enumerate(res):
            if status["inst"][j]["found"]:
                frozen[offs[j]:offs[j + 1]] = True
            if status["inst"][j]["found"] and status["inst"][j]["found_step"] < t:
                continue
            assert status["inst"][j]["min_unsat"] == int(r["unsat"].min())
            assert status["inst"][j]["best_sample"] == oracle.best_sample(r["unsat"])
            assert abs(status["inst"][j]["loss"] - r["L"]) <= TOL_F32 * abs(r["L"])
        live = ~frozen
        if live.any():
            assert_adamw_z(s1["z"][live], z[live], s1["m"][live], m[live], s1["v"][live], v[live], t, hp)
        X = binarize_like_gpu(s1["z"], s1["nu"], hp, t + 1, offs)
        np.testing.assert_array_equal(s1["X"][live], X[live])
        np.testing.assert_array_equal(s1["X"][frozen], s0["X"][frozen])
        nu_ref = oracle.nu_f32(s1["z"], hp.norm)
        assert np.all(np.abs(s1["nu"] - nu_ref) <= 2e-6 * np.abs(s1["z"]).mean(axis=1) + 2e-6 * np.abs(nu_ref))
        assert status["step"] == t + 1


def test_persistent_solves_and_stops_like_the_graph_path():
    """A batch solved to the end: every instance frozen on a model of its own
    formula, the step counter at the step that froze the last one, no further
    work once stopped; the same launch with stop_on_sat off keeps counting."""
    insts = [cnfgen.planted_ksat(100, 400, 3, j) for j in range(12)]
    prob, st, cnfs = make(insts, 64)
    hp = ts.hparams(seed=3, norm=ts.NORM_ABSMEAN, tau=2.0, lr0=0.5)
    ts.tsat_init(st.h, hp)
    ts.tsat_step_persistent(st.h, hp, 600, stop_on_sat=True)
    status = ts.tsat_status(st.h, len(insts))
    found = [x["found"] for x in status["inst"]]
    assert sum(found) >= 9
    X = snapshot(st)["X"]
    offs = prob.var_offsets
    for j, x in enumerate(status["inst"]):
        if x["found"]:
            u, _ = oracle.check(cnfs[j], X[offs[j]:offs[j + 1]])
            assert u[x["found_sample"]] == 0 and x["min_unsat"] == 0
    if all(found):
        assert status["all_done"]
        assert status["step"] == max(x["found_step"] for x in status["inst"])
        before = snapshot(st)
        ts.tsat_step_persistent(st.h, hp, 50, stop_on_sat=True)   # stopped: nothing changes
        after = snapshot(st)
        assert ts.tsat_status(st.h, len(insts))["step"] == status["step"]
        np.testing.assert_array_equal(before["z"], after["z"])
    else:
        assert status["step"] == 600 and not status["all_done"]
    # without the stop the counter advances by the launch's steps
    st2 = ts.State(prob, 64)
    ts.tsat_init(st2.h, hp)
    ts.tsat_step_persistent(st2.h, hp, 37, stop_on_sat=False)
    ts.tsat_step_persistent(st2.h, hp, 5, stop_on_sat=False)
    assert ts.tsat_status(st2.h, len(insts))["step"] == 42


def test_persistent_rejects_what_it_does_not_run():
    inst = cnfgen.planted_ksat(100, 426, 3, 0)
    prob, st, _ = make([inst], 64)
    hp = ts.hparams(seed=1)
    ts.tsat_init(st.h, hp)
    with pytest.raises(ts.TsatError) as e:
        ts.tsat_step_persistent(st.h, ts.hparams(seed=1, mix_restart=1), 1)
    assert e.value.status == -1
    long = cnfgen.planted_ksat(60, 200, 9, 2)
    prob2, st2, _ = make([long], 64)
    ts.tsat_init(st2.h, hp)
    with pytest.raises(ts.TsatError):
        ts.tsat_step_persistent(st2.h, hp, 1)
    rel = ts.State(prob, 64, ts.LAYER_RELAXED)
    hr = ts.hparams(seed=1, layer=ts.LAYER_RELAXED)
    ts.tsat_init(rel.h, hr)
    with pytest.raises(ts.TsatError):
        ts.tsat_step_persistent(rel.h, hr, 1)


KSTEP_CASES = [
    # resident: z, m, v and nu stay in shared memory for the whole launch
    ("resident-3sat-n100-N64", lambda: [cnfgen.planted_ksat(100, 426, 3, 0)], 64,
     dict(norm=1, binarize=0, tau=2.0, lr0=0.5)),
    ("resident-batch-k3..5-N64-philox", lambda: cnfgen.batch_ksat(6, 40, n_lo=40, n_hi=150, ks=[3, 4, 5]), 64,
     dict(norm=0, binarize=1, bin_temp=0.5)),
    # not resident: z, m, v and nu read and written in global memory every step
    ("global-3sat-n1000-N64", lambda: [cnfgen.planted_ksat(1000, 4000, 3, 2)], 64,
     dict(norm=1, binarize=0, tau=2.0, lr0=0.5)),
    ("global-k5-n60-N1024-philox", lambda: [cnfgen.planted_ksat(60, 1200, 5, 13)], 1024,
     dict(norm=2, binarize=1)),
]


@pytest.mark.parametrize("k", [7, 300])
@pytest.mark.parametrize("name,gen,N,kw", KSTEP_CASES, ids=[c[0] for c in KSTEP_CASES])
def test_persistent_k_steps_equal_k_single_step_launches(name, gen, N, kw, k):
    """One launch of k steps leaves the state bit for bit as k launches of one
    step: the carried shared-memory state and its write-back, the step scalars
    formed 256 steps at a time (k = 300 crosses that batch), the bits ping-pong
    inside a launch, and the freezing of solved instances (found step, sample)."""
    insts = gen()
    hp = ts.hparams(seed=21, **kw)
    prob, st_a, _ = make(insts, N)
    st_b = ts.State(prob, N)
    for st in (st_a, st_b):
        ts.tsat_init(st.h, hp)
    ts.tsat_step_persistent(st_a.h, hp, k, stop_on_sat=False)
    for _ in range(k):
        ts.tsat_step_persistent(st_b.h, hp, 1, stop_on_sat=False)
    a, b = snapshot(st_a), snapshot(st_b)
    for key in ("z", "m", "v", "nu", "bits"):
        np.testing.assert_array_equal(a[key].view(np.uint32), b[key].view(np.uint32), err_msg=key)
    sa, sb = ts.tsat_status(st_a.h, len(insts)), ts.tsat_status(st_b.h, len(insts))
    assert sa["step"] == sb["step"] == k
    assert sa["inst"] == sb["inst"]
    if name.startswith("resident-3sat") and k == 300:
        assert sa["inst"][0]["found"]        # the freezing path ran inside the long launch


def test_persistent_launches_from_two_host_threads():
    """Two host threads, each with its own problem and state, launch the
    persistent solver at the same time (the kernels' launch settings are
    library state shared by the threads): each thread's z, m, v and bits equal
    those of the same launches run alone, bit for bit."""
    import threading
    insts = [cnfgen.planted_ksat(100, 426, 3, 40 + j) for j in range(2)]
    hp = ts.hparams(seed=3, norm=1, tau=2.0, lr0=0.5)

    def run(inst):
        prob, st, _ = make([inst], 64)
        ts.tsat_init(st.h, hp)
        for _ in range(4):
            ts.tsat_step_persistent(st.h, hp, 30, stop_on_sat=False)
        torch.cuda.synchronize()
        return snapshot(st)

    alone = [run(i) for i in insts]
    out = [None, None]
    errs = []

    def worker(j):
        try:
            out[j] = run(insts[j])
        except Exception as e:          # reported by the main thread
            errs.append(e)

    th = [threading.Thread(target=worker, args=(j,)) for j in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errs, errs
    for a, b in zip(alone, out):
        for key in ("z", "m", "v", "bits"):
            np.testing.assert_array_equal(a[key], b[key])


SPLIT_CASES = [
    # resident with every block count; solved inside the 300-step launch
    ("3sat-n100-N64", lambda: [cnfgen.planted_ksat(100, 426, 3, 0)], 64, dict(norm=1, binarize=0, tau=2.0, lr0=0.5)),
    # a batch: one cluster per instance, Philox bits, clause lengths 3..5
    ("batch-k3..5-N64-philox", lambda: cnfgen.batch_ksat(6, 40, n_lo=40, n_hi=150, ks=[3, 4, 5]), 64,
     dict(norm=0, binarize=1, bin_temp=0.5)),
    # global z, m, v with one block, resident in the blocks of a cluster of 8
    ("3sat-n1000-N64", lambda: [cnfgen.planted_ksat(1000, 4000, 3, 2)], 64, dict(norm=1, binarize=0, tau=2.0, lr0=0.5)),
    # clause pointers and literals (length 5), no normalisation, N = 256
    ("k5-n200-N256-philox", lambda: [cnfgen.planted_ksat(200, 3000, 5, 13)], 256, dict(norm=2, binarize=1)),
    # N = 32, duplicated literals and short clauses, signed mean
    ("short-dup-n300-N32", lambda: [cnfgen.tiny_random(300, 2000, 9, kmin=1, kmax=5)], 32, dict(norm=0, binarize=1)),
]


@pytest.mark.parametrize("k", [7, 300])
@pytest.mark.parametrize("blocks", [2, 4, 8])
@pytest.mark.parametrize("name,gen,N,kw", SPLIT_CASES, ids=[c[0] for c in SPLIT_CASES])
def test_persistent_cluster_of_blocks_equals_one_block(name, gen, N, kw, blocks, k):
    """An instance split over a cluster of 2, 4 or 8 blocks (clauses and rows
    dealt to the blocks, histograms summed over distributed shared memory)
    leaves z, m, v, the normaliser, both bits buffers and the status records
    bit for bit as one block per instance, over a launch of k steps (k = 300
    crosses the 256-step batch of step scalars and, for the first case, the
    freezing of the solved instance inside the launch)."""
    insts = gen()
    hp = ts.hparams(seed=21, **kw)
    prob, st_a, _ = make(insts, N)
    st_b = ts.State(prob, N)
    ts.tsat_set_persist_blocks(st_a.h, 1)
    ts.tsat_set_persist_blocks(st_b.h, blocks)
    (ba, ra), (bb, rb) = ts.tsat_persist_blocks(st_a.h, True), ts.tsat_persist_blocks(st_b.h, True)
    assert ba == 1 and bb == blocks
    if ra != rb:
        # z, m, v in shared memory with the cluster but global with one block
        # (another number of samples per thread, so the Eq. 5 row sums round
        # in another order): the split layout against the oracle instead
        assert rb and not ra
        if k == 7:
            _persistent_lockstep(insts, N, kw, blocks, 3)
        return
    for st in (st_a, st_b):
        ts.tsat_init(st.h, hp)
        ts.tsat_step_persistent(st.h, hp, k, stop_on_sat=False)
    a, b = snapshot(st_a), snapshot(st_b)
    for key in ("z", "m", "v", "nu", "bits"):
        np.testing.assert_array_equal(a[key].view(np.uint32), b[key].view(np.uint32), err_msg=key)
    sa, sb = ts.tsat_status(st_a.h, len(insts)), ts.tsat_status(st_b.h, len(insts))
    assert sa["step"] == sb["step"] == k
    assert sa["inst"] == sb["inst"]
    if name == "3sat-n100-N64" and k == 300:
        assert sa["inst"][0]["found"]
    # and a continuation launch of the split state with stop_on_sat: the same
    # stop as one block
    for st in (st_a, st_b):
        ts.tsat_step_persistent(st.h, hp, 20, stop_on_sat=True)
    a, b = snapshot(st_a), snapshot(st_b)
    for key in ("z", "bits"):
        np.testing.assert_array_equal(a[key].view(np.uint32), b[key].view(np.uint32), err_msg=key)
    assert ts.tsat_status(st_a.h, len(insts)) == ts.tsat_status(st_b.h, len(insts))


@pytest.mark.parametrize("name,gen,N", [
    # fewer rows than blocks: some blocks of the cluster own no row and no forward task
    ("tiny-n6-x8", lambda: [cnfgen.tiny_random(6, 20, 3, kmin=1, kmax=3)], 64),
    # more clusters than fit on the device at once (40 x 8 blocks): they run in waves
    ("waves-40x-n60-x8", lambda: [cnfgen.planted_ksat(60, 250, 3, 70 + j) for j in range(40)], 32),
    # instances of different sizes in one launch, one cluster each
    ("mixed-sizes-x8", lambda: cnfgen.batch_ksat(5, 77, n_lo=10, n_hi=400, ks=[3, 4]), 32),
])
def test_persistent_cluster_edge_cases_equal_one_block(name, gen, N):
    insts = gen()
    hp = ts.hparams(seed=5, norm=1, binarize=1, bin_temp=0.5)
    prob, st_a, _ = make(insts, N)
    st_b = ts.State(prob, N)
    ts.tsat_set_persist_blocks(st_a.h, 1)
    ts.tsat_set_persist_blocks(st_b.h, 8)
    assert ts.tsat_persist_blocks(st_a.h, True)[1] == ts.tsat_persist_blocks(st_b.h, True)[1]
    for st in (st_a, st_b):
        ts.tsat_init(st.h, hp)
        ts.tsat_step_persistent(st.h, hp, 40, stop_on_sat=True)
    a, b = snapshot(st_a), snapshot(st_b)
    for key in ("z", "m", "v", "nu", "bits"):
        np.testing.assert_array_equal(a[key].view(np.uint32), b[key].view(np.uint32), err_msg=key)
    assert ts.tsat_status(st_a.h, len(insts)) == ts.tsat_status(st_b.h, len(insts))


def _auto_blocks(n_inst):
    """The automatic choice for instances one block cannot keep resident."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cs = 1
    while cs < 8 and n_inst * cs * 2 <= sms:
        cs *= 2
    return cs


def test_persist_blocks_setting_is_checked():
    inst = cnfgen.planted_ksat(100, 426, 3, 0)
    prob, st, _ = make([inst], 64)
    assert ts.tsat_persist_blocks(st.h, True) == (1, True)    # resident in one block: one block
    mid = cnfgen.planted_ksat(1000, 4260, 3, 0)
    prob1, st1, _ = make([mid], 64)
    assert ts.tsat_persist_blocks(st1.h, True) == (_auto_blocks(1), True) == (8, True)   # resident from 8 blocks
    for bad in (3, 16, -1):
        with pytest.raises(ts.TsatError) as e:
            ts.tsat_set_persist_blocks(st.h, bad)
        assert e.value.status == -1
    big = ts.State(prob, 1024)
    assert ts.tsat_persist_blocks(big.h) == 1         # N > 256: one block per instance
    with pytest.raises(ts.TsatError):
        ts.tsat_set_persist_blocks(big.h, 2)
    batch = [cnfgen.planted_ksat(1000, 4260, 3, j) for j in range(40)]
    prob2, st2, _ = make(batch, 64)
    assert ts.tsat_persist_blocks(st2.h) == _auto_blocks(40)   # 2 on 148 SMs: 40 x 4 blocks would not fit


def test_autotune_persistent_keeps_the_state_and_picks_the_cluster_where_it_pays():
    """The persistent autotuner times each candidate number of blocks per
    instance from the saved state, puts the state back, and keeps the fastest:
    at n = 1,000 (N = 64) an instance is resident only on a cluster of 8 blocks,
    which takes about a tenth of one block's step time; at n = 100 (resident in
    every shape) any shape it keeps steps bit for bit like the others."""
    hp = ts.hparams(seed=2, norm=1, tau=2.0, lr0=0.5)
    for n, m, expect in ((1000, 4000, 8), (100, 426, None)):
        inst = cnfgen.planted_ksat(n, m, 3, 0)
        prob, st, _ = make([inst], 64)
        ts.tsat_init(st.h, hp)
        ts.tsat_step_persistent(st.h, hp, 3, stop_on_sat=False)
        torch.cuda.synchronize()
        nb = ts.tsat_autotune_bytes(st.h)
        before = st.buf.view(torch.uint8)[:nb].clone()
        b = ts.tsat_autotune_persistent(st.h, hp, 40)
        assert b in (1, 2, 4, 8) and ts.tsat_persist_blocks(st.h) == b
        assert torch.equal(st.buf.view(torch.uint8)[:nb], before)
        if expect is not None:
            assert b == expect
        # the tuned shape steps like any other: continuing gives the one-block result
        st_b = ts.State(prob, 64)
        ts.tsat_set_persist_blocks(st_b.h, b)
        ts.tsat_init(st_b.h, hp)
        ts.tsat_step_persistent(st_b.h, hp, 3, stop_on_sat=False)
        ts.tsat_step_persistent(st.h, hp, 5, stop_on_sat=False)
        ts.tsat_step_persistent(st_b.h, hp, 5, stop_on_sat=False)
        a, c = snapshot(st), snapshot(st_b)
        if ts.tsat_persist_blocks(st.h, True)[1] == ts.tsat_persist_blocks(st_b.h, True)[1]:
            np.testing.assert_array_equal(a["bits"], c["bits"])


@pytest.mark.gpu
def test_autotune_persistent_failure_keeps_setting_and_state():
    """When no candidate runs the batch (N = 512 allows one block only, and an
    n = 3,000 instance's bits do not fit its shared memory), the tuner reports
    TSAT_ERANGE, keeps the caller's blocks-per-instance setting and leaves the
    state as it was; the refusal is decided on the host before any launch."""
    hp = ts.hparams(seed=4, norm=1, tau=2.0, lr0=0.5)
    inst = cnfgen.planted_ksat(3000, 12000, 3, 1)
    prob, st, _ = make([inst], 512)
    ts.tsat_init(st.h, hp)
    ts.tsat_step(st.h, hp, 2, stop_on_sat=False)
    ts.tsat_set_persist_blocks(st.h, 1)
    torch.cuda.synchronize()
    nb = ts.tsat_autotune_bytes(st.h)
    before = st.buf.view(torch.uint8)[:nb].clone()
    with pytest.raises(ts.TsatError) as e:
        ts.tsat_autotune_persistent(st.h, hp, 10)
    assert e.value.status == -10
    assert ts.tsat_persist_blocks(st.h) == 1
    torch.cuda.synchronize()
    assert torch.equal(st.buf.view(torch.uint8)[:nb], before)
    # the state still steps on the graph path
    ts.tsat_step(st.h, hp, 1, stop_on_sat=False)
    assert ts.tsat_status(st.h, 1)["inst"][0]["min_unsat"] >= 0
