"""The two multi-GPU splits on one GPU, through the C ABI.

Instance split: an instance loaded in a sub-batch with its batch position as
stream id computes, bit for bit, what it computes inside the whole batch
(init, the multi-kernel steps and the persistent solver, Philox bits).

Sample split: two shards of one problem (samples [0, N/2) and [N/2, N)) as
two "ranks" of one process, whose all-reduces are sums over both shards
(host threads meet at a barrier; no kernel waits on another).  The init
equals the oracle's at the global sample indices, and every step is checked
against one oracle step from the shards' joined FP32 state: status, z / m / v
after AdamW, the new normaliser and the next bits."""
import threading

import numpy as np
import pytest
import torch

import oracle
from paper_2511_07737_b300 import cnfgen
from paper_2511_07737_b300 import turbosat as ts
from paper_2511_07737_b300.sharding import (CudaShardEngine, SampleShards, balance_by_nnz, instance_nnz,
                                            merge_shard_status)
from tests.gpu_util import TOL_F32, assert_adamw_z, binarize_like_gpu, lockstep, snapshot, stream_seed

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    torch.cuda.set_device(0)


def _descs(insts):
    return [(i.n_vars, i.clause_ptr, i.lits) for i in insts]


@pytest.mark.parametrize("name,gen,N,persistent", [
    ("k3..7", lambda: cnfgen.batch_ksat(9, 61, n_lo=60, n_hi=900), 64, False),
    ("3sat", lambda: [cnfgen.planted_ksat(300 + 50 * j, 1250 + 210 * j, 3, 70 + j) for j in range(7)], 128, False),
    ("3sat-persistent", lambda: [cnfgen.planted_ksat(100, 420, 3, 80 + j) for j in range(6)], 64, True),
])
def test_instance_split_matches_the_whole_batch(name, gen, N, persistent):
    insts = _descs(gen())
    hp = ts.hparams(seed=0x1234_0000_FFFF_FFFE, norm=1, binarize=1, bin_temp=0.5, tau=2.0, lr0=0.5)
    whole = ts.Problem(insts)
    sw = ts.State(whole, N)
    ts.tsat_init(sw.h, hp)
    step = ts.tsat_step_persistent if persistent else ts.tsat_step
    step(sw.h, hp, 5, stop_on_sat=False)
    W = snapshot(sw)
    offs = whole.var_offsets
    for owned in balance_by_nnz(instance_nnz(insts), 2):
        sub = ts.Problem([insts[j] for j in owned])
        ts.tsat_problem_set_instance_ids(sub.h, owned)
        ss = ts.State(sub, N)
        ts.tsat_init(ss.h, hp)
        step(ss.h, hp, 5, stop_on_sat=False)
        S = snapshot(ss)
        so = sub.var_offsets
        for k, j in enumerate(owned):
            for key in ("z", "m", "v", "nu", "bits"):
                np.testing.assert_array_equal(S[key][so[k]:so[k + 1]], W[key][offs[j]:offs[j + 1]],
                                              err_msg=f"{key} of instance {j}")
        st_sub = ts.tsat_status(ss.h, len(owned))["inst"]
        st_all = ts.tsat_status(sw.h, len(insts))["inst"]
        assert st_sub == [st_all[j] for j in owned]


class ThreadComm:
    """`world` host threads of one process as ranks: an all-reduce waits for
    every rank's tensor at a barrier, sums them on the device and hands each
    rank the sum.  Only host threads wait; no kernel waits on another."""

    def __init__(self, world):
        self.world = world
        self.bar = threading.Barrier(world, timeout=120)
        self.slots = [None] * world
        self.local = threading.local()

    def bind(self, rank):
        self.local.rank = rank
        return self

    @property
    def rank(self):
        return self.local.rank

    def allreduce_sum_(self, t):
        torch.cuda.synchronize()
        self.slots[self.rank] = t
        self.bar.wait()
        total = sum(x.clone() for x in self.slots)
        torch.cuda.synchronize()
        self.bar.wait()
        t.copy_(total)
        torch.cuda.synchronize()
        self.bar.wait()
        return t

    def all_gather_object(self, obj):
        self.slots[self.rank] = obj
        self.bar.wait()
        out = list(self.slots)
        self.bar.wait()
        return out


def _run_ranks(world, fn):
    errs = []

    def body(r):
        try:
            torch.cuda.set_device(0)
            fn(r)
        except BaseException as e:   # noqa: BLE001 - reported below
            errs.append(e)

    th = [threading.Thread(target=body, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    if errs:
        raise errs[0]


def _joined(engines):
    snaps = [snapshot(e.st) for e in engines]
    out = {k: np.concatenate([s[k] for s in snaps], axis=1) for k in ("z", "m", "v", "X")}
    out["nu"] = snaps[0]["nu"]
    for s in snaps[1:]:
        np.testing.assert_array_equal(s["nu"], out["nu"])   # every shard holds the same normaliser
    return out


@pytest.mark.parametrize("name,gen,N,kw", [
    ("3sat-N128-signed-philox", lambda: [cnfgen.planted_ksat(400, 1700, 3, 3)], 128, dict(norm=0, binarize=1)),
    ("3sat-N2048-absmean-det", lambda: [cnfgen.planted_ksat(200, 850, 3, 4)], 2048, dict(norm=1, binarize=0, tau=2.0)),
    ("k5-N64-none-philox", lambda: [cnfgen.planted_ksat(120, 1400, 5, 5)], 64, dict(norm=2, binarize=1)),
    ("batch-k3..7-N128-absmean-philox", lambda: cnfgen.batch_ksat(3, 9, n_lo=50, n_hi=300), 128,
     dict(norm=1, binarize=1, bin_temp=0.5)),
])
def test_sample_split_lockstep(name, gen, N, kw):
    insts = gen()
    hp = ts.hparams(seed=19, **kw)
    world = 2
    comm = ThreadComm(world)
    engines = [None] * world
    shards = [None] * world

    def setup(r):
        engines[r] = CudaShardEngine(_descs(insts), N, r, world)
        shards[r] = SampleShards(engines[r], comm.bind(r))
        shards[r].init(hp)

    _run_ranks(world, setup)
    cnfs = [oracle.CNF(i.n_vars, i.clause_ptr, i.lits) for i in insts]
    offs = engines[0].prob.var_offsets
    s = _joined(engines)
    # init: the oracle's Irwin-Hall draws at the global sample indices, per instance stream
    for j in range(len(insts)):
        a, b = offs[j], offs[j + 1]
        np.testing.assert_array_equal(s["z"][a:b], oracle.init_normal(b - a, N, stream_seed(hp.seed, j)))
    nu_ref = oracle.nu_f32(s["z"], hp.norm)
    assert np.all(np.abs(s["nu"] - nu_ref) <= 2e-6 * np.abs(s["z"]).mean(axis=1) + 2e-6 * np.abs(nu_ref))
    np.testing.assert_array_equal(s["X"], binarize_like_gpu(s["z"], s["nu"], hp, 0, offs))
    for t in range(4):
        s0 = _joined(engines)
        _run_ranks(world, lambda r: (comm.bind(r), shards[r].step(hp))[1])
        s1 = _joined(engines)
        z, m, v, res = lockstep(cnfs, offs, hp, t, s0)
        merged = merge_shard_status([e.status() for e in engines], N // world)
        frozen = np.zeros(s1["z"].shape[0], bool)
        for j, r in enumerate(res):
            assert merged[j]["min_unsat"] == int(r["unsat"].min())
            assert merged[j]["best_sample"] == oracle.best_sample(r["unsat"])
            assert abs(merged[j]["loss"] - r["L"]) <= TOL_F32 * abs(r["L"])
            if merged[j]["found"]:
                frozen[offs[j]:offs[j + 1]] = True
        live = ~frozen
        if live.any():
            assert_adamw_z(s1["z"][live], z[live], s1["m"][live], m[live], s1["v"][live], v[live], t, hp)
        X = binarize_like_gpu(s1["z"], s1["nu"], hp, t + 1, offs)
        np.testing.assert_array_equal(s1["X"][live], X[live])
        nu_ref = oracle.nu_f32(s1["z"], hp.norm)
        assert np.all(np.abs(s1["nu"] - nu_ref) <= 2e-6 * np.abs(s1["z"]).mean(axis=1) + 2e-6 * np.abs(nu_ref))


def test_shard_states_refuse_the_whole_sample_calls():
    inst = cnfgen.planted_ksat(100, 420, 3, 1)
    eng = CudaShardEngine(_descs([inst]), 128, 1, 2)
    hp = ts.hparams(seed=1)
    for call in (lambda: ts.tsat_init(eng.st.h, hp), lambda: ts.tsat_step(eng.st.h, hp, 1),
                 lambda: ts.tsat_step_persistent(eng.st.h, hp, 1)):
        with pytest.raises(ts.TsatError) as e:
            call()
        assert e.value.status == -9
    with pytest.raises(ts.TsatError):
        ts.tsat_state_set_shard(eng.st.h, 32, 128)      # not a multiple of the shard size
    with pytest.raises(ts.TsatError):
        ts.tsat_shard_init(eng.st.h, ts.hparams(seed=1, mix_restart=1), eng.rowsum)
