"""Host side of the two multi-GPU splits, with two gloo ranks on the CPU
(127.0.0.1 rendezvous) and FP64 oracle engines in place of the GPU calls:
the instance split balances occurrences and its gathered results equal a
one-rank run; the sample split's two all-reduces per step (Eq. 5's row sums)
give the one-rank trajectory."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2511_07737_b300 import cnfgen
from paper_2511_07737_b300.sharding import (InstanceShards, LocalComm, SampleShards, TorchComm, balance_by_nnz,
                                            instance_nnz, merge_shard_status)
from tests.shard_engines import OracleBatchEngine, OracleShardEngine


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _hp(**kw):
    from paper_2511_07737_b300 import turbosat as ts
    return ts.hparams(**kw)


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_balance_by_nnz(world):
    rng = np.random.default_rng(world)
    nnz = list(rng.integers(10, 5000, size=53)) + [20000, 3]
    owned = balance_by_nnz(nnz, world)
    flat = sorted(j for o in owned for j in o)
    assert flat == list(range(len(nnz)))                      # every instance exactly once
    for o in owned:
        assert o == sorted(o)
    loads = [sum(nnz[j] for j in o) for o in owned]
    mean = sum(nnz) / world
    assert max(loads) - mean < max(nnz) or max(loads) == max(nnz)
    assert balance_by_nnz(nnz, world) == owned                 # deterministic


def test_merge_shard_status():
    a = [dict(found=0, found_sample=-1, found_step=-1, min_unsat=3, best_sample=5, loss=-1.5)]
    b = [dict(found=1, found_sample=2, found_step=7, min_unsat=3, best_sample=1, loss=-2.0)]
    m = merge_shard_status([a, b], 8)[0]
    assert m["min_unsat"] == 3 and m["best_sample"] == 5        # tie: the lower global sample (5 < 8 + 1)
    assert m["found"] and m["found_step"] == 7 and m["found_sample"] == 10
    assert m["loss"] == -3.5


def _batch():
    return [(i.n_vars, i.clause_ptr, i.lits) for i in cnfgen.batch_ksat(7, 31, n_lo=15, n_hi=60, k_hi=4)]


def _batch_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    hp = _hp(seed=77, norm=1, tau=2.0, lr0=0.5, binarize=1)
    sh = InstanceShards(_batch(), lambda insts, ids: OracleBatchEngine(insts, ids, 16), TorchComm())
    sh.init(hp)
    sh.step(hp, 6)
    out[rank] = (sh.owned, sh.gather())
    dist.destroy_process_group()


def test_instance_split_equals_one_rank():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_batch_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    insts = _batch()
    assert sorted(res[0][0] + res[1][0]) == list(range(len(insts)))
    assert res[0][1] == res[1][1]                               # every rank holds the whole gathered table
    one = InstanceShards(insts, lambda i, ids: OracleBatchEngine(i, ids, 16), LocalComm())
    hp = _hp(seed=77, norm=1, tau=2.0, lr0=0.5, binarize=1)
    one.init(hp)
    one.step(hp, 6)
    assert one.gather() == res[0][1]
    loads = [sum(instance_nnz([insts[j]])[0] for j in o) for o in (res[0][0], res[1][0])]
    assert abs(loads[0] - loads[1]) <= max(instance_nnz(insts))


def _inst():
    i = cnfgen.planted_ksat(40, 170, 3, 5)
    return (i.n_vars, i.clause_ptr, i.lits)


def _sample_worker(rank, world, port, kw, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    hp = _hp(seed=5, **kw)
    eng = OracleShardEngine(_inst(), 16, rank, world)
    sh = SampleShards(eng, TorchComm())
    sh.init(hp)
    sh.step(hp, 5)
    out[rank] = (eng.z.copy(), eng.m.copy(), eng.v.copy(), eng.X.copy(), eng.nu.copy(), sh.status())
    dist.destroy_process_group()


@pytest.mark.parametrize("kw", [dict(norm=0, binarize=1), dict(norm=1, binarize=0, tau=2.0),
                                dict(norm=2, binarize=1)], ids=["signed-philox", "absmean-det", "none-philox"])
def test_sample_split_equals_one_rank(kw):
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_sample_worker, args=(2, port, kw, out), nprocs=2, join=True)
        res = dict(out)
    hp = _hp(seed=5, **kw)
    eng = OracleShardEngine(_inst(), 16, 0, 1)
    one = SampleShards(eng, LocalComm())
    one.init(hp)
    one.step(hp, 5)
    z = np.concatenate([res[0][0], res[1][0]], axis=1)
    for k, ref in ((0, eng.z), (1, eng.m), (2, eng.v)):
        got = np.concatenate([res[0][k], res[1][k]], axis=1)
        assert np.max(np.abs(got - ref)) <= 1e-12 * max(np.max(np.abs(ref)), 1e-30)
    np.testing.assert_array_equal(np.concatenate([res[0][3], res[1][3]], axis=1), eng.X)
    np.testing.assert_allclose(res[0][4], eng.nu, rtol=1e-12)
    assert res[0][5] == res[1][5]
    a, b = res[0][5][0], one.status()[0]
    assert a["min_unsat"] == b["min_unsat"] and a["best_sample"] == b["best_sample"]
    assert abs(a["loss"] - b["loss"]) <= 1e-12 * abs(b["loss"])
    assert z.shape == eng.z.shape
