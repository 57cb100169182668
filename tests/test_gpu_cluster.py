"""Cluster-persistent solver (tsat_step_clustered: instances dealt to
thread-block clusters, every warp of a cluster on one instance, many steps per
launch) against the FP64 oracle one step at a time, and bit for bit against
the multi-kernel step (same integer histograms, same row-group update code);
its stop semantics; and tsat_step_persistent taking it for instances too large
for one block."""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_07737_b300 import cnfgen
from paper_2511_07737_b300 import turbosat as ts
from tests.gpu_util import TOL_F32, assert_adamw_z, binarize_like_gpu, lockstep, make, snapshot

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    torch.cuda.set_device(0)


def _batch(seed, n_inst=6, n_lo=300, n_hi=6000):
    # k 3..7 mixed; at least one 7-SAT instance so the longest clause is 7
    insts = cnfgen.batch_ksat(n_inst, seed, n_lo=n_lo, n_hi=n_hi)
    return insts + [cnfgen.planted_ksat(400, 25000, 7, seed + 99)]


@pytest.mark.parametrize("N,kw", [(64, dict(norm=1, binarize=0, tau=2.0)), (32, dict(norm=0, binarize=1)),
                                  (128, dict(norm=2, binarize=1, bin_temp=0.5))],
                         ids=["N64-absmean-det", "N32-signed-philox", "N128-none-philox"])
def test_cluster_lockstep_and_equal_to_the_step_graph(N, kw):
    insts = _batch(11)
    hp = ts.hparams(seed=41, **kw)
    prob, st, cnfs = make(insts, N)
    st2 = ts.State(prob, N)
    ts.tsat_init(st.h, hp)
    ts.tsat_init(st2.h, hp)
    offs = prob.var_offsets
    for t in range(3):
        s0 = snapshot(st)
        ts.tsat_step_clustered(st.h, hp, 1, stop_on_sat=False)
        ts.tsat_step(st2.h, hp, 1, stop_on_sat=False)
        s1, g1 = snapshot(st), snapshot(st2)
        for key in ("z", "m", "v", "nu", "bits"):
            np.testing.assert_array_equal(s1[key].view(np.uint32), g1[key].view(np.uint32), err_msg=key)
        z, m, v, res = lockstep(cnfs, offs, hp, t, s0)
        status = ts.tsat_status(st.h, len(insts))
        frozen = np.zeros(prob.info["n_vars"], bool)
        for j, r in enumerate(res):
            x = status["inst"][j]
            if x["found"]:
                frozen[offs[j]:offs[j + 1]] = True
                if x["found_step"] < t:
                    continue
            assert x["min_unsat"] == int(r["unsat"].min())
            assert x["best_sample"] == oracle.best_sample(r["unsat"])
            assert abs(x["loss"] - r["L"]) <= TOL_F32 * abs(r["L"])
        live = ~frozen
        if live.any():
            assert_adamw_z(s1["z"][live], z[live], s1["m"][live], m[live], s1["v"][live], v[live], t, hp)
        X = binarize_like_gpu(s1["z"], s1["nu"], hp, t + 1, offs)
        np.testing.assert_array_equal(s1["X"][live], X[live])
        assert status["step"] == t + 1


@pytest.mark.parametrize("k", [7, 300])
def test_cluster_k_steps_equal_k_single_steps_and_the_graph(k):
    insts = _batch(23, n_inst=9, n_lo=200, n_hi=3000)
    hp = ts.hparams(seed=5, norm=1, binarize=1, tau=2.0, lr0=0.5)
    prob, a, _ = make(insts, 64)
    b, c = ts.State(prob, 64), ts.State(prob, 64)
    for st in (a, b, c):
        ts.tsat_init(st.h, hp)
    ts.tsat_step_clustered(a.h, hp, k, stop_on_sat=False)
    for _ in range(k):
        ts.tsat_step_clustered(b.h, hp, 1, stop_on_sat=False)
    ts.tsat_step(c.h, hp, k, stop_on_sat=False)
    sa, sb, sc = snapshot(a), snapshot(b), snapshot(c)
    for key in ("z", "m", "v", "nu", "bits"):
        np.testing.assert_array_equal(sa[key].view(np.uint32), sb[key].view(np.uint32), err_msg=key)
        np.testing.assert_array_equal(sa[key].view(np.uint32), sc[key].view(np.uint32), err_msg=key)
    ta, tb, tc = (ts.tsat_status(x.h, len(insts)) for x in (a, b, c))
    assert ta["step"] == tb["step"] == tc["step"] == k
    for x, y, z in zip(ta["inst"], tb["inst"], tc["inst"]):
        assert x == y
        for f in ("found", "found_sample", "found_step", "min_unsat", "best_sample"):
            assert x[f] == z[f]
        assert abs(x["loss"] - z["loss"]) <= 1e-5 * abs(z["loss"])


def test_cluster_solves_stops_and_is_taken_by_the_persistent_call():
    # 4-SAT at 0.35 of the threshold solves quickly; an instance of 20,000
    # variables does not fit one block, so tsat_step_persistent takes clusters
    insts = [cnfgen.planted_ksat(20000, 70000, 4, 3)] + [cnfgen.planted_ksat(800, 2800, 4, 10 + j) for j in range(5)]
    hp = ts.hparams(seed=3, norm=1, tau=2.0, lr0=0.5)
    prob, st, cnfs = make(insts, 64)
    ts.tsat_init(st.h, hp)
    ts.tsat_step_persistent(st.h, hp, 400, stop_on_sat=True)
    status = ts.tsat_status(st.h, len(insts))
    X = snapshot(st)["X"]
    offs = prob.var_offsets
    solved = 0
    for j, x in enumerate(status["inst"]):
        if x["found"]:
            solved += 1
            u, _ = oracle.check(cnfs[j], X[offs[j]:offs[j + 1]])
            assert u[x["found_sample"]] == 0 and x["min_unsat"] == 0
    assert solved >= 3
    if status["all_done"]:
        assert status["step"] == max(x["found_step"] for x in status["inst"])
        before = snapshot(st)
        ts.tsat_step_clustered(st.h, hp, 20, stop_on_sat=True)
        np.testing.assert_array_equal(before["z"], snapshot(st)["z"])
    else:
        assert status["step"] == 400


def test_cluster_rejects_what_it_does_not_run():
    short = [cnfgen.planted_ksat(300, 1200, 3, 1)]
    _, st, _ = make(short, 64)
    hp = ts.hparams(seed=1)
    ts.tsat_init(st.h, hp)
    with pytest.raises(ts.TsatError):
        ts.tsat_step_clustered(st.h, hp, 1)                 # clause length <= 3
    _, st2, _ = make(_batch(3, n_inst=2), 256)
    ts.tsat_init(st2.h, hp)
    with pytest.raises(ts.TsatError):
        ts.tsat_step_clustered(st2.h, hp, 1)                # N > 128
    _, st3, _ = make(_batch(4, n_inst=2), 64)
    ts.tsat_init(st3.h, hp)
    with pytest.raises(ts.TsatError):
        ts.tsat_step_clustered(st3.h, ts.hparams(seed=1, mix_restart=1), 1)
