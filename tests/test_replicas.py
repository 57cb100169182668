"""The multi-GPU path is independent replicas: per-rank instances, a timing
barrier and max / sum reductions of per-rank scalars.  Checked here with two
gloo ranks on the CPU (127.0.0.1 rendezvous), plus the reference arm's rule
that only rank 0 works and prints."""
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

from paper_2511_07737_b300 import cnfgen
from paper_2511_07737_b300.replicas import Replicas, rank_env, replica_seed, whole_job_rate

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    r, w, lr = rank_env()
    rep = Replicas(w, backend="gloo")
    # per-rank instance (weak scaling) and per-rank "step time"
    inst = cnfgen.planted_ksat(50, 200, 3, replica_seed(7, r))
    ms = 10.0 + 5.0 * r
    rep.barrier()
    out[r] = (r, w, lr, rep.max(ms), rep.sum(float(inst.lits.size)), int(inst.lits[:8].sum()))
    rep.close()


def test_two_gloo_ranks_reduce_and_differ():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for r in (0, 1):
        rank, world, local, mx, sm, _ = res[r]
        assert (rank, world, local) == (r, 2, r)
        assert mx == 15.0                       # the slowest rank's time
        assert sm == 2 * 600.0                  # 200 clauses x 3 literals on each rank
    assert res[0][5] != res[1][5]               # the ranks solve different instances


def test_single_process_is_a_no_op():
    rep = Replicas(1)
    rep.barrier()
    assert rep.max(3.5) == 3.5 and rep.sum(2.0) == 2.0
    assert whole_job_rate(1e9, 10, 4, 20.0) == 1e9 * 10 * 4 / 0.02


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1")
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0
    assert p.stdout.strip() == ""
