"""Host side of the multi-GPU splits: one process per GPU.

Two ways to split the work of the method over ranks (the paper ran on up to
two GPUs, Sec. V, without saying how):

* ``InstanceShards`` -- the instances of a batch are independent, so each
  rank loads and solves a subset of them, chosen so that the ranks hold about
  the same number of literal occurrences (``balance_by_nnz``).  Nothing is
  exchanged on the data path; the per-instance results are gathered at the
  end.  Each instance keeps its position in the whole batch as its random
  stream id (``tsat_problem_set_instance_ids``), so a rank computes exactly
  what a one-rank run computes for that instance.
* ``SampleShards`` -- one problem's N samples split evenly over the ranks.
  Every part of a step but Eq. 5 reads one sample column; Eq. 5 needs two
  row sums over all N samples per step, sum_i G_vi z_vi and sum_i z_vi (or
  |z_vi|), all-reduced between the library's three shard calls.

Both take a communicator with ``rank``, ``world``, ``allreduce_sum_(tensor)``
and ``all_gather_object(obj)``: ``TorchComm`` wraps torch.distributed (NCCL
between GPUs, gloo on CPUs); ``LocalComm`` is the one-process case.  The work
itself goes through an engine (``CudaBatchEngine`` / ``CudaShardEngine``,
which call the C ABI), so the orchestration here is plain host code.
"""
from __future__ import annotations

import numpy as np


# ---------------------------------------------------------------- communicators
class LocalComm:
    """One process: reductions are the identity."""
    rank, world = 0, 1

    def allreduce_sum_(self, t):
        return t

    def all_gather_object(self, obj):
        return [obj]


class TorchComm:
    """torch.distributed process group (NCCL for device tensors, gloo for CPU)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def allreduce_sum_(self, t):
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)
        return t

    def all_gather_object(self, obj):
        out = [None] * self.world
        self.dist.all_gather_object(out, obj, group=self.group)
        return out


# ---------------------------------------------------------------- instance split
def balance_by_nnz(nnz, world: int) -> list:
    """Instances to ranks, largest first onto the rank with the fewest
    occurrences so far (ties to the lower rank); each rank's list is in batch
    order.  The heaviest rank exceeds the mean by less than the largest
    instance."""
    nnz = [int(x) for x in nnz]
    order = sorted(range(len(nnz)), key=lambda j: (-nnz[j], j))
    load = [0] * world
    owned = [[] for _ in range(world)]
    for j in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owned[r].append(j)
        load[r] += nnz[j]
    return [sorted(o) for o in owned]


def instance_nnz(instances) -> list:
    """Literal occurrences of each (n_vars, clause_ptr, lits) instance."""
    return [int(np.asarray(p)[-1]) for (_, p, _) in instances]


class InstanceShards:
    """This rank's share of a batch: load, init, steps, and the gather of every
    instance's status (rank order undone) at the end."""

    def __init__(self, instances, engine_factory, comm=None):
        self.comm = comm or LocalComm()
        self.n_inst = len(instances)
        self.owned = balance_by_nnz(instance_nnz(instances), self.comm.world)[self.comm.rank]
        self.engine = engine_factory([instances[j] for j in self.owned], list(self.owned)) if self.owned else None

    def init(self, hp):
        if self.engine is not None:
            self.engine.init(hp)

    def step(self, hp, n_steps: int, stop_on_sat: bool = True):
        if self.engine is not None:
            self.engine.step(hp, n_steps, stop_on_sat)

    def gather(self) -> list:
        """Status record of every instance of the batch, in batch order (on every rank)."""
        local = list(zip(self.owned, self.engine.status())) if self.engine is not None else []
        out = [None] * self.n_inst
        for part in self.comm.all_gather_object(local):
            for j, rec in part:
                out[j] = rec
        return out


class CudaBatchEngine:
    """A rank's instances as one loaded batch on this GPU (the library's
    multi-kernel step), each with its global batch position as stream id."""

    def __init__(self, instances, ids, N: int, device="cuda"):
        from . import turbosat as ts
        self.ts = ts
        self.prob = ts.Problem(instances, device=device)
        ts.tsat_problem_set_instance_ids(self.prob.h, ids)
        self.st = ts.State(self.prob, N)

    def init(self, hp):
        self.ts.tsat_init(self.st.h, hp)

    def step(self, hp, n_steps, stop_on_sat):
        self.ts.tsat_step(self.st.h, hp, n_steps, stop_on_sat=stop_on_sat)

    def status(self) -> list:
        return self.ts.tsat_status(self.st.h, self.prob.info["n_inst"])["inst"]


# ---------------------------------------------------------------- sample split
def merge_shard_status(parts, n_local: int) -> list:
    """Per-instance status over all shards from each shard's own records
    (shard r holds samples [r n_local, (r + 1) n_local)): the loss is the sum,
    min_unsat the minimum with the lowest global sample on ties, and an
    instance is found at the earliest step any shard found it (lowest global
    sample on ties)."""
    out = []
    for j in range(len(parts[0])):
        recs = [(r, p[j]) for r, p in enumerate(parts)]
        best = min(recs, key=lambda x: (x[1]["min_unsat"], x[0] * n_local + x[1]["best_sample"]))
        found = [(x["found_step"], r * n_local + x["found_sample"]) for r, x in recs if x["found"]]
        rec = {"loss": float(sum(x["loss"] for _, x in recs)), "min_unsat": best[1]["min_unsat"],
               "best_sample": best[0] * n_local + best[1]["best_sample"], "found": int(bool(found)),
               "found_step": -1, "found_sample": -1}
        if found:
            rec["found_step"], rec["found_sample"] = min(found)
        out.append(rec)
    return out


class SampleShards:
    """One problem whose N samples are split evenly over the ranks of `comm`.
    A step is grad -> all-reduce of sum G z -> update -> all-reduce of sum z
    -> finish (two all-reduces of V floats)."""

    def __init__(self, engine, comm=None):
        self.comm = comm or LocalComm()
        self.engine = engine

    def init(self, hp):
        rs = self.engine.init(hp)
        self.comm.allreduce_sum_(rs)
        self.engine.finish(hp, rs)

    def step(self, hp, n_steps: int = 1):
        for _ in range(n_steps):
            dot = self.engine.grad(hp)
            self.comm.allreduce_sum_(dot)
            rs = self.engine.update(hp, dot)
            self.comm.allreduce_sum_(rs)
            self.engine.finish(hp, rs)

    def status(self) -> list:
        return merge_shard_status(self.comm.all_gather_object(self.engine.status()), self.engine.n_local)


class CudaShardEngine:
    """This rank's samples [rank n_local, (rank + 1) n_local) of a problem on
    this GPU, through the library's tsat_shard_* calls."""

    def __init__(self, instances, n_total: int, rank: int, world: int, device="cuda"):
        import torch

        from . import turbosat as ts
        if n_total % world:
            raise ValueError(f"{n_total} samples do not split over {world} ranks")
        self.ts = ts
        self.n_local = n_total // world
        self.prob = ts.Problem(instances, device=device)
        self.st = ts.State(self.prob, self.n_local)
        ts.tsat_state_set_shard(self.st.h, rank * self.n_local, n_total)
        V = self.prob.info["n_vars"]
        self.G = torch.empty((V, self.n_local), dtype=torch.float32, device=device)
        self.rowdot = torch.empty(V, dtype=torch.float32, device=device)
        self.rowsum = torch.empty(V, dtype=torch.float32, device=device)

    def init(self, hp):
        self.ts.tsat_shard_init(self.st.h, hp, self.rowsum)
        return self.rowsum

    def grad(self, hp):
        self.ts.tsat_shard_grad(self.st.h, hp, self.G, self.rowdot)
        return self.rowdot

    def update(self, hp, dot_total):
        self.ts.tsat_shard_update(self.st.h, hp, self.G, dot_total, self.rowsum)
        return self.rowsum

    def finish(self, hp, rowsum_total):
        self.ts.tsat_shard_finish(self.st.h, hp, rowsum_total)

    def status(self) -> list:
        return self.ts.tsat_status(self.st.h, self.prob.info["n_inst"])["inst"]
