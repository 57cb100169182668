"""Learned proposer of initial logits: data generation, training and evaluation.

Orchestration only: every forward/backward/update runs in the library's CUDA
kernels (``tsat_mpnn_*``, ``tsat_step``, ``tsat_best``).

* ``solve``: a batch of CNFs with N samples each, optionally initialised from
  proposer logits (z_vi = logit_v * scale + noise_vi); returns per-instance
  steps-to-SAT and the satisfying assignment the solver found.
* ``Proposer``: the message-passing network's parameters (FP32 master, BF16
  compute copies inside the kernels) with an Adam optimiser; ``fit`` trains on
  (instance, assignment) pairs produced by ``solve``.
* ``compare``: learned vs random initialisation on the same instances, same
  solver settings and step cap; reports solve rates, steps and wall time.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import turbosat as ts


def _unpack_column(words: np.ndarray, col: int) -> np.ndarray:
    w = words[:, col // 32].astype(np.uint32)
    return ((w >> np.uint32(col % 32)) & np.uint32(1)).astype(np.uint8)


def solve(instances, N: int = 32, hp=None, max_steps: int = 500, logits: torch.Tensor | None = None,
          scale: float = 1.0, chunk: int = 50, device="cuda", persistent: bool = False) -> dict:
    """Run the gradient solver on a batch; returns found flags, steps-to-SAT,
    assignments (for solved instances), min-unsat trajectory and timings.
    ``persistent`` runs each chunk as one launch with a block per instance
    (tsat_step_persistent, for instances small enough for one block) instead
    of replaying the multi-kernel step graph."""
    if hp is None:
        hp = ts.hparams(seed=1, norm=ts.NORM_NONE, tau=2.0)
    prob = ts.Problem([(i.n_vars, i.clause_ptr, i.lits) for i in instances], device=device)
    st = ts.State(prob, N)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ts.tsat_init(st.h, hp, logits, scale)
    ncl = np.array([i.n_clauses for i in instances], np.float64)
    t99 = np.full(len(instances), -1, np.int64)
    done_steps = 0
    while done_steps < max_steps:
        k = min(chunk, max_steps - done_steps)
        if persistent:
            ts.tsat_step_persistent(st.h, hp, k, stop_on_sat=True)
        else:
            ts.tsat_step(st.h, hp, k, stop_on_sat=True)
        done_steps += k
        status = ts.tsat_status(st.h, len(instances))
        mu = np.array([x["min_unsat"] if not x["found"] else 0 for x in status["inst"]], np.float64)
        hit = ((ncl - mu) / ncl > 0.99) & (t99 < 0)
        t99[hit] = done_steps
        if status["all_done"]:
            break
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    status = ts.tsat_status(st.h, len(instances))
    bits = st.view("bits").cpu().numpy().view(np.uint32)
    offs = prob.var_offsets
    found, steps, assign, min_unsat = [], [], [], []
    for j, s in enumerate(status["inst"]):
        found.append(bool(s["found"]))
        steps.append(int(s["found_step"]) if s["found"] else -1)
        min_unsat.append(int(s["min_unsat"]))
        if s["found"]:
            assign.append(_unpack_column(bits[offs[j]:offs[j + 1]], s["found_sample"]))
        else:
            assign.append(None)
    return dict(found=np.array(found), steps=np.array(steps), assign=assign, min_unsat=np.array(min_unsat),
                t99=t99, wall=wall, total_steps=status["step"], ms_per_step=1e3 * wall / max(1, status["step"]))


class Proposer:
    def __init__(self, seed: int = 0, device="cuda"):
        self.n = ts.tsat_mpnn_param_count()
        self.device = device
        self.params = torch.empty(self.n, dtype=torch.float32, device=device)
        ts.tsat_mpnn_init(self.params, seed)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.step = 0

    def _ws(self, prob: ts.Problem) -> torch.Tensor:
        return ts._device_buffer(ts.tsat_mpnn_workspace_bytes(prob.h), prob.ws.device)

    def logits(self, prob: ts.Problem) -> torch.Tensor:
        out = torch.empty(prob.info["n_vars"], dtype=torch.float32, device=self.device)
        ws = self._ws(prob)
        ts.tsat_mpnn_forward(prob.h, self.params, ws, out)
        ts.tsat_mpnn_status(prob.h, ws)
        return out

    def train_step(self, prob: ts.Problem, targets: torch.Tensor, lr: float = 1e-3) -> float:
        ws = self._ws(prob)
        logits = torch.empty(prob.info["n_vars"], dtype=torch.float32, device=self.device)
        loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        ts.tsat_mpnn_loss_grad(prob.h, self.params, ws, targets, logits, loss, self.grad)
        ts.tsat_mpnn_status(prob.h, ws)
        self.step += 1
        ts.tsat_mpnn_adam(self.params, self.grad, self.m, self.v, self.step, lr)
        return float(loss.item()) / prob.info["n_inst"]

    def fit(self, data, epochs: int = 20, batch: int = 16, lr: float = 3e-3, seed: int = 0, log=None) -> list:
        """data: list of (instance, assignment uint8[n_vars])."""
        rng = np.random.default_rng(seed)
        hist = []
        batches = []
        for _ in range(epochs):
            order = rng.permutation(len(data))
            for b0 in range(0, len(order), batch):
                batches.append([data[k] for k in order[b0:b0 + batch]])
        cache = {}
        for bi, bt in enumerate(batches):
            key = tuple(id(x[0]) for x in bt)
            if key not in cache:
                prob = ts.Problem([(i.n_vars, i.clause_ptr, i.lits) for i, _ in bt], device=self.device)
                tgt = torch.tensor(np.concatenate([a for _, a in bt]), dtype=torch.uint8, device=self.device)
                cache = {key: (prob, tgt)}
            prob, tgt = cache[key]
            loss = self.train_step(prob, tgt, lr)
            hist.append(loss)
            if log and bi % 50 == 0:
                log(f"batch {bi}/{len(batches)} loss {loss:.4f}")
        return hist


def make_dataset(instances, N: int = 32, hp=None, max_steps: int = 500, batch: int = 256):
    """Solve the instances with the gradient solver (random init) and keep
    (instance, satisfying assignment) pairs; unsolved instances are dropped."""
    data, dropped = [], 0
    for b0 in range(0, len(instances), batch):
        part = instances[b0:b0 + batch]
        res = solve(part, N=N, hp=hp, max_steps=max_steps)
        for inst, f, a in zip(part, res["found"], res["assign"]):
            if f:
                data.append((inst, a))
            else:
                dropped += 1
    return data, dropped


def compare(instances, proposer: Proposer, N: int = 32, hp=None, max_steps: int = 1000, scale: float = 1.0,
            chunk: int = 50) -> dict:
    """Learned vs random initialisation on the same batch and solver settings."""
    prob = ts.Problem([(i.n_vars, i.clause_ptr, i.lits) for i in instances])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lg = proposer.logits(prob)
    torch.cuda.synchronize()
    t_prop = time.perf_counter() - t0
    rnd = solve(instances, N=N, hp=hp, max_steps=max_steps, chunk=chunk)
    lrn = solve(instances, N=N, hp=hp, max_steps=max_steps, logits=lg, scale=scale, chunk=chunk)

    def summ(r, extra=0.0):
        s = r["steps"][r["found"]]
        t99 = r["t99"][r["t99"] >= 0]
        return dict(solved=int(r["found"].sum()), rate=float(r["found"].mean()),
                    median_steps=float(np.median(s)) if s.size else None,
                    median_seconds=(float(np.median(s)) * r["ms_per_step"] / 1e3 + extra) if s.size else None,
                    reached99=int(t99.size), median_steps_to_99=float(np.median(t99)) if t99.size else None,
                    ms_per_step=r["ms_per_step"], mean_min_unsat=float(r["min_unsat"].mean()))

    out = dict(random=summ(rnd), learned=summ(lrn, t_prop), proposal_seconds=t_prop, n=len(instances))
    # solve-rate-matched comparison: the k fastest solves of each, k = min(solved)
    k = min(int(rnd["found"].sum()), int(lrn["found"].sum()))
    if k > 0:
        a = np.sort(rnd["steps"][rnd["found"]])[:k]
        b = np.sort(lrn["steps"][lrn["found"]])[:k]
        out["matched_k"] = k
        out["matched_median_steps"] = dict(random=float(np.median(a)), learned=float(np.median(b)))
    return out
