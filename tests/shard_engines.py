"""FP64 oracle engines with the interfaces of the sharding module's CUDA
engines, for checking the host-side orchestration (instance assignment,
all-reduce placement, status merging and gathers) with gloo ranks on CPUs.
Test infrastructure: it calls oracle/ and nothing of the library's kernels."""
import numpy as np
import torch

import oracle


def stream_seed(seed: int, gid: int) -> int:
    """The key the library uses for instance `gid`: low word seed_low + gid."""
    return (seed & ~0xFFFFFFFF) | ((seed + gid) & 0xFFFFFFFF)


def _hp(hp):
    return oracle.hparams(tau=hp.tau, lr0=hp.lr0, lr_factor=hp.lr_factor, lr_floor=hp.lr_floor,
                          decay_period=hp.decay_period, restart_period=hp.restart_period, beta1=hp.beta1,
                          beta2=hp.beta2, eps=hp.eps, weight_decay=hp.weight_decay, norm=hp.norm)


def _guard(mu):
    mu = np.asarray(mu, np.float64).copy()
    small = np.abs(mu) < 1e-12
    mu[small] = np.where(mu[small] < 0, -1e-12, 1e-12)
    return mu


def bits_at_global(z, nu, hp, seed, t, base, n_total):
    """Eq. 2 / Philox bits of the columns [base, base + n) of an n_total-sample
    state: the columns are placed at their global indices (others zero), so
    the oracle draws with the global counters."""
    V, n = z.shape
    pad = np.zeros((V, n_total), np.float32)
    pad[:, base:base + n] = z
    X = oracle.binarize_f32(pad, np.asarray(nu, np.float32), hp.binarize, c=0.25 / hp.bin_temp, seed=seed, t=t)
    return X[:, base:base + n]


class OracleBatchEngine:
    """Each instance solved alone in FP64, seeded by its stream id."""

    def __init__(self, instances, ids, N):
        self.cnfs = [oracle.CNF(n, p, l) for (n, p, l) in instances]
        self.ids = list(ids)
        self.N = N

    def init(self, hp):
        self.t = 0
        self.s = []
        for cnf, gid in zip(self.cnfs, self.ids):
            seed = stream_seed(hp.seed, gid)
            z = oracle.init_normal(cnf.V, self.N, seed).astype(np.float64)
            nu = oracle.nu_f32(z.astype(np.float32), hp.norm)
            X = oracle.binarize_f32(z.astype(np.float32), nu.astype(np.float32), hp.binarize, c=0.25 / hp.bin_temp,
                                    seed=seed, t=0)
            self.s.append(dict(z=z, m=np.zeros_like(z), v=np.zeros_like(z), nu=nu, X=X, seed=seed,
                               rec=dict(found=0, found_sample=-1, found_step=-1, min_unsat=-1, best_sample=-1,
                                        loss=0.0)))

    def step(self, hp, n_steps, stop_on_sat):
        ohp = _hp(hp)
        for _ in range(n_steps):
            for cnf, s in zip(self.cnfs, self.s):
                if s["rec"]["found"]:
                    continue
                out = oracle.step(cnf, ohp, self.t, s["z"], s["m"], s["v"], X=s["X"], nu_in=s["nu"])
                u = out["unsat"]
                r = s["rec"]
                r.update(loss=out["L"], min_unsat=int(u.min()), best_sample=int(np.argmin(u)))
                if u.min() == 0:          # frozen at this step: the model is kept
                    r.update(found=1, found_sample=int(np.argmin(u)), found_step=self.t)
                    continue
                z32 = s["z"].astype(np.float32)
                s["nu"] = oracle.nu_f32(z32, hp.norm)
                s["X"] = oracle.binarize_f32(z32, s["nu"].astype(np.float32), hp.binarize, c=0.25 / hp.bin_temp,
                                             seed=s["seed"], t=self.t + 1)
            self.t += 1

    def status(self):
        return [dict(s["rec"]) for s in self.s]


class OracleShardEngine:
    """Samples [rank n_local, (rank + 1) n_local) of one instance in FP64."""

    def __init__(self, inst, n_total, rank, world):
        n, p, l = inst
        self.cnf = oracle.CNF(n, p, l)
        self.n_total = n_total
        self.n_local = n_total // world
        self.base = rank * self.n_local

    def init(self, hp):
        full = oracle.init_normal(self.cnf.V, self.n_total, hp.seed).astype(np.float64)
        self.z = full[:, self.base:self.base + self.n_local].copy()
        self.m = np.zeros_like(self.z)
        self.v = np.zeros_like(self.z)
        self.t = 0
        self.rec = dict(found=0, found_sample=-1, found_step=-1, min_unsat=-1, best_sample=-1, loss=0.0)
        return self._rowsum(hp)

    def _rowsum(self, hp):
        if hp.norm == 2:
            return torch.zeros(self.cnf.V, dtype=torch.float64)
        a = np.abs(self.z) if hp.norm == 1 else self.z
        return torch.tensor(a.sum(axis=1))

    def finish(self, hp, total):
        self.nu = np.ones(self.cnf.V) if hp.norm == 2 else _guard(total.numpy() / self.n_total)
        self.X = bits_at_global(self.z.astype(np.float32), self.nu, hp, hp.seed, self.t, self.base, self.n_total)

    def grad(self, hp):
        zt = self.z / self.nu[:, None]
        S, L, G, unsat = oracle.objective(self.cnf, X=self.X, tau=hp.tau)
        self.G = G
        self.rec.update(loss=L, min_unsat=int(unsat.min()), best_sample=int(np.argmin(unsat)))
        if unsat.min() == 0 and not self.rec["found"]:
            self.rec.update(found=1, found_sample=int(np.argmin(unsat)), found_step=self.t)
        del zt
        if hp.norm == 2:
            return torch.zeros(self.cnf.V, dtype=torch.float64)
        return torch.tensor((G * self.z).sum(axis=1))

    def update(self, hp, dot_total):
        nu = self.nu[:, None]
        if hp.norm == 2:
            g = self.G
        else:
            dmu = np.sign(self.z) if hp.norm == 1 else 1.0
            g = self.G / nu - dot_total.numpy()[:, None] * dmu / (self.n_total * nu * nu)
        lr = oracle.lr_at(self.t, hp.lr0, hp.lr_factor, hp.decay_period, hp.restart_period, hp.lr_floor)
        oracle.adamw(self.z, self.m, self.v, np.ascontiguousarray(g), self.t + 1, lr, hp.beta1, hp.beta2, hp.eps,
                     hp.weight_decay)
        self.t += 1
        return self._rowsum(hp)

    def status(self):
        return [dict(self.rec)]
