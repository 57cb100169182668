"""FP64 oracle of the learned proposer (a 3-layer message-passing network on the
literal-clause graph).  TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.

Network, for literal l = 2 v + negated, its negation l ^ 1, clause c:
  f_l  = [1, log(1 + deg l), log(1 + deg l^1)]
  h0_l = relu(W0 f_l + b0)
  layer t = 1..3:
    m_c = mean over the literals of c of h_l
    e_c = relu(Wc m_c + bc)
    a_l = mean over the clauses that contain l of e_c   (0 when deg l = 0)
    h_l = relu(Wl [h_l ; a_l ; h_{l^1}] + bl)
  logit_v = wo [h_{2v} ; h_{2v+1}] + bo
  loss = sum over instances of mean over their variables of BCE(logit_v, y_v)

Weights are used as given (the GPU rounds them to BF16 first; the parity test
passes the same rounded values).  Parameters are one flat vector in the order
W0, b0, then per layer Wc, bc, Wl, bl, then wo, bo.  ``backward`` is written
out by hand; the tests pin it with central finite differences, and pin the
gathers with dense incidence matrices.
"""
from __future__ import annotations

import numpy as np

H = 64
LAYERS = 3
FEAT = 3


def layout():
    off = {}
    o = 0
    off["W0"] = (o, (H, FEAT)); o += H * FEAT
    off["b0"] = (o, (H,)); o += H
    for t in range(LAYERS):
        off[f"Wc{t}"] = (o, (H, H)); o += H * H
        off[f"bc{t}"] = (o, (H,)); o += H
        off[f"Wl{t}"] = (o, (H, 3 * H)); o += 3 * H * H
        off[f"bl{t}"] = (o, (H,)); o += H
    off["wo"] = (o, (2 * H,)); o += 2 * H
    off["bo"] = (o, (1,)); o += 1
    return off, o


def unpack(params):
    off, n = layout()
    assert params.shape[0] == n
    return {k: params[o:o + int(np.prod(s))].reshape(s) for k, (o, s) in off.items()}


def bf16_round(x):
    """Round FP32 values to BF16 (nearest, ties to even), returned as float64."""
    a = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((a + 0x7FFF + ((a >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


class Graph:
    """Literal-clause incidence of a (possibly concatenated) problem."""

    def __init__(self, cnfs):
        lits, owner, inst_of_var = [], [], []
        v0 = 0
        c0 = 0
        self.n_vars_inst = []
        for j, cnf in enumerate(cnfs):
            L = 2 * (cnf.var.astype(np.int64) + v0) + cnf.neg
            lits.append(L)
            owner.append(np.repeat(np.arange(cnf.C) + c0, np.diff(cnf.cptr)))
            inst_of_var.append(np.full(cnf.V, j))
            self.n_vars_inst.append(cnf.V)
            v0 += cnf.V
            c0 += cnf.C
        self.V, self.C = v0, c0
        self.lit = np.concatenate(lits)
        self.own = np.concatenate(owner)
        self.inst_of_var = np.concatenate(inst_of_var)
        self.clen = np.bincount(self.own, minlength=self.C).astype(np.float64)
        self.ldeg = np.bincount(self.lit, minlength=2 * self.V).astype(np.float64)

    def clause_mean(self, h):
        m = np.zeros((self.C, h.shape[1]))
        np.add.at(m, self.own, h[self.lit])
        return m / self.clen[:, None]

    def lit_mean(self, e):
        a = np.zeros((2 * self.V, e.shape[1]))
        np.add.at(a, self.lit, e[self.own])
        return a / np.maximum(self.ldeg, 1.0)[:, None]


def relu(x):
    return np.maximum(x, 0.0)


def forward(g: Graph, params, keep=False):
    P = unpack(np.asarray(params, np.float64))
    L = 2 * g.V
    neg = np.arange(L) ^ 1
    f = np.stack([np.ones(L), np.log1p(g.ldeg), np.log1p(g.ldeg[neg])], axis=1)
    h = relu(f @ P["W0"].T + P["b0"])
    cache = dict(f=f, h=[h], m=[], e=[], a=[])
    for t in range(LAYERS):
        m = g.clause_mean(h)
        e = relu(m @ P[f"Wc{t}"].T + P[f"bc{t}"])
        a = g.lit_mean(e)
        x = np.concatenate([h, a, h[neg]], axis=1)
        h = relu(x @ P[f"Wl{t}"].T + P[f"bl{t}"])
        cache["m"].append(m); cache["e"].append(e); cache["a"].append(a); cache["h"].append(h)
    hv = h.reshape(g.V, 2 * H)
    logits = hv @ P["wo"] + P["bo"][0]
    return (logits, cache) if keep else logits


def bce_loss(g: Graph, logits, y):
    """Sum over instances of the mean BCE over the instance's variables."""
    x = np.asarray(logits, np.float64)
    t = np.asarray(y, np.float64)
    per = np.maximum(x, 0) - x * t + np.log1p(np.exp(-np.abs(x)))
    w = 1.0 / np.asarray(g.n_vars_inst, np.float64)[g.inst_of_var]
    loss = float(np.sum(per * w))
    dlog = (1.0 / (1.0 + np.exp(-x)) - t) * w
    return loss, dlog


def backward(g: Graph, params, cache, dlog):
    P = unpack(np.asarray(params, np.float64))
    G = {k: np.zeros_like(v) for k, v in P.items()}
    L = 2 * g.V
    neg = np.arange(L) ^ 1
    hv = cache["h"][-1].reshape(g.V, 2 * H)
    G["wo"] = dlog @ hv
    G["bo"] = np.array([dlog.sum()])
    dh = (dlog[:, None] * P["wo"][None, :]).reshape(L, H)
    for t in reversed(range(LAYERS)):
        h_in, a, h_out = cache["h"][t], cache["a"][t], cache["h"][t + 1]
        dz = dh * (h_out > 0)
        x = np.concatenate([h_in, a, h_in[neg]], axis=1)
        G[f"Wl{t}"] = dz.T @ x
        G[f"bl{t}"] = dz.sum(axis=0)
        dx = dz @ P[f"Wl{t}"]
        dh_in = dx[:, :H] + dx[neg, 2 * H:]
        da = dx[:, H:2 * H]
        # a = lit_mean(e): de_c = sum_{l in c} da_l / deg_l
        de = np.zeros((g.C, H))
        np.add.at(de, g.own, (da / np.maximum(g.ldeg, 1.0)[:, None])[g.lit])
        dze = de * (cache["e"][t] > 0)
        G[f"Wc{t}"] = dze.T @ cache["m"][t]
        G[f"bc{t}"] = dze.sum(axis=0)
        dm = dze @ P[f"Wc{t}"]
        # m = clause_mean(h): dh_l += sum_{c owns l} dm_c / |c|
        np.add.at(dh_in, g.lit, (dm / g.clen[:, None])[g.own])
        dh = dh_in
    dz0 = dh * (cache["h"][0] > 0)
    G["W0"] = dz0.T @ cache["f"]
    G["b0"] = dz0.sum(axis=0)
    off, n = layout()
    flat = np.zeros(n)
    for k, (o, s) in off.items():
        flat[o:o + int(np.prod(s))] = G[k].reshape(-1)
    return flat


def loss_and_grad(g: Graph, params, y):
    logits, cache = forward(g, params, keep=True)
    loss, dlog = bce_loss(g, logits, y)
    return loss, backward(g, params, cache, dlog), logits
