"""Pins of the proposer oracle: gathers against dense incidence matrices,
the loss against scipy's logistic, and the hand-written backward against
central finite differences (FP64)."""
import numpy as np
import pytest
from scipy.special import expit

import oracle
from oracle import mpnn
from paper_2511_07737_b300 import cnfgen


def _graph(seed=0):
    insts = [cnfgen.planted_ksat(12, 40, 3, seed), cnfgen.planted_ksat(9, 60, 4, seed + 1)]
    cnfs = [oracle.CNF(i.n_vars, i.clause_ptr, i.lits) for i in insts]
    return mpnn.Graph(cnfs), insts


def _params(seed):
    _, n = mpnn.layout()
    rng = np.random.default_rng(seed)
    return rng.normal(size=n) * 0.3


def test_gathers_match_dense_incidence():
    g, _ = _graph()
    L = 2 * g.V
    P = np.zeros((g.C, L))
    P[g.own, g.lit] = 1.0
    rng = np.random.default_rng(1)
    h = rng.normal(size=(L, 5))
    e = rng.normal(size=(g.C, 5))
    np.testing.assert_allclose(g.clause_mean(h), (P @ h) / P.sum(axis=1, keepdims=True), rtol=1e-13)
    deg = np.maximum(P.sum(axis=0), 1.0)
    np.testing.assert_allclose(g.lit_mean(e), (P.T @ e) / deg[:, None], rtol=1e-13, atol=1e-15)


def test_bce_matches_logistic():
    g, _ = _graph()
    rng = np.random.default_rng(2)
    x = rng.normal(size=g.V) * 3
    y = rng.integers(0, 2, size=g.V)
    loss, dlog = mpnn.bce_loss(g, x, y)
    p = expit(x)
    w = 1.0 / np.asarray(g.n_vars_inst, float)[g.inst_of_var]
    ref = -np.sum(w * (y * np.log(p) + (1 - y) * np.log(1 - p)))
    assert abs(loss - ref) < 1e-12 * abs(ref)
    np.testing.assert_allclose(dlog, w * (p - y), rtol=1e-12)


@pytest.mark.parametrize("seed", [0, 1])
def test_backward_finite_differences(seed):
    g, insts = _graph(seed)
    params = _params(seed)
    y = np.concatenate([i.planted for i in insts])
    loss, grad, _ = mpnn.loss_and_grad(g, params, y)
    rng = np.random.default_rng(seed + 10)
    idx = rng.choice(params.shape[0], size=60, replace=False)
    off, _ = mpnn.layout()
    idx = np.concatenate([idx, [off["bo"][0], off["wo"][0], off["W0"][0], off["bc0"][0]]])
    for i in idx:
        h = 1e-6
        p1, p2 = params.copy(), params.copy()
        p1[i] += h
        p2[i] -= h
        l1, _ = mpnn.bce_loss(g, mpnn.forward(g, p1), y)
        l2, _ = mpnn.bce_loss(g, mpnn.forward(g, p2), y)
        fd = (l1 - l2) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, grad[i])


def test_bf16_rounding():
    # BF16 keeps 7 mantissa bits: spacing 2^-7 on [1, 2)
    x = np.array([1.0, 1.00390625, 1.01171875, 1.001953125, -3.14159, 0.0], np.float32)
    r = mpnn.bf16_round(x)
    assert r[0] == 1.0
    assert r[1] == 1.0              # 1 + 2^-8: tie, rounds to the even neighbour 1.0
    assert r[2] == 1.015625         # 1 + 3 * 2^-8: tie, rounds to the even neighbour 1 + 2^-6
    assert r[3] == 1.0              # below half a spacing
    assert abs(r[4] + 3.140625) < 1e-12
    assert r[5] == 0.0


def _selector_params():
    """Sparse weights that route chosen inputs to chosen hidden units, so the
    network's output has a closed form (all values exact in BF16):
      input layer : unit 0 = f0 (= 1), unit 1 = f1 = log(1 + deg l), unit 2 = f2 = log(1 + deg l')
      clause MLP  : e_c = mean over the literals of c of h (units 0 and 1 copied)
      literal MLP : unit 0 <- block h unit 0, unit 1 <- block a unit 1, unit 2 <- block h_neg unit 1
      head        : logit_v = h_{x_v}[1] - h_{x_v'}[1] + 0.5 h_{x_v}[2] + 0.25"""
    H = mpnn.H
    P = {k: np.zeros(s) for k, (o, s) in mpnn.layout()[0].items()}
    P["W0"][0, 0] = P["W0"][1, 1] = P["W0"][2, 2] = 1.0
    for t in range(mpnn.LAYERS):
        P[f"Wc{t}"][0, 0] = P[f"Wc{t}"][1, 1] = 1.0
        P[f"Wl{t}"][0, 0] = 1.0              # [h ; a ; h_neg]: column 0 is block h
        P[f"Wl{t}"][1, H + 1] = 1.0          # column H + 1 is block a, unit 1
        P[f"Wl{t}"][2, 2 * H + 1] = 1.0      # column 2H + 1 is block h_neg, unit 1
    P["wo"][1] = 1.0                         # [h_{x_v} ; h_{x_v'}]
    P["wo"][H + 1] = -1.0
    P["wo"][2] = 0.5
    P["bo"][0] = 0.25
    off, n = mpnn.layout()
    flat = np.zeros(n)
    for k, (o, s) in off.items():
        flat[o:o + int(np.prod(s))] = P[k].reshape(-1)
    return flat


def _selector_logits_by_hand(n_vars, clauses):
    """The closed form of the selector network, from the clause lists alone
    (no Graph helper): u_l = log(1 + deg l) at layer 0, then per layer
    u'_l = mean over the clauses c containing l of (mean over the literals of
    c of u), 0 for a literal in no clause; unit 2 after a layer is the previous
    layer's u of the negated literal."""
    import math
    lits = [(v, s) for v in range(n_vars) for s in (0, 1)]       # s = 1: negated literal
    deg = {l: sum(l in c for c in clauses) for l in lits}
    u = {l: math.log1p(deg[l]) for l in lits}
    u_neg_prev = None
    for _ in range(mpnn.LAYERS):
        cmean = [sum(u[l] for l in c) / len(c) for c in clauses]
        new = {}
        for l in lits:
            holders = [cmean[j] for j, c in enumerate(clauses) if l in c]
            new[l] = sum(holders) / len(holders) if holders else 0.0
        u_neg_prev = {l: u[(l[0], 1 - l[1])] for l in lits}
        u = new
    return np.array([u[(v, 0)] - u[(v, 1)] + 0.5 * u_neg_prev[(v, 0)] + 0.25 for v in range(n_vars)])


def test_forward_composition_closed_form_on_a_hand_sized_graph():
    """Pins the layer composition of the proposer: the feature vector
    [1, log(1+deg l), log(1+deg l')], the concatenation order [h ; a ; h_neg]
    and the output head [h_{x_v} ; h_{x_v'}].  Four variables, four clauses
    with unequal literal degrees: (x1 or not x2), (x1 or x2 or x3),
    (x1 or not x3 or x4), (not x1 or x4).  Any other block order, a swapped
    feature pair or swapped head halves change the logits."""
    clauses = [[(0, 0), (1, 1)], [(0, 0), (1, 0), (2, 0)], [(0, 0), (2, 1), (3, 0)], [(0, 1), (3, 0)]]
    ptr = np.array([0, 2, 5, 8, 10], np.int64)
    lits = np.array([1, -2, 1, 2, 3, 1, -3, 4, -1, 4], np.int32)
    cnf = oracle.CNF(4, ptr, lits)
    g = mpnn.Graph([cnf])
    params = _selector_params()
    got = mpnn.forward(g, params)
    want = _selector_logits_by_hand(4, clauses)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-14)
    # x4' is in no clause, so its u is 0 after every layer and logit(x4) is
    # u(x4) + 0.25 with u(x4) > 0; x1 occurs three times and x1' once
    assert want[3] > 0.25 and want[0] != want[1]
    # swapping the head halves changes the result
    H = mpnn.H
    swapped = params.copy()
    o = mpnn.layout()[0]["wo"][0]
    swapped[o:o + 2 * H] = np.concatenate([params[o + H:o + 2 * H], params[o:o + H]])
    assert np.abs(mpnn.forward(g, swapped) - want).max() > 1e-2


def test_forward_matches_a_dense_restatement():
    """Random weights: the oracle's forward against a restatement with an
    explicit dense clause-literal incidence matrix and explicit per-literal
    concatenation (no Graph helper)."""
    insts = [cnfgen.planted_ksat(7, 20, 3, 4)]
    cnf = oracle.CNF(insts[0].n_vars, insts[0].clause_ptr, insts[0].lits)
    g = mpnn.Graph([cnf])
    params = _params(5)
    P = mpnn.unpack(params)
    V, C, H = cnf.V, cnf.C, mpnn.H
    M = np.zeros((C, 2 * V))                     # M[c, l] = 1 if literal l is in clause c
    for c in range(C):
        for j in range(cnf.cptr[c], cnf.cptr[c + 1]):
            M[c, 2 * cnf.var[j] + cnf.neg[j]] = 1.0
    deg = M.sum(axis=0)
    h = np.zeros((2 * V, H))
    for l in range(2 * V):
        f = np.array([1.0, np.log1p(deg[l]), np.log1p(deg[l ^ 1])])
        h[l] = np.maximum(P["W0"] @ f + P["b0"], 0.0)
    for t in range(mpnn.LAYERS):
        e = np.maximum((M @ h) / M.sum(axis=1, keepdims=True) @ P[f"Wc{t}"].T + P[f"bc{t}"], 0.0)
        a = (M.T @ e) / np.maximum(deg, 1.0)[:, None]
        hn = np.zeros_like(h)
        for l in range(2 * V):
            x = np.concatenate([h[l], a[l], h[l ^ 1]])
            hn[l] = np.maximum(P[f"Wl{t}"] @ x + P[f"bl{t}"], 0.0)
        h = hn
    want = np.array([P["wo"] @ np.concatenate([h[2 * v], h[2 * v + 1]]) + P["bo"][0] for v in range(V)])
    np.testing.assert_allclose(mpnn.forward(g, params), want, rtol=1e-12, atol=1e-12)
