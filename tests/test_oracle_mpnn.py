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
