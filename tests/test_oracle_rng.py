"""Pins of the oracle's Philox4x32-10, random-normal init and binarisation
(Eq. 2 and its Philox-sampled form), and the hand-off selection (Sec. IV-B)."""
import json
import os

import numpy as np
import pytest
from scipy.stats import chisquare

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_answer_vectors():
    g = json.load(open(os.path.join(GOLD, "philox4x32_10_kat.json")))
    for vec in g["vectors"]:
        ctr = [int(x, 16) for x in vec["ctr"]]
        key = [int(x, 16) for x in vec["key"]]
        out = [int(x, 16) for x in vec["out"]]
        assert list(oracle.philox4x32_10(ctr, key)) == out


def test_philox_uniformity():
    vals = []
    for i in range(4000):
        vals.extend(oracle.philox4x32_10([i, 7, 3, 1], [0x1234, 0x5678]))
    u = np.array(vals, np.uint64) >> np.uint64(24)        # top 8 bits
    counts = np.bincount(u.astype(np.int64), minlength=256)
    assert chisquare(counts).pvalue > 1e-4


def test_init_moments_and_balance():
    z = oracle.init_normal(200, 256, seed=3)
    assert z.dtype == np.float32
    n = z.size
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / n) + 0.02
    assert np.abs(z).max() < 6.0
    assert abs((z > 0).mean() - 0.5) < 5 * 0.5 / np.sqrt(n)
    # values are integers scaled by 2^-24 (exact construction)
    k = z.astype(np.float64) * 2**24
    np.testing.assert_array_equal(k, np.round(k))
    # seeds differ -> streams differ; same seed -> identical
    np.testing.assert_array_equal(z, oracle.init_normal(200, 256, seed=3))
    assert not np.array_equal(z, oracle.init_normal(200, 256, seed=4))


def test_init_with_logits_shifts_rows():
    lg = np.linspace(-2, 2, 16).astype(np.float32)
    z0 = oracle.init_normal(16, 64, seed=1)
    z1 = oracle.init_normal(16, 64, seed=1, logits=lg, scale=3.0)
    np.testing.assert_array_equal(z1, (lg[:, None] * np.float32(3.0)) + z0)


def test_binarize_det_is_sign_rule():
    rng = np.random.default_rng(0)
    z = rng.normal(size=(30, 64)).astype(np.float32)
    z[0, :4] = [0.0, -0.0, 1e-30, -1e-30]
    nu = np.where(rng.random(30) < 0.5, -1.0, 1.0).astype(np.float32) * rng.random(30).astype(np.float32)
    X = oracle.binarize_f32(z, nu, 0)
    # B(x) = clip(sign(x), 0, 1) of Eq. 2 on the FP32 quotient
    q = (z / nu[:, None]).astype(np.float32)
    np.testing.assert_array_equal(X, np.clip(np.sign(q), 0, 1).astype(np.uint8))


def test_binarize_philox_cold_limit_is_det():
    rng = np.random.default_rng(1)
    z = rng.normal(size=(20, 96)).astype(np.float32)
    nu = np.ones(20, np.float32)
    Xd = oracle.binarize_f32(z, nu, 0)
    Xp = oracle.binarize_f32(z, nu, 1, c=1e30, seed=9, t=4)
    np.testing.assert_array_equal(Xd, Xp)


def test_binarize_philox_frequency():
    V, N = 64, 1024
    z = np.full((V, N), 1.0, np.float32)
    nu = np.ones(V, np.float32)
    X = oracle.binarize_f32(z, nu, 1, c=0.25, seed=5, t=2)   # p = 0.75
    p = X.mean()
    assert abs(p - 0.75) < 5 * np.sqrt(0.75 * 0.25 / X.size)
    X2 = oracle.binarize_f32(z, nu, 1, c=0.25, seed=5, t=3)
    assert not np.array_equal(X, X2)                         # fresh draw per step


def test_best_sample_and_topk_bruteforce():
    rng = np.random.default_rng(2)
    for _ in range(20):
        u = rng.integers(0, 4, size=50).astype(np.int32)
        assert oracle.best_sample(u) == int(np.argmin(u))
        a = np.round(rng.random(300), 2)                      # many ties
        k = int(rng.integers(1, 60))
        got = oracle.topk_confident(a, k)
        ref = np.lexsort((np.arange(300), a))[:k]
        np.testing.assert_array_equal(got, ref)
    assert oracle.partial_k(100) == 20
    assert oracle.partial_k(1_000_000) == 100
    assert oracle.partial_k(1_000_001) == 101
    assert oracle.partial_k(7) == 7


def test_binarize_philox_counter_layout_and_halves():
    # sample i of variable v at step t uses the 16-bit half i mod 8 of the
    # Philox output for counter (i / 8, v, t, 0x42494E41) (low half of word 0
    # first); with p fixed, x = [half / 2^16 < p]
    V, N, t, seed = 5, 64, 7, 0x1234_5678_9ABC
    z = np.zeros((V, N), np.float32)          # p = 0.5 + c * 0 = 0.5
    nu = np.ones(V, np.float32)
    X = oracle.binarize_f32(z, nu, 1, c=0.25, seed=seed, t=t)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for v in range(V):
        for i in range(N):
            o = oracle.philox4x32_10((i // 8, v, t, 0x42494E41), key)
            half = (int(o[(i % 8) // 2]) >> (16 * (i % 2))) & 0xFFFF
            assert X[v, i] == (1 if half / 65536.0 < 0.5 else 0), (v, i)


def test_binarize_philox_halves_are_independent():
    # the eight samples that share one draw get distinct 16-bit halves: at
    # p = 1/2 neighbours agree half the time and every sample is a fair coin
    V, N = 256, 1024
    z = np.zeros((V, N), np.float32)
    nu = np.ones(V, np.float32)
    X = oracle.binarize_f32(z, nu, 1, c=0.25, seed=11, t=1).astype(np.int8)
    n = X.size
    assert abs(X.mean() - 0.5) < 5 * np.sqrt(0.25 / n)
    for d in (1, 2, 4):                        # same draw, other half / word
        agree = (X[:, :-d] == X[:, d:]).mean()
        assert abs(agree - 0.5) < 5 * np.sqrt(0.25 / (V * (N - d)))
