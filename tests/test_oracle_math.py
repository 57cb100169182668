"""Pins of the oracle's SmoothMin (Eq. 4), loss (Eq. 3), straight-through
gradient, Eq. 5 chain rule, AdamW and the learning-rate schedule (Sec. IV-A).

Independent references: scipy's logistic function for a two-valued column,
the tau -> infinity limit stated after Eq. 4, central finite differences
(of the smooth surrogate for the STE layer, directly for the relaxed layer),
numpy means for Eq. 5, and torch.optim.AdamW + LambdaLR in FP64."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.special import expit

import oracle
from paper_2511_07737_b300 import cnfgen
from tests.conftest import rel_err


def test_smoothmin_two_values_is_logistic():
    for tau in (0.3, 1.0, 2.5):
        R = np.array([[0.0], [1.0]])
        S = oracle.smoothmin(R, tau)
        assert abs(S[0] - expit(-tau)) < 1e-15


def test_smoothmin_constant_column_and_shift():
    R = np.full((7, 3), 2.0)
    S, d = oracle.smoothmin(R, 1.7, grad=True)
    np.testing.assert_allclose(S, 2.0, rtol=0, atol=1e-14)
    np.testing.assert_allclose(d.sum(axis=0), 1.0, atol=1e-14)
    rng = np.random.default_rng(0)
    R = rng.integers(0, 4, size=(9, 5)).astype(float)
    S0, d0 = oracle.smoothmin(R, 1.3, grad=True)
    S1 = oracle.smoothmin(R + 0.75, 1.3)
    np.testing.assert_allclose(S1 - S0, 0.75, atol=1e-13)
    np.testing.assert_allclose(d0.sum(axis=0), 1.0, atol=1e-13)


def test_smoothmin_tends_to_min():
    rng = np.random.default_rng(1)
    R = rng.integers(0, 5, size=(40, 16)).astype(float)
    S = oracle.smoothmin(R, 50.0)
    np.testing.assert_allclose(S, R.min(axis=0), atol=40 * 4 * np.exp(-50.0) * 5)


def test_smoothmin_finite_difference():
    rng = np.random.default_rng(2)
    R = rng.normal(size=(11, 4)) + 1.0
    tau = 1.4
    S, d = oracle.smoothmin(R, tau, grad=True)
    h = 1e-6
    for c in range(11):
        Rp, Rm = R.copy(), R.copy()
        Rp[c] += h
        Rm[c] -= h
        fd = (oracle.smoothmin(Rp, tau) - oracle.smoothmin(Rm, tau)) / (2 * h)
        assert rel_err(d[c], fd) < 1e-8


def _PD(cnf):
    """Sparse C x V matrix P D: +1 for x_v in clause c, -1 for x_v'."""
    rows = np.repeat(np.arange(cnf.C), np.diff(cnf.cptr))
    vals = np.where(cnf.neg.astype(bool), -1.0, 1.0)
    return sp.csr_matrix((vals, (rows, cnf.var)), shape=(cnf.C, cnf.V))


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_ste_gradient_surrogate_fd(mode):
    """F(z) = -sum_i SmoothMin(R0 + P D (zt(z) - zt(z0))) has gradient equal
    to the STE gradient at z0 (Sec. III-B, Fig. 3), chained through Eq. 5."""
    inst = cnfgen.planted_ksat(30, 120, 3, 5)
    cnf = oracle.CNF(30, inst.clause_ptr, inst.lits)
    N, tau = 6, 1.2
    rng = np.random.default_rng(3)
    z0 = rng.normal(size=(30, N)) + 0.3
    nu0, zt0 = oracle.normalize(z0, mode)
    X = (zt0 > 0).astype(np.uint8)
    R0 = oracle.result_matrix(cnf, X).astype(float)
    S, L, G, _ = oracle.objective(cnf, X=X, tau=tau)
    g = oracle.normalize_backward(z0, nu0, G, mode)
    PD = _PD(cnf)

    def F(z):
        _, zt = oracle.normalize(z, mode)
        return -oracle.smoothmin(R0 + PD @ (zt - zt0), tau).sum()

    assert abs(F(z0) - L) < 1e-12
    fd = np.zeros_like(z0)
    for v in range(30):
        for i in range(N):
            h = 1e-6 * max(1.0, abs(z0[v, i]))
            zp, zm = z0.copy(), z0.copy()
            zp[v, i] += h
            zm[v, i] -= h
            fd[v, i] = (F(zp) - F(zm)) / (2 * h)
    assert rel_err(g, fd) < 1e-6
    # at mode 2 the chain rule is the identity, so G itself is pinned
    if mode == 2:
        assert rel_err(G, fd) < 1e-6


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_relaxed_gradient_fd(mode):
    inst = cnfgen.structured_mixed(64, 200, 4, communities=4)
    cnf = oracle.CNF(64, inst.clause_ptr, inst.lits)
    N, tau = 4, 0.9
    rng = np.random.default_rng(4)
    z0 = rng.normal(size=(64, N)) + 0.2

    def Lz(z):
        _, zt = oracle.normalize(z, mode)
        return oracle.objective(cnf, zt=zt, tau=tau, grad=False)[1]

    nu, zt = oracle.normalize(z0, mode)
    _, L, G, _ = oracle.objective(cnf, zt=zt, tau=tau)
    g = oracle.normalize_backward(z0, nu, G, mode)
    fd = np.zeros_like(z0)
    for v in range(64):
        for i in range(N):
            h = 1e-6 * max(1.0, abs(z0[v, i]))
            zp, zm = z0.copy(), z0.copy()
            zp[v, i] += h
            zm[v, i] -= h
            fd[v, i] = (Lz(zp) - Lz(zm)) / (2 * h)
    assert rel_err(g, fd) < 1e-6


def test_normalize_matches_numpy_means():
    rng = np.random.default_rng(5)
    z = rng.normal(size=(8, 32))
    nu, zt = oracle.normalize(z, 0)
    np.testing.assert_allclose(nu, z.mean(axis=1), rtol=1e-14)
    np.testing.assert_allclose(zt, z / z.mean(axis=1, keepdims=True), rtol=1e-14)
    nu1, _ = oracle.normalize(z, 1)
    np.testing.assert_allclose(nu1, np.abs(z).mean(axis=1), rtol=1e-14)
    nu2, zt2 = oracle.normalize(z, 2)
    np.testing.assert_array_equal(nu2, 1.0)
    np.testing.assert_array_equal(zt2, z)
    # guard: a row with zero mean is divided by +1e-12
    zz = np.array([[1.0, -1.0, 2.0, -2.0]])
    nug, _ = oracle.normalize(zz, 0)
    assert nug[0] == 1e-12


def test_lr_schedule_values_of_sec_iv_a():
    assert oracle.lr_at(0) == pytest.approx(1e-1, rel=1e-15)
    assert oracle.lr_at(29) == pytest.approx(1e-1, rel=1e-15)
    assert oracle.lr_at(30) == pytest.approx(1e-2, rel=1e-15)
    assert oracle.lr_at(359) == pytest.approx(1e-12, rel=1e-12)
    assert oracle.lr_at(360) == pytest.approx(1e-1, rel=1e-15)          # restart
    assert oracle.lr_at(390) == pytest.approx(1e-2, rel=1e-15)
    assert oracle.lr_at(20, restart=10_000, period=1) == pytest.approx(1e-15)   # floor


def test_adamw_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(6)
    V, N = 5, 7
    z = rng.normal(size=(V, N))
    m = np.zeros_like(z)
    v = np.zeros_like(z)
    p = torch.nn.Parameter(torch.tensor(z.copy(), dtype=torch.float64))
    opt = torch.optim.AdamW([p], lr=0.1, betas=(0.9, 0.999), eps=1e-8, weight_decay=0.01)
    sched = torch.optim.lr_scheduler.LambdaLR(opt, lambda t: 0.1 ** ((t % 360) // 30))
    for t in range(75):
        g = rng.normal(size=(V, N)) * (0.1 + t % 3)
        p.grad = torch.tensor(g)
        opt.step()
        sched.step()
        oracle.adamw(z, m, v, g, t + 1, oracle.lr_at(t))
        assert rel_err(z, p.detach().numpy()) < 1e-12, t


def test_step_composes_the_pinned_pieces():
    inst = cnfgen.planted_ksat(40, 170, 3, 9)
    cnf = oracle.CNF(40, inst.clause_ptr, inst.lits)
    rng = np.random.default_rng(7)
    N = 8
    z = rng.normal(size=(40, N)) + 0.1
    m = rng.normal(size=(40, N)) * 0.01
    v = np.abs(rng.normal(size=(40, N))) * 0.01
    hp = oracle.hparams(tau=1.5, norm=0)
    nu, zt = oracle.normalize(z, 0)
    X = (zt > 0).astype(np.uint8)
    S, L, G, unsat = oracle.objective(cnf, X=X, tau=1.5)
    g = oracle.normalize_backward(z, nu, G, 0)
    z2, m2, v2 = z.copy(), m.copy(), v.copy()
    oracle.adamw(z2, m2, v2, g, 13, oracle.lr_at(12))
    out = oracle.step(cnf, hp, 12, z, m, v, X=X)
    assert rel_err(out["G"], G) == 0.0 and rel_err(out["g"], g) == 0.0
    assert rel_err(z, z2) == 0.0 and rel_err(m, m2) == 0.0 and rel_err(v, v2) == 0.0
    np.testing.assert_array_equal(out["unsat"], unsat)
    np.testing.assert_allclose(out["nu_next"], z.mean(axis=1), rtol=1e-14)


def test_oracle_solves_small_planted():
    """End to end: the method finds a model of a small planted formula under
    the sign-keeping normaliser (mean |z|); the exact check confirms it.
    (Eq. 5 read as the signed mean drives rows to one sign, after which every
    sample sets the variable True; that reading stalls on this instance.)"""
    inst = cnfgen.planted_ksat(30, 120, 3, 11)
    cnf = oracle.CNF(30, inst.clause_ptr, inst.lits)
    N = 32
    hp = oracle.hparams(tau=1.0, norm=1)
    z = oracle.init_normal(30, N, 5).astype(np.float64)
    m = np.zeros_like(z)
    v = np.zeros_like(z)
    found = False
    for t in range(300):
        nu = oracle.nu_f32(z.astype(np.float32), 1)
        X = oracle.binarize_f32(z.astype(np.float32), nu.astype(np.float32), 0)
        out = oracle.step(cnf, hp, t, z, m, v, X=X)
        if (out["unsat"] == 0).any():
            i = int(np.argmax(out["unsat"] == 0))
            u, _ = oracle.check(cnf, X[:, i:i + 1])
            assert u[0] == 0
            found = True
            break
    assert found


def _mix_case(seed=0, V=12, N=16, R=3):
    from paper_2511_07737_b300 import cnfgen
    inst = cnfgen.planted_ksat(V, 40, 3, seed)
    cnf = oracle.CNF(inst.n_vars, inst.clause_ptr, inst.lits)
    rng = np.random.default_rng(seed)
    z = rng.normal(size=(V, N))
    m = rng.normal(size=(V, N)) * 0.1
    v = rng.random((V, N)) * 0.1
    X = (rng.random((V, N)) < 0.5).astype(np.uint8)
    return cnf, z, m, v, X, R


def test_mixing_step_keeps_best_and_averages_the_rest():
    # at an lr restart t = R with mixing on: i* = the sample with the fewest
    # unsatisfied clauses (lowest index on ties) keeps its z, every other
    # sample moves half way to it, the moments are zeroed, no gradient step
    cnf, z, m, v, X, R = _mix_case()
    hp = oracle.hparams(norm=1, restart_period=R, mix=1)
    unsat, _ = oracle.check(cnf, X)
    best = int(np.argmin(unsat))
    z0 = z.copy()
    out = oracle.step(cnf, hp, R, z, m, v, X=X)
    np.testing.assert_array_equal(out["unsat"], unsat)
    np.testing.assert_array_equal(z[:, best], z0[:, best])
    others = np.arange(z.shape[1]) != best
    np.testing.assert_allclose(z[:, others], 0.5 * (z0[:, others] + z0[:, [best]]), rtol=0, atol=0)
    assert not m.any() and not v.any()
    # not a restart step, or mixing off: an ordinary AdamW step
    for t, mix in ((R + 1, 1), (R, 0)):
        cnf, z, m, v, X, R = _mix_case(1)
        z0 = z.copy()
        oracle.step(cnf, oracle.hparams(norm=1, restart_period=R, mix=mix), t, z, m, v, X=X)
        assert m.any() and not np.array_equal(z, z0)


def test_first_step_after_a_mixing_restart_is_a_fresh_adam_step():
    # after the reset m = v = 0 and the step count restarts at 1, so the bias
    # corrected update is g / (|g| + eps) per element (closed form of AdamW's
    # first step): z' = z (1 - lr wd) - lr g / (|g| + eps)
    cnf, z, m, v, X, R = _mix_case(2)
    hp = oracle.hparams(norm=1, restart_period=R, mix=1, weight_decay=0.01)
    oracle.step(cnf, hp, R, z, m, v, X=X)               # mixing step: m = v = 0
    z1 = z.copy()
    out = oracle.step(cnf, hp, R + 1, z, m, v, X=X)
    g = out["g"]
    lr = oracle.lr_at(R + 1, hp.lr0, hp.lr_factor, hp.decay_period, hp.restart_period, hp.lr_floor)
    ref = z1 * (1 - lr * hp.weight_decay) - lr * g / (np.abs(g) + hp.eps)
    np.testing.assert_allclose(z, ref, rtol=1e-12, atol=1e-15)


def test_nu_f32_exact_means_guard_and_fp64_accumulation():
    """The FP32-input normaliser of Eq. 5 (the statistic the GPU's nu is held
    to).  Rows are built from dyadic values, so every mean below is exact in
    FP64 and known in closed form; the guard replaces magnitudes below 1e-12
    by +-1e-12 (0 -> +1e-12); the sums run in FP64, not FP32."""
    N = 64
    half = N // 2
    dev = (np.arange(half) % 5 + 1) / 8.0                    # 1/8 .. 5/8, dyadic
    rows, mean0, mean1 = [], [], []
    for c in (0.75, -1.5, 3.0):                               # c + d, c - d pairs: mean c exactly
        rows.append(np.concatenate([c + dev, c - dev]))
        mean0.append(c)
        mean1.append(abs(c))                                  # |c| > 5/8: no value changes sign
    a, b, k = 1.25, 0.5, 40                                   # k values a, N - k values -b
    rows.append(np.array([a] * k + [-b] * (N - k)))
    mean0.append((k * a - (N - k) * b) / N)
    mean1.append((k * a + (N - k) * b) / N)
    big = 2.0 ** 24                                           # FP32 would lose the ones next to 2^24
    rows.append(np.array([big] + [1.0] * (N - 2) + [-big]))
    mean0.append((N - 2) / N)
    mean1.append((2 * big + N - 2) / N)
    z = np.array(rows, np.float32)
    assert np.array_equal(z.astype(np.float64), np.array(rows))   # every value is exact in FP32
    np.testing.assert_array_equal(oracle.nu_f32(z, 0), mean0)
    np.testing.assert_array_equal(oracle.nu_f32(z, 1), mean1)
    np.testing.assert_array_equal(oracle.nu_f32(z, 2), 1.0)
    # permutation invariance and exact scaling by a power of two
    perm = np.random.default_rng(0).permutation(N)
    np.testing.assert_array_equal(oracle.nu_f32(z[:, perm], 0), mean0)
    np.testing.assert_array_equal(oracle.nu_f32(z * np.float32(0.25), 1), np.array(mean1) * 0.25)
    # the guard: exact zero, mean -1e-13, mean +5e-13, and a mean just outside it
    tiny_neg = np.float32(-1e-13 * N)
    tiny_pos = np.float32(5e-13 * N)
    outside = np.float32(-2e-12 * N)
    g = np.zeros((5, N), np.float32)
    g[1, 0] = tiny_neg
    g[2, 0] = tiny_pos
    g[3, 0] = outside
    g[4, :half], g[4, half:] = 1.5, -1.5                      # signed mean 0, mean |z| 1.5
    nu0 = oracle.nu_f32(g, 0)
    assert nu0[0] == 1e-12 and nu0[1] == -1e-12 and nu0[2] == 1e-12 and nu0[4] == 1e-12
    assert nu0[3] == float(outside) / N and nu0[3] < -1e-12
    nu1 = oracle.nu_f32(g, 1)
    assert nu1[0] == 1e-12 and nu1[1] == 1e-12 and nu1[2] == 1e-12   # mean |z| is never negative
    assert nu1[3] == -float(outside) / N and nu1[4] == 1.5
    # the FP64 normaliser of the same values agrees (same definition, FP64 inputs)
    np.testing.assert_array_equal(oracle.normalize(z.astype(np.float64), 0)[0], mean0)
