"""Helpers shared by the GPU parity tests (CUDA path through the C ABI vs oracle)."""
import numpy as np
import torch

import oracle
from paper_2511_07737_b300 import turbosat as ts

# Tolerances (max-norm relative error, see tests/conftest.rel_err):
#   FP32 objective, gradient and state after one step: 1e-5
#   BF16 storage of relaxed literal values (FP32 sums): 1e-2
TOL_F32 = 1e-5
TOL_BF16 = 1e-2


def unpack_bits(words: np.ndarray, N: int) -> np.ndarray:
    """[V][N/32] uint32 words -> [V][N] 0/1 (bit i%32 of word i/32 = sample i)."""
    w = np.ascontiguousarray(words).view(np.uint32)
    return np.unpackbits(w.view(np.uint8), axis=1, bitorder="little")[:, :N]


def stream_seed(seed: int, gid: int) -> int:
    """Philox key of instance `gid`: the library offsets the key's low word by
    the instance's id (its position in the loaded batch by default)."""
    return (seed & ~0xFFFFFFFF) | ((seed + gid) & 0xFFFFFFFF)


def binarize_like_gpu(z, nu, hp, t, offsets):
    """The oracle's Eq. 2 / Philox bits of a loaded batch: each instance's rows
    with its own key and instance-local row indices (its random stream)."""
    X = np.zeros(z.shape, np.uint8)
    for j in range(len(offsets) - 1):
        a, b = int(offsets[j]), int(offsets[j + 1])
        X[a:b] = oracle.binarize_f32(z[a:b], nu[a:b], hp.binarize, c=0.25 / hp.bin_temp,
                                     seed=stream_seed(hp.seed, j), t=t)
    return X


def snapshot(st: ts.State) -> dict:
    torch.cuda.synchronize()
    out = {k: st.view(k).cpu().numpy().copy() for k in ("z", "m", "v", "nu")}
    out["bits"] = st.view("bits").cpu().numpy().view(np.uint32).copy()
    out["X"] = unpack_bits(out["bits"], st.N)
    return out


def oracle_hp(hp: ts.tsat_hparams) -> oracle.HParams:
    return oracle.hparams(tau=hp.tau, lr0=hp.lr0, lr_factor=hp.lr_factor, lr_floor=hp.lr_floor,
                          decay_period=hp.decay_period, restart_period=hp.restart_period, beta1=hp.beta1,
                          beta2=hp.beta2, eps=hp.eps, weight_decay=hp.weight_decay, norm=hp.norm,
                          relaxed=hp.layer, mix=hp.mix_restart)


def lockstep(cnfs, offsets, hp, t, snap):
    """One oracle step per instance from the GPU's FP32 state (as FP64), using
    the GPU's bits and normaliser; returns concatenated z, m, v and per-instance
    (S, L, unsat)."""
    z = snap["z"].astype(np.float64)
    m = snap["m"].astype(np.float64)
    v = snap["v"].astype(np.float64)
    ohp = oracle_hp(hp)
    res = []
    for j, cnf in enumerate(cnfs):
        a, b = offsets[j], offsets[j + 1]
        zj, mj, vj = z[a:b].copy(), m[a:b].copy(), v[a:b].copy()
        out = oracle.step(cnf, ohp, t, zj, mj, vj, X=snap["X"][a:b], nu_in=snap["nu"][a:b].astype(np.float64))
        z[a:b], m[a:b], v[a:b] = zj, mj, vj
        res.append(out)
    return z, m, v, res


def make(instances, N, layer=ts.LAYER_STE, dtype=ts.DTYPE_F32, locality=False):
    prob = ts.Problem([(i.n_vars, i.clause_ptr, i.lits) for i in instances], locality=locality)
    st = ts.State(prob, N, layer, dtype)
    cnfs = [oracle.CNF(i.n_vars, i.clause_ptr, i.lits) for i in instances]
    return prob, st, cnfs


def assert_adamw_z(z_gpu, z_ref, m_gpu, m_ref, v_gpu, v_ref, t, hp, tol=TOL_F32, cnt=None):
    """z after AdamW, element by element, within a bound propagated from the
    measured m / v differences (which are themselves held to `tol`).

    z' = z (1 - lr wd) - lr u,  u = (m / bc1) / (sqrt(v / bc2) + eps).
    First order: |dz'| <= lr (|du/dm| |dm| + |du/dv| |dv|) + tol max|z'|, with
    du/dm = 1 / (bc1 (sqrt(vh) + eps)) and
    |du/dv| = |mh| / (2 bc2 sqrt(vh) (sqrt(vh) + eps)^2), vh = v / bc2, mh = m / bc1.
    Where |g| is comparable to eps the update is ill-conditioned and this
    bound, not the flat tolerance, is what FP32 arithmetic can meet."""
    from tests.conftest import rel_err
    assert rel_err(m_gpu, m_ref) < tol
    assert rel_err(v_gpu, v_ref) < tol
    lr = oracle.lr_at(t, hp.lr0, hp.lr_factor, hp.decay_period, hp.restart_period, hp.lr_floor)
    cnt = t + 1 if cnt is None else cnt        # AdamW step count (restarts with assignment mixing)
    bc1 = 1.0 - float(hp.beta1) ** cnt
    bc2 = 1.0 - float(hp.beta2) ** cnt
    vh = np.maximum(v_ref / bc2, 0.0)
    sq = np.sqrt(vh)
    eps = float(hp.eps)
    dm = np.abs(m_gpu.astype(np.float64) - m_ref)
    dv = np.abs(v_gpu.astype(np.float64) - v_ref)
    du_dm = 1.0 / (bc1 * (sq + eps))
    du_dv = np.abs(m_ref / bc1) / (2.0 * bc2 * np.maximum(sq, 1e-30) * (sq + eps) ** 2)
    du_dv = np.where(sq > 0, du_dv, 0.0)
    bound = 2.0 * lr * (du_dm * dm + du_dv * dv) + tol * np.abs(z_ref).max()
    err = np.abs(z_gpu.astype(np.float64) - z_ref)
    bad = err > bound
    assert not bad.any(), (int(bad.sum()), float(err[bad].max()), float(bound[bad].min()))


def run_lockstep(insts, N, hp, steps, step_fn=None):
    """Run `steps` steps of `insts` (one call of step_fn per step, tsat_step by
    default) and check every step against one oracle step taken from the GPU's
    FP32 state: status records, z / m / v after AdamW, the bits of the next
    step and the new normaliser.  Returns the last status."""
    if step_fn is None:
        step_fn = lambda st: ts.tsat_step(st.h, hp, 1, stop_on_sat=False)   # noqa: E731
    prob, st, cnfs = make(insts, N)
    ts.tsat_init(st.h, hp)
    offs = prob.var_offsets
    status = None
    for t in range(steps):
        s0 = snapshot(st)
        step_fn(st)
        s1 = snapshot(st)
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
            assert abs(x["loss"] - r["L"]) <= TOL_F32 * max(abs(r["L"]), 1e-30)
        live = ~frozen
        if live.any():
            assert_adamw_z(s1["z"][live], z[live], s1["m"][live], m[live], s1["v"][live], v[live], t, hp)
        X = binarize_like_gpu(s1["z"], s1["nu"], hp, t + 1, offs)
        np.testing.assert_array_equal(s1["X"][live], X[live])
        np.testing.assert_array_equal(s1["X"][frozen], s0["X"][frozen])
        nu_ref = oracle.nu_f32(s1["z"], hp.norm)
        assert np.all(np.abs(s1["nu"] - nu_ref) <= 2e-6 * np.abs(s1["z"]).mean(axis=1) + 2e-6 * np.abs(nu_ref))
    return status, prob, st, cnfs
