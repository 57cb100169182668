"""Seeded synthetic CNF generators (inputs only; no solver arithmetic).

Both the CUDA path and the FP64 oracle are fed from here.  Every random draw
comes from SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) used as a counter-based
hash, so a (seed, stream, index) triple always gives the same value on any
machine and numpy version.

Workloads (sizes as used by the tests and the benchmark):
  * planted random k-SAT: k distinct variables per clause drawn uniformly; the
    sign pattern is uniform over the 2^k - 1 patterns the planted assignment
    satisfies (the all-false pattern is excluded), so the planted assignment is
    a model and no variable is made pure;
  * structured mixed-length k-SAT: clause length 2 + Geometric(p) truncated to
    <= 16, 64 communities of variables with power-law (alpha = 2.2) occurrence
    weights, 80 % of clauses inside one community, planted signs as above;
  * batches of planted k-SAT with k uniform in 3..7 and n log-uniform.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Satisfiability thresholds of random k-SAT from the cavity method
# (Mertens, Mezard, Zecchina, Random Struct. Alg. 28, 2006), k = 3..7.
KSAT_THRESHOLD = {3: 4.267, 4: 9.931, 5: 21.117, 6: 43.37, 7: 87.79}


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _stream_seed(seed: int, stream: int) -> np.uint64:
    s = np.array([(seed * 0x100000001B3 + stream * 0xC2B2AE3D27D4EB4F) & (2**64 - 1)], np.uint64)
    return _mix(s)[0]


def u64(seed: int, stream: int, start: int, n: int) -> np.ndarray:
    """n SplitMix64 outputs of (seed, stream) at positions start..start+n-1."""
    base = _stream_seed(seed, stream)
    k = np.arange(start + 1, start + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(base + k * _GAMMA)


def uniform_int(seed, stream, start, n, hi) -> np.ndarray:
    """Integers in [0, hi) via the multiply-shift map of the top 32 bits."""
    x = u64(seed, stream, start, n) >> np.uint64(32)
    return ((x * np.uint64(hi)) >> np.uint64(32)).astype(np.int64)


def uniform01(seed, stream, start, n) -> np.ndarray:
    return (u64(seed, stream, start, n) >> np.uint64(11)).astype(np.float64) * (1.0 / 2**53)


@dataclass
class Instance:
    n_vars: int
    clause_ptr: np.ndarray          # int64 [C+1]
    lits: np.ndarray                # int32 [nnz], DIMACS signed, no zeros
    planted: np.ndarray             # uint8 [n_vars], a satisfying assignment
    meta: dict = field(default_factory=dict)

    @property
    def n_clauses(self) -> int:
        return int(self.clause_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.lits.shape[0])


def _distinct_rows(seed, stream, rows: np.ndarray, hi: int, draw) -> np.ndarray:
    """Redraw rows that repeat a variable until every row is duplicate-free."""
    k = rows.shape[1]
    ctr = rows.size
    for it in range(1000):
        srt = np.sort(rows, axis=1)
        bad = np.nonzero((srt[:, 1:] == srt[:, :-1]).any(axis=1))[0] if k > 1 else np.zeros(0, np.int64)
        if bad.size == 0:
            return rows
        rows[bad] = draw(seed, stream + 1 + it, ctr, bad.size * k).reshape(bad.size, k)
        ctr += bad.size * k
    raise RuntimeError("could not draw distinct variables")


def _planted_signs(seed, stream, vars_: np.ndarray, planted: np.ndarray, lens=None) -> np.ndarray:
    """Signs such that the planted assignment satisfies every clause.

    For a clause of length L draw t uniform in [1, 2^L - 1]; bit j of t says
    whether literal j is true under the planted assignment."""
    if lens is None:
        C, k = vars_.shape
        t = 1 + uniform_int(seed, stream, 0, C, (1 << k) - 1)
        bits = ((t[:, None] >> np.arange(k)[None, :]) & 1).astype(np.uint8)
        neg = planted[vars_] ^ bits
        return neg.astype(np.uint8)
    # ragged: vars_ is flat, lens gives the clause lengths
    C = lens.shape[0]
    span = (np.left_shift(np.int64(1), lens.astype(np.int64)) - 1)
    r = u64(seed, stream, 0, C) >> np.uint64(32)
    t = 1 + ((r * span.astype(np.uint64)) >> np.uint64(32)).astype(np.int64)
    pos = np.arange(vars_.shape[0]) - np.repeat(np.concatenate([[0], np.cumsum(lens)[:-1]]), lens)
    bits = ((np.repeat(t, lens) >> pos) & 1).astype(np.uint8)
    return (planted[vars_] ^ bits).astype(np.uint8)


def _dimacs(vars_flat: np.ndarray, neg_flat: np.ndarray) -> np.ndarray:
    v = vars_flat.astype(np.int64) + 1
    return np.where(neg_flat.astype(bool), -v, v).astype(np.int32)


def planted_ksat(n: int, m: int, k: int, seed: int) -> Instance:
    """Uniform random k-SAT with a planted model (Sec. V workloads stand-in)."""
    planted = (u64(seed, 1, 0, n) >> np.uint64(63)).astype(np.uint8)
    rows = uniform_int(seed, 2, 0, m * k, n).reshape(m, k)
    rows = _distinct_rows(seed, 100, rows, n, lambda s, st, c0, cnt: uniform_int(s, st, c0, cnt, n))
    neg = _planted_signs(seed, 3, rows, planted)
    ptr = np.arange(m + 1, dtype=np.int64) * k
    return Instance(n, ptr, _dimacs(rows.reshape(-1), neg.reshape(-1)), planted,
                    dict(kind="planted", k=k, ratio=m / n, seed=seed))


def structured_mixed(n: int, m: int, seed: int, communities: int = 64, alpha: float = 2.2,
                     cross: float = 0.2, p_geom: float = 0.4, lmax: int = 16) -> Instance:
    """Mixed-length planted k-SAT with community structure and power-law
    occurrences (clause length 2 + Geometric(p_geom) <= lmax)."""
    planted = (u64(seed, 1, 0, n) >> np.uint64(63)).astype(np.uint8)
    # clause lengths: 2 + G, G = number of failures before the first success
    lens = np.zeros(m, np.int64)
    todo = np.arange(m)
    ctr = 0
    while todo.size:
        u = uniform01(seed, 5, ctr, todo.size)
        ctr += todo.size
        g = np.floor(np.log1p(-u) / math.log1p(-p_geom)).astype(np.int64)
        L = 2 + g
        ok = L <= lmax
        lens[todo[ok]] = L[ok]
        todo = todo[~ok]
    perm = np.argsort(u64(seed, 6, 0, n), kind="stable")       # random relabelling
    csize = n // communities
    rank = np.arange(1, csize + 1, dtype=np.float64)
    w = rank ** (-1.0 / (alpha - 1.0))
    cdf_local = np.cumsum(w) / w.sum()
    nnz = int(lens.sum())
    which = uniform_int(seed, 7, 0, m, communities)
    is_cross = uniform01(seed, 8, 0, m) < cross
    total_w = np.tile(w, communities)
    cdf_global = np.cumsum(total_w) / total_w.sum()
    owner = np.repeat(np.arange(m), lens)

    def draw_vars(stream, start, idx_flat):
        u = uniform01(seed, stream, start, idx_flat.size)
        cl = owner[idx_flat]
        loc = np.minimum(np.searchsorted(cdf_local, u, side="right"), csize - 1)
        glob = np.minimum(np.searchsorted(cdf_global, u, side="right"), csize * communities - 1)
        slot = np.where(is_cross[cl], glob, which[cl] * csize + loc)
        return perm[slot]

    flat = draw_vars(9, 0, np.arange(nnz))
    offs = np.concatenate([[0], np.cumsum(lens)])
    ctr = nnz
    for it in range(200):
        # duplicates inside a clause: sort (clause, var) pairs and compare neighbours
        key = owner * np.int64(n) + flat
        order = np.argsort(key, kind="stable")
        sk = key[order]
        dup_sorted = np.zeros(nnz, bool)
        dup_sorted[1:] = sk[1:] == sk[:-1]
        dup = np.zeros(nnz, bool)
        dup[order[dup_sorted]] = True
        bad = np.nonzero(dup)[0]
        if bad.size == 0:
            break
        flat[bad] = draw_vars(10 + it, ctr, bad)
        ctr += bad.size
    else:
        raise RuntimeError("could not draw distinct variables")
    neg = _planted_signs(seed, 4, flat, planted, lens=lens)
    return Instance(n, offs.astype(np.int64), _dimacs(flat, neg), planted,
                    dict(kind="structured", communities=communities, alpha=alpha, seed=seed))


def batch_ksat(n_inst: int, seed: int, n_lo: int = 200, n_hi: int = 50_000, k_lo: int = 3,
               k_hi: int = 7, ratio_scale: float = 0.9, ks=None) -> list:
    """Planted random k-SAT instances of uneven size: k uniform in
    [k_lo, k_hi] (or drawn from ``ks``), n log-uniform in [n_lo, n_hi],
    m = round(ratio_scale * threshold_k * n)."""
    u = uniform01(seed, 11, 0, n_inst)
    kk = uniform_int(seed, 12, 0, n_inst, (k_hi - k_lo + 1)) + k_lo
    if ks is not None:
        kk = np.asarray(ks)[uniform_int(seed, 13, 0, n_inst, len(ks))]

    def one(j):
        n = int(round(math.exp(math.log(n_lo) + u[j] * (math.log(n_hi) - math.log(n_lo)))))
        k = int(kk[j])
        m = int(round(ratio_scale * KSAT_THRESHOLD[k] * n))
        return planted_ksat(n, m, k, seed * 1_000_003 + j + 1)

    # each instance depends only on its own seed; numpy releases the GIL in
    # the array work, so threads give the same list faster
    with ThreadPoolExecutor(max(1, min(32, os.cpu_count() or 1))) as ex:
        return list(ex.map(one, range(n_inst)))


def tiny_random(n: int, m: int, seed: int, kmin: int = 1, kmax: int = 4, dup: bool = True) -> Instance:
    """Small unstructured CNF (any satisfiability), clause lengths uniform in
    [kmin, kmax], variables drawn with repetition (duplicate literals and
    tautologies allowed when ``dup``); used for brute-force pins."""
    lens = uniform_int(seed, 21, 0, m, kmax - kmin + 1) + kmin
    nnz = int(lens.sum())
    v = uniform_int(seed, 22, 0, nnz, n)
    s = (u64(seed, 23, 0, nnz) >> np.uint64(63)).astype(np.uint8)
    if not dup:
        pass
    ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    return Instance(n, ptr, _dimacs(v, s), np.zeros(n, np.uint8), dict(kind="tiny", seed=seed))
