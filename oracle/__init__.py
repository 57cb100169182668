"""FP64 CPU oracle for the gradient-guided SAT method (TurboSAT, arXiv 2511.07737).

TEST INFRASTRUCTURE ONLY: this package is the slow, obviously correct reference
the CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it; the library never does.
It shares no code with the CUDA path.

The arithmetic lives in ``oracle.c`` (compiled by :func:`build` into
``liboracle.so``); this module only marshals numpy arrays.  ``mpnn.py`` holds
the FP64 numpy oracle of the learned proposer.

Parity status per function (the pins live in ``tests/test_oracle_*.py``):
  parse / check / result_matrix : brute force over all assignments, dense
                                  integer matmul, Fig. 2 fragments
  smoothmin                     : closed forms, tau -> inf limit, FD
  objective (STE and relaxed)   : FD on the smooth surrogate / direct FD
  normalize(+_backward)         : FD through the surrogate
  nu_f32                        : exact means of dyadic FP32 rows (closed
                                  form), the +-1e-12 guard cases, FP64 (not
                                  FP32) accumulation, permutation / scaling
  lr / adamw                    : torch.optim.AdamW + LambdaLR in FP64,
                                  the schedule values stated in Sec. IV-A
  philox4x32_10                 : published answer vectors (SC'11 / Random123)
  init_normal                   : moments of the Irwin-Hall law
  binarize_f32                  : deterministic mode vs sign rule, T -> 0
                                  reduction to it, Philox mode frequency
  best_sample / topk            : brute force on small arrays
  partial_k                     : the sizes of the top-k rule at small,
                                  round and just-above-round V
  step                          : equal to the pinned pieces composed by
                                  hand; the mixing reading's closed forms
                                  (best sample kept, the rest averaged,
                                  moments zeroed, first AdamW step after it)
  mpnn.forward                  : closed form of a selector network on a
                                  hand-sized graph (feature vector, block
                                  order [h; a; h_neg], output head), a dense
                                  incidence restatement, FD of the backward
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

NORM_SIGNED_MEAN, NORM_ABSMEAN, NORM_NONE = 0, 1, 2
BIN_DET, BIN_PHILOX = 0, 1


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, FP64, OpenMP, no contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i32, i64, u64, f64, f32 = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                   ctypes.c_double, ctypes.c_float)
        sig = {
            "orc_num_threads": (ctypes.c_int, []),
            "orc_set_threads": (None, [ctypes.c_int]),
            "orc_parse": (ctypes.c_int, [i32, i32, P, P, P, P, P]),
            "orc_check": (None, [i32, i32, P, P, P, i32, P, P, P]),
            "orc_result_matrix": (None, [i32, i32, P, P, P, i32, P, P]),
            "orc_smoothmin": (None, [i32, i32, P, f64, P, P]),
            "orc_objective": (ctypes.c_int, [i32, i32, P, P, P, i32, i32, P, P, f64, P, P, P, P]),
            "orc_normalize": (None, [i32, i32, P, i32, P, P]),
            "orc_normalize_backward": (None, [i32, i32, P, P, P, i32, P]),
            "orc_lr": (f64, [i64, f64, f64, i32, i32, f64]),
            "orc_adamw": (None, [i64, P, P, P, P, i64, f64, f64, f64, f64, f64]),
            "orc_philox4x32_10": (None, [P, P, P]),
            "orc_init_normal": (None, [i32, i32, u64, P, f32, P]),
            "orc_nu_f32": (None, [i32, i32, P, i32, P]),
            "orc_binarize_f32": (None, [i32, i32, P, P, i32, f32, u64, i64, P]),
            "orc_step": (ctypes.c_int, [i32, i32, P, P, P, i32, P, i64, P, P, P, P, P,
                                        P, P, P, P, P, P]),
            "orc_best_sample": (i32, [i32, P]),
            "orc_partial_k": (i32, [i32]),
            "orc_topk_confident": (None, [i32, P, i32, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def num_threads() -> int:
    return int(lib().orc_num_threads())


class CNF:
    """Problem matrix P of Sec. III-A as per-clause literal lists.

    Built from DIMACS-signed literals (``lits``, no zeros) and clause offsets
    ``clause_ptr`` (length C+1).  Duplicate literals inside a clause are kept
    once (P is 0/1); empty clauses and out-of-range literals are errors.
    """

    def __init__(self, n_vars: int, clause_ptr, lits):
        clause_ptr = _c(clause_ptr, np.int64)
        lits = _c(lits, np.int32)
        self.V = int(n_vars)
        self.C = int(clause_ptr.shape[0] - 1)
        ocptr = np.zeros(self.C + 1, np.int64)
        ovar = np.zeros(max(1, lits.shape[0]), np.int32)
        oneg = np.zeros(max(1, lits.shape[0]), np.uint8)
        rc = lib().orc_parse(self.V, self.C, _p(clause_ptr), _p(lits), _p(ocptr), _p(ovar), _p(oneg))
        if rc != 0:
            raise ValueError(f"oracle parse failed with status {rc}")
        nnz = int(ocptr[-1])
        self.cptr, self.var, self.neg = ocptr, ovar[:nnz].copy(), oneg[:nnz].copy()
        self.nnz = nnz
        self.lens = np.diff(ocptr)
        self.lmax = int(self.lens.max())

    def _args(self):
        return (self.V, self.C, _p(self.cptr), _p(self.var), _p(self.neg))


def check(cnf: CNF, X):
    """Exact satisfaction check: (unsat[N] int32, satmask[ceil(N/32)] uint32)."""
    X = _c(X, np.uint8)
    N = X.shape[1]
    unsat = np.zeros(N, np.int32)
    sm = np.zeros((N + 31) // 32, np.uint32)
    lib().orc_check(*cnf._args(), N, _p(X), _p(unsat), _p(sm))
    return unsat, sm


def result_matrix(cnf: CNF, X):
    """Eq. 1: R = P A as a C x N int32 matrix."""
    X = _c(X, np.uint8)
    N = X.shape[1]
    R = np.zeros((cnf.C, N), np.int32)
    lib().orc_result_matrix(*cnf._args(), N, _p(X), _p(R))
    return R


def smoothmin(R, tau: float, grad: bool = False):
    """Eq. 4 column-wise on a real C x N matrix; optionally dS/dR."""
    R = _c(R, np.float64)
    C, N = R.shape
    S = np.zeros(N)
    d = np.zeros((C, N)) if grad else None
    lib().orc_smoothmin(C, N, _p(R), float(tau), _p(S), _p(d))
    return (S, d) if grad else S


def objective(cnf: CNF, *, X=None, zt=None, tau: float = 1.0, grad: bool = True):
    """S[N], L, G[V,N] (dL/d normalised assignment), unsat[N] (STE only).

    ``X`` (0/1, V x N) selects the paper's STE layer; ``zt`` (real, V x N)
    selects the relaxed sigmoid layer."""
    relaxed = X is None
    if relaxed:
        zt = _c(zt, np.float64)
        N = zt.shape[1]
    else:
        X = _c(X, np.uint8)
        N = X.shape[1]
    S = np.zeros(N)
    L = np.zeros(1)
    G = np.zeros((cnf.V, N)) if grad else None
    unsat = np.zeros(N, np.int32)
    rc = lib().orc_objective(*cnf._args(), N, int(relaxed), _p(X), _p(zt), float(tau),
                             _p(S), _p(L), _p(G), _p(unsat))
    if rc != 0:
        raise RuntimeError(f"oracle objective failed {rc}")
    return S, float(L[0]), G, (None if relaxed else unsat)


def normalize(z, mode: int):
    z = _c(z, np.float64)
    V, N = z.shape
    nu = np.zeros(V)
    zt = np.zeros((V, N))
    lib().orc_normalize(V, N, _p(z), int(mode), _p(nu), _p(zt))
    return nu, zt


def normalize_backward(z, nu, G, mode: int):
    z = _c(z, np.float64)
    V, N = z.shape
    g = np.zeros((V, N))
    lib().orc_normalize_backward(V, N, _p(z), _p(_c(nu, np.float64)), _p(_c(G, np.float64)),
                                 int(mode), _p(g))
    return g


def lr_at(t: int, lr0=0.1, factor=0.1, period=30, restart=360, floor=1e-15) -> float:
    return float(lib().orc_lr(int(t), lr0, factor, int(period), int(restart), floor))


def adamw(z, m, v, g, step: int, lr: float, b1=0.9, b2=0.999, eps=1e-8, wd=0.01):
    """In-place AdamW on FP64 arrays (PyTorch semantics, 1-based step)."""
    for a in (z, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = _c(g, np.float64)
    lib().orc_adamw(z.size, _p(z), _p(m), _p(v), _p(g), int(step), lr, b1, b2, eps, wd)


def philox4x32_10(ctr, key):
    c = _c(ctr, np.uint32)
    k = _c(key, np.uint32)
    o = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(o))
    return o


def init_normal(V: int, N: int, seed: int, logits=None, scale: float = 1.0):
    z = np.zeros((V, N), np.float32)
    lg = None if logits is None else _c(logits, np.float32)
    lib().orc_init_normal(V, N, int(seed), _p(lg), float(scale), _p(z))
    return z


def nu_f32(z, mode: int):
    z = _c(z, np.float32)
    V, N = z.shape
    nu = np.zeros(V)
    lib().orc_nu_f32(V, N, _p(z), int(mode), _p(nu))
    return nu


def binarize_f32(z, nu, mode: int, c: float = 0.25, seed: int = 0, t: int = 0):
    """Eq. 2 (mode 0) or the Philox-sampled form (mode 1), decided in FP32."""
    z = _c(z, np.float32)
    nu = _c(nu, np.float32)
    V, N = z.shape
    X = np.zeros((V, N), np.uint8)
    lib().orc_binarize_f32(V, N, _p(z), _p(nu), int(mode), float(c), int(seed), int(t), _p(X))
    return X


class HParams(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("lr0", ctypes.c_double),
                ("lr_factor", ctypes.c_double), ("lr_floor", ctypes.c_double),
                ("decay_period", ctypes.c_int32), ("restart_period", ctypes.c_int32),
                ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double), ("weight_decay", ctypes.c_double),
                ("norm", ctypes.c_int32), ("relaxed", ctypes.c_int32),
                ("mix", ctypes.c_int32), ("pad", ctypes.c_int32)]


def hparams(**kw) -> HParams:
    d = dict(tau=1.0, lr0=0.1, lr_factor=0.1, lr_floor=1e-15, decay_period=30,
             restart_period=360, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.01,
             norm=NORM_SIGNED_MEAN, relaxed=0, mix=0)
    d.update(kw)
    return HParams(**d)


def step(cnf: CNF, hp: HParams, t: int, z, m, v, X=None, nu_in=None):
    """One optimisation step in FP64.  z, m, v (float64, V x N) are updated
    in place.  Returns dict(S, L, G, g, nu_next, unsat)."""
    for a in (z, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    V, N = z.shape
    Xc = None if X is None else _c(X, np.uint8)
    nu_c = None if nu_in is None else _c(nu_in, np.float64)
    S = np.zeros(N)
    L = np.zeros(1)
    G = np.zeros((V, N))
    g = np.zeros((V, N))
    nu_next = np.zeros(V)
    unsat = np.zeros(N, np.int32)
    rc = lib().orc_step(*cnf._args(), N, ctypes.byref(hp), int(t), _p(z), _p(m), _p(v),
                        _p(Xc), _p(nu_c), _p(S), _p(L), _p(G), _p(g), _p(nu_next), _p(unsat))
    if rc != 0:
        raise RuntimeError(f"oracle step failed {rc}")
    return dict(S=S, L=float(L[0]), G=G, g=g, nu_next=nu_next, unsat=unsat)


def best_sample(unsat) -> int:
    u = _c(unsat, np.int32)
    return int(lib().orc_best_sample(u.shape[0], _p(u)))


def partial_k(V: int) -> int:
    return int(lib().orc_partial_k(int(V)))


def topk_confident(absG, k: int):
    a = _c(absG, np.float64)
    out = np.zeros(k, np.int32)
    lib().orc_topk_confident(a.shape[0], _p(a), int(k), _p(out))
    return out
