"""ctypes binding of the C ABI in ``include/turbosat.h`` (``libturbosat.so``).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  Device buffers are torch tensors (the library never allocates device
memory); streams are torch CUDA streams.  The functions keep the C names.

``Problem`` and ``State`` below only tie a library handle to the torch tensor
that backs it, so that the buffer outlives the handle.
"""
from __future__ import annotations

import ctypes
import os
from typing import Sequence

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libturbosat.so")

TSAT_OK = 0
NORM_SIGNED_MEAN, NORM_ABSMEAN, NORM_NONE = 0, 1, 2
BIN_DET, BIN_PHILOX = 0, 1
LAYER_STE, LAYER_RELAXED = 0, 1
DTYPE_F32, DTYPE_BF16 = 0, 1
MAX_PARTIAL_K = 16384


class TsatError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: status {status} ({strerror(status)}): {last_error()}")
        self.status = status


class tsat_hparams(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_float), ("lr0", ctypes.c_float), ("lr_factor", ctypes.c_float),
                ("lr_floor", ctypes.c_float), ("decay_period", ctypes.c_int32),
                ("restart_period", ctypes.c_int32), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_float), ("weight_decay", ctypes.c_float), ("norm", ctypes.c_int32),
                ("binarize", ctypes.c_int32), ("bin_temp", ctypes.c_float), ("layer", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("mix_restart", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class tsat_cnf_desc(ctypes.Structure):
    _fields_ = [("n_vars", ctypes.c_int32), ("n_clauses", ctypes.c_int32),
                ("h_clause_ptr", ctypes.c_void_p), ("h_lits", ctypes.c_void_p)]


class tsat_inst_status(ctypes.Structure):
    _fields_ = [("found", ctypes.c_int32), ("found_sample", ctypes.c_int32), ("found_step", ctypes.c_int64),
                ("min_unsat", ctypes.c_int32), ("best_sample", ctypes.c_int32), ("loss", ctypes.c_float),
                ("pad", ctypes.c_float)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(the CUDA library has no fallback)")
        L = ctypes.CDLL(LIB_PATH)
        P, i32, i64, f32, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_size_t
        sigs = {
            "tsat_strerror": (ctypes.c_char_p, [ctypes.c_int]),
            "tsat_last_error": (ctypes.c_char_p, []),
            "tsat_hparams_default": (None, [P]),
            "tsat_problem_bytes": (ctypes.c_int, [i32, P, P]),
            "tsat_load_batch": (ctypes.c_int, [i32, P, P, sz, P, P]),
            "tsat_load": (ctypes.c_int, [i32, i32, P, P, P, sz, P, P]),
            "tsat_load_batch_ex": (ctypes.c_int, [i32, P, ctypes.c_uint32, P, sz, P, P]),
            "tsat_problem_free": (None, [P]),
            "tsat_problem_info": (ctypes.c_int, [P, P]),
            "tsat_problem_csr": (ctypes.c_int, [P, P, P]),
            "tsat_state_bytes": (ctypes.c_int, [P, i32, i32, i32, P]),
            "tsat_state_create": (ctypes.c_int, [P, P, sz, i32, i32, i32, P]),
            "tsat_state_free": (None, [P]),
            "tsat_init": (ctypes.c_int, [P, P, P, f32, P]),
            "tsat_step": (ctypes.c_int, [P, P, i32, i32, P]),
            "tsat_step_prepare": (ctypes.c_int, [P, P, i32, i32]),
            "tsat_profile_step": (ctypes.c_int, [P, P, i32, P]),
            "tsat_evaluate": (ctypes.c_int, [P, P, P, P, P, P]),
            "tsat_histogram": (ctypes.c_int, [P, P, P]),
            "tsat_step_persistent": (ctypes.c_int, [P, P, i32, i32, P]),
            "tsat_step_clustered": (ctypes.c_int, [P, P, i32, i32, P]),
            "tsat_set_persist_blocks": (ctypes.c_int, [P, i32]),
            "tsat_persist_blocks": (ctypes.c_int, [P, P, P]),
            "tsat_autotune_persistent": (ctypes.c_int, [P, P, P, sz, i32, P, P]),
            "tsat_best": (ctypes.c_int, [P, P, i32, i32, P, P, P, P, P, P, P]),
            "tsat_partial_k": (i32, [i32]),
            "tsat_status": (ctypes.c_int, [P, P, P, P, P]),
            "tsat_state_views": (ctypes.c_int, [P, P, P, P, P, P, P, P]),
            "tsat_forward": (ctypes.c_int, [P, P, P, i64, P, P, P]),
            "tsat_backward": (ctypes.c_int, [P, P, P, f32, P, P]),
            "tsat_problem_set_instance_ids": (ctypes.c_int, [P, P, P]),
            "tsat_state_set_shard": (ctypes.c_int, [P, i32, i32]),
            "tsat_shard_init": (ctypes.c_int, [P, P, P, P]),
            "tsat_shard_grad": (ctypes.c_int, [P, P, P, P, P]),
            "tsat_shard_update": (ctypes.c_int, [P, P, P, P, P, P]),
            "tsat_shard_finish": (ctypes.c_int, [P, P, P, P]),
            "tsat_autotune_bytes": (ctypes.c_int, [P, P]),
            "tsat_tuning_space": (ctypes.c_int, [P, P, P, P]),
            "tsat_autotune": (ctypes.c_int, [P, P, P, sz, P, P]),
            "tsat_get_tuning": (ctypes.c_int, [P, P]),
            "tsat_set_tuning": (ctypes.c_int, [P, P]),
            "tsat_launches_per_step": (i32, [P]),
            "tsat_evaluate_bits_noalloc": (ctypes.c_int, [P, P, i32, f32, P, P, P, P]),
            "tsat_mpnn_param_count": (i32, []),
            "tsat_mpnn_workspace_bytes": (ctypes.c_int, [P, P]),
            "tsat_mpnn_init": (ctypes.c_int, [P, ctypes.c_uint64, P]),
            "tsat_mpnn_forward": (ctypes.c_int, [P, P, P, sz, P, P]),
            "tsat_mpnn_loss_grad": (ctypes.c_int, [P, P, P, sz, P, P, P, P, P]),
            "tsat_mpnn_adam": (ctypes.c_int, [P, P, P, P, i64, f32, P]),
            "tsat_mpnn_status": (ctypes.c_int, [P, P, sz, P]),
        }
        for name, (res, args) in sigs.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def strerror(status: int) -> str:
    return lib().tsat_strerror(int(status)).decode()


def last_error() -> str:
    return lib().tsat_last_error().decode()


def _ck(rc: int, what: str) -> int:
    if rc < 0:
        raise TsatError(rc, what)
    return rc


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t) -> ctypes.c_void_p:
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return ctypes.c_void_p(t.data_ptr())
    return t.ctypes.data_as(ctypes.c_void_p)


def hparams(**kw) -> tsat_hparams:
    """tsat_hparams_default() with keyword overrides."""
    hp = tsat_hparams()
    lib().tsat_hparams_default(ctypes.byref(hp))
    for k, v in kw.items():
        if not hasattr(hp, k):
            raise KeyError(k)
        setattr(hp, k, v)
    return hp


def _descs(instances):
    keep = []
    arr = (tsat_cnf_desc * len(instances))()
    for j, inst in enumerate(instances):
        n_vars, ptr, lits = inst
        ptr = np.ascontiguousarray(ptr, dtype=np.int64)
        lits = np.ascontiguousarray(lits, dtype=np.int32)
        keep += [ptr, lits]
        arr[j] = tsat_cnf_desc(int(n_vars), int(ptr.shape[0] - 1), ptr.ctypes.data, lits.ctypes.data)
    return arr, keep


def tsat_problem_bytes(instances) -> int:
    """instances: sequence of (n_vars, clause_ptr int64[C+1], lits int32 DIMACS)."""
    arr, keep = _descs(instances)
    out = ctypes.c_size_t(0)
    _ck(lib().tsat_problem_bytes(len(instances), arr, ctypes.byref(out)), "tsat_problem_bytes")
    return int(out.value)


LOAD_CLAUSE_LOCALITY = 1


def tsat_load_batch(instances, ws: torch.Tensor, stream=None, flags: int = 0) -> ctypes.c_void_p:
    arr, keep = _descs(instances)
    h = ctypes.c_void_p()
    _ck(lib().tsat_load_batch_ex(len(instances), arr, int(flags), _ptr(ws), ws.numel() * ws.element_size(),
                                 _stream(stream), ctypes.byref(h)), "tsat_load_batch")
    return h


def tsat_problem_info(h) -> dict:
    a = (ctypes.c_int64 * 8)()
    _ck(lib().tsat_problem_info(h, a), "tsat_problem_info")
    return dict(n_inst=a[0], n_vars=a[1], n_clauses=a[2], nnz=a[3], lmax=a[4], n_items=a[5], xrec_words=a[6],
                ws_bytes=a[7])


def tsat_problem_csr(h):
    info = tsat_problem_info(h)
    cptr = np.zeros(info["n_clauses"] + 1, np.int32)
    clit = np.zeros(max(1, info["nnz"]), np.int32)
    _ck(lib().tsat_problem_csr(h, _ptr(cptr), _ptr(clit)), "tsat_problem_csr")
    return cptr, clit[: info["nnz"]]


def tsat_problem_set_instance_ids(h, ids, stream=None):
    """Per-instance random-stream ids (default: position in the loaded batch)."""
    a = np.ascontiguousarray(ids, dtype=np.int32)
    _ck(lib().tsat_problem_set_instance_ids(h, _ptr(a), _stream(stream)), "tsat_problem_set_instance_ids")


def tsat_state_set_shard(s, sample_base: int, n_total: int):
    _ck(lib().tsat_state_set_shard(s, int(sample_base), int(n_total)), "tsat_state_set_shard")


def tsat_shard_init(s, hp, rowsum: torch.Tensor, stream=None):
    _ck(lib().tsat_shard_init(s, ctypes.byref(hp), _ptr(rowsum), _stream(stream)), "tsat_shard_init")


def tsat_shard_grad(s, hp, G: torch.Tensor, rowdot: torch.Tensor, stream=None):
    _ck(lib().tsat_shard_grad(s, ctypes.byref(hp), _ptr(G), _ptr(rowdot), _stream(stream)), "tsat_shard_grad")


def tsat_shard_update(s, hp, G: torch.Tensor, rowdot_total: torch.Tensor, rowsum: torch.Tensor, stream=None):
    _ck(lib().tsat_shard_update(s, ctypes.byref(hp), _ptr(G), _ptr(rowdot_total), _ptr(rowsum), _stream(stream)),
        "tsat_shard_update")


def tsat_shard_finish(s, hp, rowsum_total: torch.Tensor, stream=None):
    _ck(lib().tsat_shard_finish(s, ctypes.byref(hp), _ptr(rowsum_total), _stream(stream)), "tsat_shard_finish")


def tsat_state_bytes(h, n_samples: int, layer: int = LAYER_STE, dtype: int = DTYPE_F32) -> int:
    out = ctypes.c_size_t(0)
    _ck(lib().tsat_state_bytes(h, int(n_samples), int(layer), int(dtype), ctypes.byref(out)), "tsat_state_bytes")
    return int(out.value)


def tsat_state_create(h, state: torch.Tensor, n_samples: int, layer: int = LAYER_STE, dtype: int = DTYPE_F32):
    s = ctypes.c_void_p()
    _ck(lib().tsat_state_create(h, _ptr(state), state.numel() * state.element_size(), int(n_samples), int(layer),
                                int(dtype), ctypes.byref(s)), "tsat_state_create")
    return s


def tsat_init(s, hp: tsat_hparams, logits: torch.Tensor | None = None, scale: float = 1.0, stream=None):
    _ck(lib().tsat_init(s, ctypes.byref(hp), _ptr(logits), float(scale), _stream(stream)), "tsat_init")


def tsat_step(s, hp: tsat_hparams, n_steps: int, stop_on_sat: bool = True, stream=None):
    _ck(lib().tsat_step(s, ctypes.byref(hp), int(n_steps), int(bool(stop_on_sat)), _stream(stream)), "tsat_step")


def tsat_step_persistent(s, hp: tsat_hparams, n_steps: int, stop_on_sat: bool = True, stream=None):
    """n_steps steps of a batch of small instances in one launch (one block, or a
    cluster of blocks, per instance)."""
    _ck(lib().tsat_step_persistent(s, ctypes.byref(hp), int(n_steps), int(bool(stop_on_sat)), _stream(stream)),
        "tsat_step_persistent")


def tsat_set_persist_blocks(s, blocks: int):
    """Blocks per instance of tsat_step_persistent: 0 automatic, 1, 2, 4 or 8."""
    _ck(lib().tsat_set_persist_blocks(s, int(blocks)), "tsat_set_persist_blocks")


def tsat_persist_blocks(s, with_residency: bool = False):
    """Blocks per instance of the next tsat_step_persistent call (and, with
    with_residency, whether they keep z, m, v in shared memory)."""
    out, res = ctypes.c_int32(0), ctypes.c_int32(0)
    _ck(lib().tsat_persist_blocks(s, ctypes.byref(out), ctypes.byref(res)), "tsat_persist_blocks")
    return (int(out.value), bool(res.value)) if with_residency else int(out.value)


def tsat_autotune_persistent(s, hp: tsat_hparams, n_steps: int = 50, stream=None) -> int:
    """Times the persistent solver with each candidate number of blocks per
    instance from the current state, keeps the fastest and returns it (the
    state is left as it was)."""
    nbytes = tsat_autotune_bytes(s)
    snap = torch.empty(max(nbytes, 1), dtype=torch.uint8, device="cuda")
    out = ctypes.c_int32(0)
    _ck(lib().tsat_autotune_persistent(s, ctypes.byref(hp), _ptr(snap), nbytes, int(n_steps), _stream(stream),
                                       ctypes.byref(out)), "tsat_autotune_persistent")
    torch.cuda.synchronize()
    return int(out.value)


def tsat_step_clustered(s, hp: tsat_hparams, n_steps: int, stop_on_sat: bool = True, stream=None):
    """n_steps steps of a batch of larger instances in one launch of thread-block clusters."""
    _ck(lib().tsat_step_clustered(s, ctypes.byref(hp), int(n_steps), int(bool(stop_on_sat)), _stream(stream)),
        "tsat_step_clustered")


def tsat_step_prepare(s, hp: tsat_hparams, n_steps: int, stop_on_sat: bool = True):
    _ck(lib().tsat_step_prepare(s, ctypes.byref(hp), int(n_steps), int(bool(stop_on_sat))), "tsat_step_prepare")


def tsat_profile_step(s, hp: tsat_hparams, n_steps: int) -> list:
    a = (ctypes.c_float * 4)()
    _ck(lib().tsat_profile_step(s, ctypes.byref(hp), int(n_steps), a), "tsat_profile_step")
    return [float(x) for x in a]


def tsat_evaluate(s, hp, unsat: torch.Tensor, satmask: torch.Tensor, loss: torch.Tensor | None = None, stream=None):
    _ck(lib().tsat_evaluate(s, ctypes.byref(hp), _ptr(unsat), _ptr(satmask), _ptr(loss), _stream(stream)),
        "tsat_evaluate")


def tsat_histogram(s, hist: torch.Tensor, stream=None):
    """Per-sample histograms of R = P A at the current bits, int32 [n_inst][lmax+1][N]."""
    _ck(lib().tsat_histogram(s, _ptr(hist), _stream(stream)), "tsat_histogram")


def tsat_evaluate_bits_noalloc(h, bits: torch.Tensor, n_samples: int, tau: float, unsat: torch.Tensor,
                               satmask: torch.Tensor, loss: torch.Tensor | None = None, stream=None):
    """Evaluation of a caller-supplied bit matrix with no device allocation (see the C header)."""
    _ck(lib().tsat_evaluate_bits_noalloc(h, _ptr(bits), int(n_samples), float(tau), _ptr(unsat), _ptr(satmask),
                                         _ptr(loss), _stream(stream)), "tsat_evaluate_bits_noalloc")


def tsat_partial_k(n_vars: int) -> int:
    return int(lib().tsat_partial_k(int(n_vars)))


def tsat_best(s, hp, inst: int, n_vars: int, k: int | None = None, stream=None) -> dict:
    if k is None:
        k = tsat_partial_k(n_vars)
    bits = np.zeros((n_vars + 31) // 32, np.uint32)
    unsat = ctypes.c_int32(0)
    sample = ctypes.c_int32(0)
    ready = ctypes.c_int32(0)
    pv = np.zeros(k, np.int32)
    pval = np.zeros(k, np.uint8)
    rc = _ck(lib().tsat_best(s, ctypes.byref(hp), int(inst), int(k), _ptr(bits), ctypes.byref(unsat),
                             ctypes.byref(sample), _ptr(pv), _ptr(pval), ctypes.byref(ready), _stream(stream)),
             "tsat_best")
    assign = np.unpackbits(bits.view(np.uint8), bitorder="little")[:n_vars]
    return dict(complete=bool(rc), unsat=int(unsat.value), sample=int(sample.value), assignment=assign,
                part_var=pv, part_val=pval, ready=bool(ready.value))


def tsat_status(s, n_inst: int, stream=None) -> dict:
    step = ctypes.c_int64(0)
    done = ctypes.c_int32(0)
    arr = (tsat_inst_status * n_inst)()
    _ck(lib().tsat_status(s, ctypes.byref(step), ctypes.byref(done), arr, _stream(stream)), "tsat_status")
    insts = [dict(found=a.found, found_sample=a.found_sample, found_step=a.found_step, min_unsat=a.min_unsat,
                  best_sample=a.best_sample, loss=a.loss) for a in arr]
    return dict(step=int(step.value), all_done=bool(done.value), inst=insts)


def tsat_state_views(s) -> dict:
    ptrs = [ctypes.c_void_p() for _ in range(7)]
    _ck(lib().tsat_state_views(s, *[ctypes.byref(p) for p in ptrs]), "tsat_state_views")
    names = ["z", "m", "v", "bits", "nu", "gamma", "hist"]
    return {n: (p.value or 0) for n, p in zip(names, ptrs)}


def tsat_forward(s, hp, z: torch.Tensor, t_bin: int, S_out: torch.Tensor, loss_out: torch.Tensor, stream=None):
    _ck(lib().tsat_forward(s, ctypes.byref(hp), _ptr(z), int(t_bin), _ptr(S_out), _ptr(loss_out), _stream(stream)),
        "tsat_forward")


def tsat_backward(s, hp, z: torch.Tensor, dL: float, grad_out: torch.Tensor, stream=None):
    _ck(lib().tsat_backward(s, ctypes.byref(hp), _ptr(z), float(dL), _ptr(grad_out), _stream(stream)),
        "tsat_backward")


def tsat_tuning_space(s) -> dict:
    """The candidate launch shapes tsat_autotune tries on this state."""
    a, b, c = (ctypes.c_int32 * 4)(), (ctypes.c_int32 * 5)(), (ctypes.c_int32 * 3)()
    _ck(lib().tsat_tuning_space(s, a, b, c), "tsat_tuning_space")
    return dict(fwd_items=list(a), upd_blocks_per_sm=list(b), upd_rows_per_item=list(c))


def tsat_autotune_bytes(s) -> int:
    out = ctypes.c_size_t(0)
    _ck(lib().tsat_autotune_bytes(s, ctypes.byref(out)), "tsat_autotune_bytes")
    return int(out.value)


def tsat_autotune(s, hp, snapshot: torch.Tensor | None = None, stream=None) -> list:
    """Tune the launch shapes on the state as it stands (left unchanged).
    ``snapshot``: device buffer of at least tsat_autotune_bytes(s) bytes; one
    is allocated for the call when omitted."""
    if snapshot is None:
        snapshot = _device_buffer(tsat_autotune_bytes(s), torch.device("cuda", torch.cuda.current_device()))
    a = (ctypes.c_int32 * 4)()
    _ck(lib().tsat_autotune(s, ctypes.byref(hp), _ptr(snapshot), snapshot.numel() * snapshot.element_size(),
                            _stream(stream), a), "tsat_autotune")
    return list(a)


def tsat_get_tuning(s) -> list:
    a = (ctypes.c_int32 * 4)()
    _ck(lib().tsat_get_tuning(s, a), "tsat_get_tuning")
    return list(a)


def tsat_set_tuning(s, tuning: Sequence[int]):
    a = (ctypes.c_int32 * 4)(*[int(x) for x in tuning])
    _ck(lib().tsat_set_tuning(s, a), "tsat_set_tuning")


def tsat_launches_per_step(s) -> int:
    return int(lib().tsat_launches_per_step(s))


def tsat_mpnn_param_count() -> int:
    return int(lib().tsat_mpnn_param_count())


def tsat_mpnn_workspace_bytes(h) -> int:
    out = ctypes.c_size_t(0)
    _ck(lib().tsat_mpnn_workspace_bytes(h, ctypes.byref(out)), "tsat_mpnn_workspace_bytes")
    return int(out.value)


def tsat_mpnn_init(params: torch.Tensor, seed: int, stream=None):
    _ck(lib().tsat_mpnn_init(_ptr(params), int(seed), _stream(stream)), "tsat_mpnn_init")


def tsat_mpnn_forward(h, params: torch.Tensor, ws: torch.Tensor, logits: torch.Tensor, stream=None):
    _ck(lib().tsat_mpnn_forward(h, _ptr(params), _ptr(ws), ws.numel() * ws.element_size(), _ptr(logits),
                                _stream(stream)), "tsat_mpnn_forward")


def tsat_mpnn_loss_grad(h, params, ws, targets, logits, loss, grad, stream=None):
    _ck(lib().tsat_mpnn_loss_grad(h, _ptr(params), _ptr(ws), ws.numel() * ws.element_size(), _ptr(targets),
                                  _ptr(logits), _ptr(loss), _ptr(grad), _stream(stream)), "tsat_mpnn_loss_grad")


def tsat_mpnn_adam(params, grad, m, v, step: int, lr: float, stream=None):
    _ck(lib().tsat_mpnn_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), int(step), float(lr), _stream(stream)),
        "tsat_mpnn_adam")


def tsat_mpnn_status(h, ws: torch.Tensor, stream=None):
    """Raise if a tensor-core layer of the last proposer call on `ws` gave up
    waiting for its MMAs (TSAT_ETIMEOUT); synchronises the stream."""
    _ck(lib().tsat_mpnn_status(h, _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)), "tsat_mpnn_status")


# ---------------------------------------------------------------- lifetime holders
def _device_buffer(nbytes: int, device) -> torch.Tensor:
    # 256-byte aligned by the caching allocator; int64 elements
    return torch.empty((nbytes + 7) // 8, dtype=torch.int64, device=device)


class Problem:
    """A loaded batch of CNFs: the library handle plus its workspace tensor."""

    def __init__(self, instances, device="cuda", stream=None, locality: bool = False):
        """locality: store each instance's clauses ordered by their smallest
        variable (TSAT_LOAD_CLAUSE_LOCALITY; for the relaxed layer)."""
        self.instances = [(int(n), np.asarray(p), np.asarray(l)) for (n, p, l) in instances]
        self.ws = _device_buffer(tsat_problem_bytes(self.instances), device)
        self.h = tsat_load_batch(self.instances, self.ws, stream, LOAD_CLAUSE_LOCALITY if locality else 0)
        self.info = tsat_problem_info(self.h)
        self.var_offsets = np.concatenate([[0], np.cumsum([n for (n, _, _) in self.instances])]).astype(np.int64)

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.tsat_problem_free(self.h)
            self.h = None


class State:
    """N assignment samples per instance over a Problem: handle + state tensor."""

    def __init__(self, prob: Problem, n_samples: int, layer: int = LAYER_STE, dtype: int = DTYPE_F32):
        self.prob = prob
        self.N = int(n_samples)
        self.layer = layer
        nbytes = tsat_state_bytes(prob.h, n_samples, layer, dtype)
        self.buf = _device_buffer(nbytes, prob.ws.device)
        self.h = tsat_state_create(prob.h, self.buf, n_samples, layer, dtype)

    def view(self, name: str, dtype=torch.float32) -> torch.Tensor:
        """Tensor view of one state array (z, m, v, nu, bits)."""
        V, N = self.prob.info["n_vars"], self.N
        ptrs = tsat_state_views(self.h)
        base = self.buf.data_ptr()
        off = ptrs[name] - base
        shape = {"z": (V, N), "m": (V, N), "v": (V, N), "nu": (V,), "bits": (V, N // 32)}[name]
        dt = torch.int32 if name == "bits" else dtype
        n = int(np.prod(shape))
        flat = self.buf.view(torch.uint8)[off: off + n * 4].view(dt)
        return flat.view(*shape)

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.tsat_state_free(self.h)
            self.h = None
