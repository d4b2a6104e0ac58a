"""ctypes binding of libgcp_gb300.so (include/gcp.h), same names as the C ABI.

Argument marshalling only: every step of the sampled-gradient path runs in the
library's CUDA kernels.  torch tensors supply device memory and streams.
Importing this module loads the library and raises ImportError when it has
not been built (``python -m paper_1906_01687_gb300.build``); there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgcp_gb300.so")
if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1906_01687_gb300.build` "
                      "(the CUDA library is the only implementation; there is no fallback)")
_lib = ctypes.CDLL(LIB_PATH)

MAX_MODES = 8
STREAM_EST = 0xFFFFFFFFFFFFFFFF

# enums (include/gcp.h)
OK, ERR_INVALID_ARG, ERR_CUDA, ERR_NO_MEMORY, ERR_SAMPLE_SHORTFALL, ERR_TIMEOUT, ERR_NONFINITE, ERR_UNSUPPORTED = range(8)
LOSS_GAUSSIAN, LOSS_BERNOULLI_LOGIT, LOSS_POISSON_LOG = 0, 1, 2
LOSS_BERNOULLI_ODDS, LOSS_POISSON_IDENTITY, LOSS_GAMMA, LOSS_BETA_HALF = 3, 4, 5, 6
SAMPLER_UNIFORM, SAMPLER_STRATIFIED, SAMPLER_SEMI_STRATIFIED, SAMPLER_OBSERVED = 0, 1, 2, 3
CLS_UNIFORM, CLS_STRAT_NZ, CLS_STRAT_ZERO, CLS_SEMI_NZ, CLS_SEMI_ZERO = range(5)
LOSSES = {"gaussian": LOSS_GAUSSIAN, "bernoulli_logit": LOSS_BERNOULLI_LOGIT, "poisson_log": LOSS_POISSON_LOG,
          "bernoulli_odds": LOSS_BERNOULLI_ODDS, "poisson_identity": LOSS_POISSON_IDENTITY, "gamma": LOSS_GAMMA,
          "beta_half": LOSS_BETA_HALF}
SAMPLERS = {"uniform": SAMPLER_UNIFORM, "stratified": SAMPLER_STRATIFIED, "semi_stratified": SAMPLER_SEMI_STRATIFIED,
            "observed": SAMPLER_OBSERVED}

_vp = ctypes.c_void_p
_P8 = _vp * MAX_MODES


class gcp_tensor(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("sparse", ctypes.c_int32), ("dims", ctypes.c_int64 * MAX_MODES),
                ("nnz", ctypes.c_int64), ("vals", _vp), ("idx", _P8), ("weights", _vp)]


class gcp_factors(ctypes.Structure):
    _fields_ = [("rank", ctypes.c_int32), ("ld", ctypes.c_int32), ("bf16", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("A", _P8), ("A_bf16", _P8)]


class gcp_sampling(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32), ("p", ctypes.c_int64),
                ("q", ctypes.c_int64), ("seed", ctypes.c_uint64), ("problem", ctypes.c_uint64),
                ("stream", ctypes.c_uint64), ("oversample", ctypes.c_double)]


class gcp_samples(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("idx", _P8), ("x", _vp), ("w", _vp), ("cls", _vp)]


class gcp_adam_params(ctypes.Structure):
    _fields_ = [("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("lower", ctypes.c_float), ("eps_inside_sqrt", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class gcp_epoch_params(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_int64), ("nu", ctypes.c_float), ("kappa", ctypes.c_int32)]


class gcp_tuning(ctypes.Structure):
    _fields_ = [("lanes", ctypes.c_int32), ("chunks", ctypes.c_int32), ("block", ctypes.c_int32),
                ("grid_blocks", ctypes.c_int32), ("smem_bytes", ctypes.c_int32), ("smem_min_hits", ctypes.c_int32),
                ("max_replicas", ctypes.c_int32), ("replica_target", ctypes.c_int32),
                ("group_draws", ctypes.c_int32), ("prefetch", ctypes.c_int32), ("early_draws", ctypes.c_int32),
                ("zero_pass", ctypes.c_int32), ("warp_combine", ctypes.c_int32),
                ("tail_work", ctypes.c_int32)]


class gcp_launch_info(ctypes.Structure):
    _fields_ = [("lanes", ctypes.c_int32), ("chunks", ctypes.c_int32), ("block", ctypes.c_int32),
                ("grid_blocks", ctypes.c_int32), ("smem_bytes", ctypes.c_int32), ("smem_mode_mask", ctypes.c_uint32),
                ("replicas", ctypes.c_int32 * MAX_MODES), ("group_draws", ctypes.c_int32),
                ("prefetch", ctypes.c_int32), ("early_draws", ctypes.c_int32), ("zero_tiles", ctypes.c_int32),
                ("combine_mode_mask", ctypes.c_uint32), ("adam_tail_blocks", ctypes.c_int32)]


class gcp_batch_problem(ctypes.Structure):
    _fields_ = [("X", gcp_tensor), ("F", gcp_factors), ("loss", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("S", gcp_sampling), ("est", gcp_samples), ("G", _P8), ("B", _P8), ("C", _P8), ("SA", _P8),
                ("SB", _P8), ("SC", _P8), ("adam", gcp_adam_params), ("epoch", gcp_epoch_params),
                ("state", _vp)]


_i32, _i64 = ctypes.c_int32, ctypes.c_int64
_P = ctypes.POINTER
_SIGS = {
    "gcp_version": ([], ctypes.c_char_p),
    "gcp_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "gcp_last_cuda_error": ([], ctypes.c_int32),
    "gcp_last_cuda_error_name": ([], ctypes.c_char_p),
    "gcp_sample_count": ([_P(gcp_sampling)], _i64),
    "gcp_create": ([_P(_vp), _P(gcp_tensor), _vp], ctypes.c_int),
    "gcp_destroy": ([_vp], ctypes.c_int),
    "gcp_get_device_status": ([_vp, _P(_i32)], ctypes.c_int),
    "gcp_set_tuning": ([_vp, _P(gcp_tuning)], ctypes.c_int),
    "gcp_get_launch": ([_vp, _P(gcp_factors), _i64, _P(gcp_launch_info)], ctypes.c_int),
    "gcp_profile": ([_vp, _i32, _i32], ctypes.c_int),
    "gcp_profile_read": ([_vp, _i32, _P(ctypes.c_double), _P(_i64)], ctypes.c_int),
    "gcp_sample": ([_vp, _P(gcp_sampling), _P(gcp_samples), _vp], ctypes.c_int),
    "gcp_reserve": ([_vp, _P(gcp_sampling), _vp], ctypes.c_int),
    "gcp_grad": ([_vp, _P(gcp_factors), ctypes.c_int, _P(gcp_sampling), _P(gcp_samples), _vp, _P8, _vp], ctypes.c_int),
    "gcp_grad_range": ([_vp, _P(gcp_factors), ctypes.c_int, _P(gcp_sampling), _i64, _i64, _vp, _P8, _vp],
                       ctypes.c_int),
    "gcp_refresh": ([_vp, _vp], ctypes.c_int),
    "gcp_full_grad": ([_vp, _P(gcp_factors), ctypes.c_int, _P8, _vp], ctypes.c_int),
    "gcp_full_loss": ([_vp, _P(gcp_factors), ctypes.c_int, _vp, _vp], ctypes.c_int),
    "gcp_loss_est": ([_vp, _P(gcp_factors), ctypes.c_int, _P(gcp_samples), _vp, _vp], ctypes.c_int),
    "gcp_loss_est_noalloc": ([_i32, _P(gcp_factors), ctypes.c_int, _P(gcp_samples), _vp, _vp], ctypes.c_int),
    "gcp_state_init": ([_vp, ctypes.c_float, _vp], ctypes.c_int),
    "gcp_adam_step": ([_P(gcp_factors), _i32, _P(_i64), _P8, _P8, _P8, _P(gcp_adam_params), _vp, _vp], ctypes.c_int),
    "gcp_iteration": ([_vp, _P(gcp_factors), ctypes.c_int, _P(gcp_sampling), _vp, _P8, _P8, _P8,
                       _P(gcp_adam_params), _vp, _vp], ctypes.c_int),
    "gcp_epoch_begin": ([_P(gcp_factors), _i32, _P(_i64), _P8, _P8, _P8, _P8, _P8, _vp, _vp], ctypes.c_int),
    "gcp_epoch_end": ([_P(gcp_factors), _i32, _P(_i64), _P8, _P8, _P8, _P8, _P8, _P(gcp_epoch_params), _vp, _vp],
                      ctypes.c_int),
    "gcp_batch_create": ([_P(_vp), _P(gcp_batch_problem), _i32, _vp], ctypes.c_int),
    "gcp_batch_destroy": ([_vp], ctypes.c_int),
    "gcp_batch_set_tuning": ([_vp, _i32, _i32], ctypes.c_int),
    "gcp_batch_set_shape": ([_vp, _i32, _i32, _i32, _vp], ctypes.c_int),
    "gcp_batch_get_shape": ([_vp, _i32, _P(_i32), _P(_i32), _P(_i32)], ctypes.c_int),
    "gcp_batch_grad": ([_vp, _vp], ctypes.c_int),
    "gcp_batch_adam_step": ([_vp, _vp], ctypes.c_int),
    "gcp_batch_iteration": ([_vp, _vp], ctypes.c_int),
    "gcp_batch_iteration_fused": ([_vp, _vp], ctypes.c_int),
    "gcp_batch_loss_est": ([_vp, _vp], ctypes.c_int),
    "gcp_batch_epoch_begin": ([_vp, _vp], ctypes.c_int),
    "gcp_batch_epoch_end": ([_vp, _vp], ctypes.c_int),
    "gcp_factors_to_bf16": ([_P(gcp_factors), _i32, _P(_i64), _vp], ctypes.c_int),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res

EXPORTED = tuple(_SIGS)


class GcpError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = f"{where}: {_lib.gcp_status_string(status).decode()} (status {status})"
        if status in (ERR_CUDA, ERR_NO_MEMORY):
            msg += f" [{_lib.gcp_last_cuda_error_name().decode()}]"
        super().__init__(msg)
        self.status = status


def _check(status: int, where: str):
    if status != OK:
        raise GcpError(status, where)


def version() -> str:
    return _lib.gcp_version().decode()


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _p8(tensors: Sequence[Optional[torch.Tensor]]):
    arr = _P8()
    for k, t in enumerate(tensors):
        arr[k] = None if t is None else t.data_ptr()
    return arr


def _dims(dims) -> ctypes.Array:
    arr = (_i64 * MAX_MODES)()
    for k, n in enumerate(dims):
        arr[k] = int(n)
    return arr


# ---------------------------------------------------------------------------
# data holders (device memory owned by torch)
# ---------------------------------------------------------------------------

def padded_ld(rank: int) -> int:
    """Row stride: rank rounded up to a multiple of 4 (16-byte FP32 rows)."""
    return (rank + 3) // 4 * 4


@dataclass
class DataTensor:
    """The data tensor X on the device: dense FP32 row-major ``vals`` or COO
    int32 ``idx`` (one array per mode) with FP32 ``vals`` (None = all ones)."""
    dims: tuple
    vals: Optional[torch.Tensor] = None
    idx: Optional[List[torch.Tensor]] = None
    weights: Optional[torch.Tensor] = None  # dense entry weights (Eq. (4.5)), None = all ones

    @property
    def sparse(self) -> bool:
        return self.idx is not None

    @property
    def nnz(self) -> int:
        return int(self.idx[0].numel()) if self.sparse else 0

    def _c(self) -> gcp_tensor:
        t = gcp_tensor()
        t.d = len(self.dims)
        t.sparse = int(self.sparse)
        t.dims = _dims(self.dims)
        t.nnz = self.nnz
        t.vals = None if self.vals is None else self.vals.data_ptr()
        if self.sparse:
            t.idx = _p8(self.idx)
        t.weights = None if self.weights is None else self.weights.data_ptr()
        return t

    @staticmethod
    def dense(X, device="cuda", weights=None) -> "DataTensor":
        x = torch.as_tensor(X).to(device=device, dtype=torch.float32).contiguous()
        w = None if weights is None else torch.as_tensor(weights).to(device=device, dtype=torch.float32).contiguous()
        return DataTensor(tuple(x.shape), vals=x.reshape(-1), weights=None if w is None else w.reshape(-1))

    @staticmethod
    def coo(dims, idx, vals=None, device="cuda") -> "DataTensor":
        ii = [torch.as_tensor(i).to(device=device, dtype=torch.int32).contiguous() for i in idx]
        vv = None if vals is None else torch.as_tensor(vals).to(device=device, dtype=torch.float32).contiguous()
        return DataTensor(tuple(int(n) for n in dims), vals=vv, idx=ii)


class Factors:
    """Factor matrices A_k as n_k x ld FP32 device tensors (columns rank..ld-1
    zero), with optional BF16 copies that the kernels gather from."""

    def __init__(self, mats: Sequence, rank: Optional[int] = None, bf16: bool = False, device="cuda"):
        mats = [torch.as_tensor(a) for a in mats]
        self.rank = int(rank if rank is not None else mats[0].shape[1])
        self.ld = padded_ld(self.rank)
        self.dims = tuple(int(a.shape[0]) for a in mats)
        self.A = []
        for a in mats:
            buf = torch.zeros((a.shape[0], self.ld), dtype=torch.float32, device=device)
            buf[:, : self.rank] = a[:, : self.rank].to(device=device, dtype=torch.float32)
            self.A.append(buf)
        self.bf16 = bool(bf16)
        self.A_bf16 = [torch.zeros((n, self.ld), dtype=torch.bfloat16, device=device) for n in self.dims] if bf16 else None
        if bf16:
            gcp_factors_to_bf16(self)

    def _c(self, gather_bf16: Optional[bool] = None) -> gcp_factors:
        f = gcp_factors()
        f.rank = self.rank
        f.ld = self.ld
        f.bf16 = int(self.bf16 if gather_bf16 is None else gather_bf16)
        f.A = _p8(self.A)
        if self.A_bf16 is not None:
            f.A_bf16 = _p8(self.A_bf16)
        return f

    def like(self) -> List[torch.Tensor]:
        """Zeroed FP32 buffers with the factors' layout (G, B, C, snapshots)."""
        return [torch.zeros_like(a) for a in self.A]

    def numpy(self):
        return [a[:, : self.rank].double().cpu().numpy() for a in self.A]


@dataclass
class SampleList:
    """Materialised drawn entries on the device (struct of arrays)."""
    idx: List[torch.Tensor]
    x: torch.Tensor
    w: torch.Tensor
    cls: torch.Tensor

    @property
    def n(self) -> int:
        return int(self.x.numel())

    @staticmethod
    def empty(d: int, n: int, device="cuda") -> "SampleList":
        return SampleList([torch.zeros(n, dtype=torch.int32, device=device) for _ in range(d)],
                          torch.zeros(n, dtype=torch.float32, device=device),
                          torch.zeros(n, dtype=torch.float32, device=device),
                          torch.zeros(n, dtype=torch.int8, device=device))

    def _c(self) -> gcp_samples:
        s = gcp_samples()
        s.n = self.n
        s.idx = _p8(self.idx)
        s.x = self.x.data_ptr()
        s.w = self.w.data_ptr()
        s.cls = self.cls.data_ptr()
        return s


@dataclass
class Sampling:
    """A sampling spec (Sections 4.1-4.3): uniform draws q; (semi-)stratified p + q."""
    kind: int
    p: int
    q: int
    seed: int
    stream: int = 0
    problem: int = 0
    oversample: float = 1.1

    def _c(self) -> gcp_sampling:
        s = gcp_sampling()
        s.kind = int(self.kind)
        s.p = int(self.p)
        s.q = int(self.q)
        s.seed = int(self.seed) & 0xFFFFFFFFFFFFFFFF
        s.problem = int(self.problem) & 0xFFFFFFFFFFFFFFFF
        s.stream = int(self.stream) & 0xFFFFFFFFFFFFFFFF
        s.oversample = float(self.oversample)
        return s

    def count(self) -> int:
        return int(_lib.gcp_sample_count(ctypes.byref(self._c())))


# ---------------------------------------------------------------------------
# entry points
# ---------------------------------------------------------------------------

class Handle:
    """gcp_create / gcp_destroy around a prepared data tensor."""

    def __init__(self, X: DataTensor, stream=None):
        self.X = X  # keeps X's device arrays alive
        self.d = len(X.dims)
        self.dims = tuple(X.dims)
        self._h = ctypes.c_void_p()
        _check(_lib.gcp_create(ctypes.byref(self._h), ctypes.byref(X._c()), _stream(stream)), "gcp_create")

    def close(self):
        if self._h:
            _lib.gcp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def ptr(self):
        return self._h


def gcp_get_device_status(h: Handle) -> int:
    v = ctypes.c_int32(0)
    _check(_lib.gcp_get_device_status(h.ptr, ctypes.byref(v)), "gcp_get_device_status")
    return int(v.value)


TUNING_FIELDS = ("lanes", "chunks", "block", "grid_blocks", "smem_bytes", "smem_min_hits", "max_replicas",
                 "replica_target", "group_draws", "prefetch", "early_draws", "zero_pass", "warp_combine",
                 "tail_work")
TUNING_DEFAULT = dict(lanes=0, chunks=0, block=0, grid_blocks=0, smem_bytes=-1, smem_min_hits=-1,
                      max_replicas=-1, replica_target=0, group_draws=0, prefetch=0, early_draws=0, zero_pass=0,
                      warp_combine=0, tail_work=0)


def gcp_set_tuning(h: Handle, reset: bool = False, **kw):
    """Sets the handle's launch shape (fields of gcp_tuning; missing = automatic)."""
    if reset:
        _check(_lib.gcp_set_tuning(h.ptr, None), "gcp_set_tuning")
        return
    vals = dict(TUNING_DEFAULT)
    for k, v in kw.items():
        if k not in vals:
            raise TypeError(f"unknown tuning field {k}")
        vals[k] = int(v)
    t = gcp_tuning(*[vals[f] for f in TUNING_FIELDS])
    _check(_lib.gcp_set_tuning(h.ptr, ctypes.byref(t)), "gcp_set_tuning")


def gcp_get_launch(h: Handle, F: Factors, n_draws: int) -> dict:
    t = gcp_launch_info()
    _check(_lib.gcp_get_launch(h.ptr, ctypes.byref(F._c()), int(n_draws), ctypes.byref(t)), "gcp_get_launch")
    return dict(lanes=t.lanes, chunks=t.chunks, block=t.block, grid_blocks=t.grid_blocks,
                smem_bytes=t.smem_bytes, smem_mode_mask=t.smem_mode_mask, replicas=list(t.replicas)[: h.d],
                group_draws=t.group_draws, prefetch=t.prefetch, early_draws=t.early_draws, zero_tiles=t.zero_tiles,
                combine_mode_mask=t.combine_mode_mask, adam_tail_blocks=t.adam_tail_blocks)


def gcp_profile(h: Handle, enable: bool, capacity: int = 1024):
    """Records CUDA events around each following fused-gradient kernel launch."""
    _check(_lib.gcp_profile(h.ptr, int(bool(enable)), int(capacity)), "gcp_profile")


def gcp_profile_read(h: Handle, which: int = 0):
    """(total device milliseconds, launches) of the recorded gradient kernels
    (which = 0) or of gcp_iteration's Adam kernels (which = 1)."""
    ms, n = ctypes.c_double(0.0), ctypes.c_int64(0)
    _check(_lib.gcp_profile_read(h.ptr, int(which), ctypes.byref(ms), ctypes.byref(n)), "gcp_profile_read")
    return ms.value, n.value


def gcp_sample(h: Handle, S: Sampling, out: Optional[SampleList] = None, stream=None) -> SampleList:
    if out is None:
        out = SampleList.empty(h.d, S.count(), device=h.X.vals.device if h.X.vals is not None else h.X.idx[0].device)
    _check(_lib.gcp_sample(h.ptr, ctypes.byref(S._c()), ctypes.byref(out._c()), _stream(stream)), "gcp_sample")
    return out


def gcp_reserve(h: Handle, S: Sampling, stream=None):
    """Makes every lazy library allocation for spec S now (call before graph capture)."""
    _check(_lib.gcp_reserve(h.ptr, ctypes.byref(S._c()), _stream(stream)), "gcp_reserve")


def gcp_grad(h: Handle, F: Factors, loss: int, G: Sequence[torch.Tensor], S: Optional[Sampling] = None,
             samples: Optional[SampleList] = None, stream_dev: Optional[torch.Tensor] = None, stream=None,
             gather_bf16: Optional[bool] = None):
    """Accumulates the sampled gradient into G (n_k x ld FP32 device tensors)."""
    sp = ctypes.byref(S._c()) if S is not None else None
    lp = ctypes.byref(samples._c()) if samples is not None else None
    _check(_lib.gcp_grad(h.ptr, ctypes.byref(F._c(gather_bf16)), int(loss), sp, lp, _ptr(stream_dev), _p8(G),
                         _stream(stream)), "gcp_grad")


def gcp_grad_range(h: Handle, F: Factors, loss: int, G: Sequence[torch.Tensor], S: Sampling, first: int,
                   count: int, stream_dev: Optional[torch.Tensor] = None, stream=None,
                   gather_bf16: Optional[bool] = None):
    """Accumulates into G the sampled gradient of the draws [first, first + count) of spec S."""
    _check(_lib.gcp_grad_range(h.ptr, ctypes.byref(F._c(gather_bf16)), int(loss), ctypes.byref(S._c()), int(first),
                               int(count), _ptr(stream_dev), _p8(G), _stream(stream)), "gcp_grad_range")


def gcp_refresh(h: Handle, stream=None):
    """Takes up new contents of the handle's tensor arrays (rewritten in place by the caller)."""
    _check(_lib.gcp_refresh(h.ptr, _stream(stream)), "gcp_refresh")


def gcp_full_grad(h: Handle, F: Factors, loss: int, G, stream=None):
    """Full gradient G_k = Y_(k) Z_k of a dense tensor over every index (accumulates into G)."""
    _check(_lib.gcp_full_grad(h.ptr, ctypes.byref(F._c()), int(loss), _p8(G), _stream(stream)), "gcp_full_grad")


def gcp_full_loss(h: Handle, F: Factors, loss: int, out: torch.Tensor, stream=None):
    """Exact objective F(X, M) of a dense tensor into out (device float64)."""
    assert out.dtype == torch.float64 and out.is_cuda
    _check(_lib.gcp_full_loss(h.ptr, ctypes.byref(F._c()), int(loss), _ptr(out), _stream(stream)), "gcp_full_loss")


def gcp_loss_est(h: Handle, F: Factors, loss: int, samples: SampleList, out: torch.Tensor, stream=None,
                 gather_bf16: Optional[bool] = None):
    """Writes F-hat (FP64) for the fixed list into out (a device float64 tensor, first element)."""
    assert out.dtype == torch.float64 and out.is_cuda
    _check(_lib.gcp_loss_est(h.ptr, ctypes.byref(F._c(gather_bf16)), int(loss), ctypes.byref(samples._c()),
                             _ptr(out), _stream(stream)), "gcp_loss_est")


def gcp_loss_est_noalloc(d: int, F: Factors, loss: int, samples: SampleList, out: torch.Tensor, stream=None,
                         gather_bf16: Optional[bool] = None):
    """gcp_loss_est without a handle and without any allocation by the library
    (scratch in a static device array; overlapping calls race)."""
    assert out.dtype == torch.float64 and out.is_cuda
    _check(_lib.gcp_loss_est_noalloc(int(d), ctypes.byref(F._c(gather_bf16)), int(loss), ctypes.byref(samples._c()),
                                     _ptr(out), _stream(stream)), "gcp_loss_est_noalloc")


STATE_FIELDS = ("F", "F_old", "t", "iter", "alpha", "bad", "done", "status")


def new_state(device="cuda") -> torch.Tensor:
    """A 64-byte device buffer for gcp_adam_state."""
    return torch.zeros(8, dtype=torch.float64, device=device)


def read_state(state: torch.Tensor) -> dict:
    raw = state.cpu().numpy().tobytes()
    import struct
    F, F_old, t, it, alpha, bad, done, status = struct.unpack_from("<ddqqfiii", raw)
    return dict(F=F, F_old=F_old, t=t, iter=it, alpha=alpha, bad=bad, done=done, status=status)


def gcp_state_init(state: torch.Tensor, alpha: float, stream=None):
    _check(_lib.gcp_state_init(_ptr(state), ctypes.c_float(alpha), _stream(stream)), "gcp_state_init")


def _adam_params(beta1, beta2, eps, lower, eps_inside_sqrt):
    return gcp_adam_params(beta1, beta2, eps, lower, int(bool(eps_inside_sqrt)), 0)


def gcp_adam_step(F: Factors, G, B, C, state: torch.Tensor, beta1=0.9, beta2=0.999, eps=1e-8,
                  lower=-math.inf, eps_inside_sqrt=True, stream=None):
    d = len(F.dims)
    dims = (_i64 * d)(*F.dims)
    prm = _adam_params(beta1, beta2, eps, lower, eps_inside_sqrt)
    _check(_lib.gcp_adam_step(ctypes.byref(F._c()), d, dims, _p8(G), _p8(B), _p8(C), ctypes.byref(prm),
                              _ptr(state), _stream(stream)), "gcp_adam_step")


def gcp_iteration(h: Handle, F: Factors, loss: int, S: Sampling, G, B, C, state: torch.Tensor,
                  stream_dev: Optional[torch.Tensor] = None, beta1=0.9, beta2=0.999, eps=1e-8, lower=-math.inf,
                  eps_inside_sqrt=True, stream=None):
    """One fused GCP-Adam iteration: sampled gradient + Adam step (G zero on entry and exit)."""
    prm = _adam_params(beta1, beta2, eps, lower, eps_inside_sqrt)
    _check(_lib.gcp_iteration(h.ptr, ctypes.byref(F._c()), int(loss), ctypes.byref(S._c()), _ptr(stream_dev),
                              _p8(G), _p8(B), _p8(C), ctypes.byref(prm), _ptr(state), _stream(stream)),
           "gcp_iteration")


def gcp_epoch_begin(F: Factors, B, C, SA, SB, SC, state: torch.Tensor, stream=None):
    d = len(F.dims)
    dims = (_i64 * d)(*F.dims)
    _check(_lib.gcp_epoch_begin(ctypes.byref(F._c()), d, dims, _p8(B), _p8(C), _p8(SA), _p8(SB), _p8(SC),
                                _ptr(state), _stream(stream)), "gcp_epoch_begin")


def gcp_epoch_end(F: Factors, B, C, SA, SB, SC, state: torch.Tensor, tau: int, nu: float = 0.1, kappa: int = 1,
                  stream=None):
    d = len(F.dims)
    dims = (_i64 * d)(*F.dims)
    ep = gcp_epoch_params(int(tau), float(nu), int(kappa))
    _check(_lib.gcp_epoch_end(ctypes.byref(F._c()), d, dims, _p8(B), _p8(C), _p8(SA), _p8(SB), _p8(SC),
                              ctypes.byref(ep), _ptr(state), _stream(stream)), "gcp_epoch_end")


def gcp_factors_to_bf16(F: Factors, stream=None):
    d = len(F.dims)
    dims = (_i64 * d)(*F.dims)
    _check(_lib.gcp_factors_to_bf16(ctypes.byref(F._c()), d, dims, _stream(stream)), "gcp_factors_to_bf16")


# ---------------------------------------------------------------------------
# batched form
# ---------------------------------------------------------------------------

class Batch:
    """gcp_batch_create / gcp_batch_destroy over a list of problem dicts with
    keys X (DataTensor, dense), F (Factors), loss, S (uniform Sampling), est
    (SampleList), G, B, C, SA, SB, SC (buffer lists), state, and optional
    adam (dict of beta1, beta2, eps, lower, eps_inside_sqrt) and epoch (dict
    of tau, nu, kappa)."""

    def __init__(self, problems, stream=None):
        self.problems = problems  # keeps every device buffer alive
        arr = (gcp_batch_problem * len(problems))()
        for i, p in enumerate(problems):
            c = arr[i]
            c.X = p["X"]._c()
            c.F = p["F"]._c()
            c.loss = int(p["loss"])
            c.S = p["S"]._c()
            c.est = p["est"]._c()
            for name in ("G", "B", "C", "SA", "SB", "SC"):
                setattr(c, name, _p8(p[name]))
            ad = dict(beta1=0.9, beta2=0.999, eps=1e-8, lower=-math.inf, eps_inside_sqrt=True)
            ad.update(p.get("adam", {}))
            c.adam = _adam_params(**ad)
            ep = dict(tau=1000, nu=0.1, kappa=1)
            ep.update(p.get("epoch", {}))
            c.epoch = gcp_epoch_params(int(ep["tau"]), float(ep["nu"]), int(ep["kappa"]))
            c.state = p["state"].data_ptr()
        self._b = ctypes.c_void_p()
        _check(_lib.gcp_batch_create(ctypes.byref(self._b), arr, len(problems), _stream(stream)), "gcp_batch_create")

    def close(self):
        if self._b:
            _lib.gcp_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tuning(self, block=0, grid_blocks=0):
        _check(_lib.gcp_batch_set_tuning(self._b, int(block), int(grid_blocks)), "gcp_batch_set_tuning")

    def set_shape(self, chunks_per_lane=0, replica_target=0, max_replicas=0, stream=None):
        """Rows per warp (chunks per lane) and replica slabs of every problem (before graph capture)."""
        _check(_lib.gcp_batch_set_shape(self._b, int(chunks_per_lane), int(replica_target), int(max_replicas),
                                        _stream(stream)), "gcp_batch_set_shape")

    def get_shape(self, problem):
        """(lanes per draw, chunks per lane, replica slabs per mode) of one problem."""
        L, NC = ctypes.c_int32(0), ctypes.c_int32(0)
        reps = (ctypes.c_int32 * 4)()
        _check(_lib.gcp_batch_get_shape(self._b, int(problem), ctypes.byref(L), ctypes.byref(NC), reps),
               "gcp_batch_get_shape")
        return dict(lanes=L.value, chunks=NC.value, replicas=[r for r in reps if r > 0])

    def _call(self, name, stream):
        _check(getattr(_lib, name)(self._b, _stream(stream)), name)

    def grad(self, stream=None):
        self._call("gcp_batch_grad", stream)

    def adam_step(self, stream=None):
        self._call("gcp_batch_adam_step", stream)

    def iteration(self, stream=None):
        self._call("gcp_batch_iteration", stream)

    def iteration_fused(self, stream=None):
        """One iteration of every problem in one persistent launch."""
        self._call("gcp_batch_iteration_fused", stream)

    def loss_est(self, stream=None):
        self._call("gcp_batch_loss_est", stream)

    def epoch_begin(self, stream=None):
        self._call("gcp_batch_epoch_begin", stream)

    def epoch_end(self, stream=None):
        self._call("gcp_batch_epoch_end", stream)
