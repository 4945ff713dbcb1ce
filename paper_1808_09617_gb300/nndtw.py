"""Thin Python binding of libnndtw.so (see include/nndtw.h for the contract).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Tensors are PyTorch CUDA tensors (device memory and streams come
from PyTorch); the binding checks dtype, device and contiguity, passes raw
pointers and sizes, and turns status codes into ``NnDtwError``.  There is no
CPU fallback: if the library is missing or cannot be loaded, every call
raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libnndtw.so")

NNDTW_MAX_L = 8192
OK, EINVAL, ECUDA, ENOSPACE, EUNSUPPORTED, ENONFINITE = 0, 1, 2, 3, 4, 5
LB_KEOGH = 1 << 0
LB_SAFE = 1 << 1
LB_NEW = 1 << 18
EXACT_DIST = 1 << 2
NO_PRUNE = 1 << 3
NO_ABANDON = 1 << 4
CHECK_FINITE = 1 << 5
TIME_STAGES = 1 << 6
NO_REVERSE = 1 << 7
REVERSE = 1 << 14
LEAVE_ONE_OUT = 1 << 15
IMPROVED = 1 << 16
KEOGH_BOUND = 1 << 17


# Tuning values for full windows: the row layout with 32 lanes per pair (one
# pair per warp), 16 lanes (L <= 1024) or 8 lanes (L <= 512).
ROWS_GROUP = 64
ROWS16_GROUP = 65
ROWS8_GROUP = 66
DTW_GROUP_MASK = 7 << 8
DTW_ROWS = 7 << 8
DTW_ROWS_LANES16 = 1 << 12
DTW_ROWS_LANES8 = 2 << 12


def LB_TILE(k: int) -> int:
    """Flag selecting the bound pass's tile shape: 1 = 32 x 32, 2 = 64 x 64,
    3 = 128 x 64 (queries x training series per CTA); 0 = the library's
    choice.  A tuning choice: results never change."""
    if k not in (0, 1, 2, 3):
        raise ValueError("LB tile shape must be 0..3")
    return k << 19


LB_TILE_MASK = 3 << 19


def DTW_GROUP(g: int) -> int:
    """Flag selecting G lanes per pair in the FP32 DTW kernel's diagonal layout
    (G = 1..32), or the row layout for full windows (G = ROWS_GROUP,
    ROWS16_GROUP or ROWS8_GROUP)."""
    if g == ROWS_GROUP:
        return DTW_ROWS
    if g == ROWS16_GROUP:
        return DTW_ROWS | DTW_ROWS_LANES16
    if g == ROWS8_GROUP:
        return DTW_ROWS | DTW_ROWS_LANES8
    if g < 1 or g > 32 or g & (g - 1):
        raise ValueError("G must be a power of two in 1..32")
    return (g.bit_length()) << 8
STAGES = ("envelopes", "lb", "seed", "compact", "dtw", "recheck", "final", "total")

_lib = None
_lock = threading.Lock()

_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int
_uint = ctypes.c_uint
_sz = ctypes.c_size_t


class NnDtwError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = f"{where}: status {code}"
        if _lib is not None:
            msg += f" ({_lib.nn_dtw_strerror(code).decode()})"
            if code == ECUDA:
                msg += f": {_lib.nn_dtw_last_cuda_error().decode()}"
        super().__init__(msg)


class NativeLibraryMissing(RuntimeError):
    pass


class Stats(ctypes.Structure):
    _fields_ = [("pairs", ctypes.c_int64), ("lb_pruned", ctypes.c_int64),
                ("dtw_started", ctypes.c_int64), ("dtw_abandoned", ctypes.c_int64),
                ("dtw_cells", ctypes.c_int64), ("rechecked", ctypes.c_int64),
                ("recheck_queries", ctypes.c_int64), ("seed_cells", ctypes.c_int64),
                ("lb_pruned_reverse", ctypes.c_int64), ("lb_pruned_improved", ctypes.c_int64),
                ("lb_pruned_live", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class DatasetDesc(ctypes.Structure):
    """Mirror of nndtw_dataset."""
    _fields_ = [("d_train", _vp), ("d_train_labels", _vp), ("N", ctypes.c_int64),
                ("d_test", _vp), ("Q", ctypes.c_int64), ("L", ctypes.c_int), ("W", ctypes.c_int),
                ("V", ctypes.c_int), ("d_env", _vp), ("d_nn_idx", _vp), ("d_nn_label", _vp),
                ("d_nn_dist", _vp), ("flags", ctypes.c_uint)]


class HostDatasetDesc(ctypes.Structure):
    """Mirror of nndtw_host_dataset."""
    _fields_ = [("h_train", _vp), ("h_train_labels", _vp), ("N", ctypes.c_int64),
                ("h_test", _vp), ("Q", ctypes.c_int64), ("L", ctypes.c_int), ("W", ctypes.c_int),
                ("V", ctypes.c_int), ("h_nn_idx", _vp), ("h_nn_label", _vp),
                ("h_nn_dist", _vp), ("flags", ctypes.c_uint)]


def _declare(lib):
    sig = {
        "nn_dtw_build_envelopes": [_vp, _i64, _int, _int, _vp, _vp],
        "nn_dtw_build_envelopes_f64": [_vp, _i64, _int, _int, _vp, _vp],
        "lb_enhanced": [_vp, _i64, _vp, _vp, _i64, _int, _int, _int, _uint, _vp, _vp],
        "lb_enhanced_f64": [_vp, _i64, _vp, _vp, _i64, _int, _int, _int, _uint, _vp, _vp],
        "nn_dtw_build_second_envelopes": [_vp, _i64, _int, _int, _vp, _vp],
        "nn_dtw_build_second_envelopes_f64": [_vp, _i64, _int, _int, _vp, _vp],
        "lb_enhanced_improved": [_vp, _vp, _i64, _vp, _vp, _vp, _i64, _int, _int, _int, _uint,
                                 _vp, _vp],
        "lb_enhanced_improved_f64": [_vp, _vp, _i64, _vp, _vp, _vp, _i64, _int, _int, _int,
                                     _uint, _vp, _vp],
        "dtw_windowed": [_vp, _vp, _vp, _i64, _int, _int, _vp, _vp],
        "dtw_windowed_ex": [_vp, _vp, _vp, _i64, _int, _int, _uint, _vp, _vp],
        "dtw_windowed_f64": [_vp, _vp, _vp, _i64, _int, _int, _vp, _vp],
        "nn_dtw_search": [_vp, _vp, _i64, _vp, _i64, _int, _int, _int, _vp, _uint, _vp, _vp, _vp,
                          _vp, _sz, _vp, _vp],
        "nn_dtw_search_f64": [_vp, _vp, _i64, _vp, _i64, _int, _int, _int, _vp, _uint, _vp, _vp,
                              _vp, _vp, _sz, _vp, _vp],
        "nn_dtw_search_host": [_vp, _vp, _i64, _vp, _i64, _int, _int, _int, _uint, _vp, _vp, _vp,
                               _vp, _sz, _vp, _vp],
        "nn_dtw_search_noalloc": [_vp, _vp, _i64, _vp, _i64, _int, _int, _int, _vp, _uint, _vp,
                                  _vp, _vp, _vp, _vp],
        "nn_dtw_build_envelopes_varlen": [_vp, _vp, _i64, _int, _int, _vp, _vp],
        "lb_enhanced_varlen": [_vp, _vp, _i64, _vp, _vp, _vp, _i64, _int, _int, _int, _uint, _vp,
                               _vp],
        "dtw_windowed_varlen": [_vp, _vp, _vp, _vp, _vp, _i64, _int, _int, _vp, _vp],
        "nn_dtw_search_varlen": [_vp, _vp, _vp, _i64, _vp, _vp, _i64, _int, _int, _int, _uint,
                                 _vp, _vp, _vp, _vp, _sz, _vp, _vp],
        "nn_dtw_search_varlen_host": [_vp, _vp, _vp, _i64, _vp, _vp, _i64, _int, _int, _int,
                                      _uint, _vp, _vp, _vp, _vp, _sz, _vp, _vp],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = _int
    lib.nn_dtw_workspace_size.argtypes = [_i64, _i64, _int, _int, _int, _int]
    lib.nn_dtw_workspace_size.restype = _sz
    lib.nn_dtw_host_buffer_size.argtypes = [_i64, _i64, _int, _int, _int]
    lib.nn_dtw_host_buffer_size.restype = _sz
    lib.nn_dtw_varlen_workspace_size.argtypes = [_i64, _i64, _int, _int, _int]
    lib.nn_dtw_varlen_workspace_size.restype = _sz
    lib.nn_dtw_varlen_host_buffer_size.argtypes = [_vp, _i64, _vp, _i64, _int, _int, _int]
    lib.nn_dtw_varlen_host_buffer_size.restype = _sz
    lib.nn_dtw_strerror.argtypes = [_int]
    lib.nn_dtw_strerror.restype = ctypes.c_char_p
    lib.nn_dtw_last_cuda_error.argtypes = []
    lib.nn_dtw_last_cuda_error.restype = ctypes.c_char_p
    lib.nn_dtw_last_call_stage_launches.argtypes = [ctypes.POINTER(ctypes.c_longlong)]
    lib.nn_dtw_last_call_stage_launches.restype = _int
    lib.nn_dtw_last_call_launches.argtypes = []
    lib.nn_dtw_last_call_launches.restype = ctypes.c_longlong
    lib.nn_dtw_version.argtypes = []
    lib.nn_dtw_version.restype = _int
    lib.nn_dtw_batch_workspace_size.argtypes = [ctypes.POINTER(DatasetDesc), _int]
    lib.nn_dtw_batch_workspace_size.restype = _sz
    lib.nn_dtw_search_batched.argtypes = [ctypes.POINTER(DatasetDesc), _int, _vp, _sz, _uint, _vp]
    lib.nn_dtw_search_batched.restype = _int
    lib.nn_dtw_batch_host_buffer_size.argtypes = [ctypes.POINTER(HostDatasetDesc), _int]
    lib.nn_dtw_batch_host_buffer_size.restype = _sz
    lib.nn_dtw_search_batched_host.argtypes = [ctypes.POINTER(HostDatasetDesc), _int, _vp, _sz,
                                               _uint, _vp]
    lib.nn_dtw_search_batched_host.restype = _int
    lib.nn_dtw_learn_window_workspace_size.argtypes = [_i64, _int, _vp, _int, _int]
    lib.nn_dtw_learn_window_workspace_size.restype = _sz
    lib.nn_dtw_learn_window.argtypes = [_vp, _vp, _i64, _int, _vp, _int, _int, _uint, _vp, _vp,
                                        _sz, _vp]
    lib.nn_dtw_learn_window.restype = _int
    lib.nn_dtw_stage_times.argtypes = [ctypes.POINTER(ctypes.c_float)]
    lib.nn_dtw_stage_times.restype = _int
    lib.nn_dtw_probe_sink_bytes.argtypes = []
    lib.nn_dtw_probe_sink_bytes.restype = _sz
    lib.nn_dtw_probe_cell_rate.argtypes = [_vp, _sz, _int, ctypes.POINTER(ctypes.c_double), _vp]
    lib.nn_dtw_probe_cell_rate.restype = _int
    return lib


def load(path: str | None = None):
    """Load libnndtw.so (built by ``paper_1808_09617_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise NativeLibraryMissing(
                    f"{p} not found: build it with `python -m paper_1808_09617_gb300.build` "
                    "(there is no CPU fallback)")
            _lib = _declare(ctypes.CDLL(p))
    return _lib


def _check(code: int, where: str):
    if code != OK:
        raise NnDtwError(code, where)


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return _vp(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def one_device(devices, stream_device=None):
    """The one CUDA device shared by every tensor argument of a call (and by
    its stream, when it names one).  Tensors on two devices, or a stream of
    another device, raise ValueError before anything reaches the library:
    its kernels would run on the current device with another GPU's
    pointers."""
    devs = {(d.type, d.index) for d in devices if d is not None}
    if len(devs) != 1:
        raise ValueError(f"all tensor arguments must be on one CUDA device, got {sorted(devs)}")
    typ, idx = devs.pop()
    if typ != "cuda":
        raise TypeError("tensor arguments must be CUDA tensors")
    if stream_device is not None and (stream_device.type, stream_device.index) != (typ, idx):
        raise ValueError(f"stream is on {stream_device}, tensors on cuda:{idx}")
    return idx


def _on(tensors, stream=None):
    """Context in which a library call runs: the tensors' device made current
    (the library launches on the current device), after one_device's check."""
    import torch
    sdev = getattr(stream, "device", None) if stream is not None else None
    idx = one_device([t.device for t in tensors if isinstance(t, torch.Tensor)], sdev)
    return torch.cuda.device(idx)


def _dev(t, dtype, name, ndim=None, shape=None):
    """Device pointer of a contiguous CUDA tensor of the given dtype, after
    checking its rank and (with shape; None entries match any size) its
    shape, so that no kernel reads or writes past a caller's buffer."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if ndim is not None and t.dim() != ndim:
        raise ValueError(f"{name} must have {ndim} dimensions")
    if shape is not None:
        if t.dim() != len(shape) or any(w is not None and int(g) != int(w)
                                        for g, w in zip(t.shape, shape)):
            want = tuple("*" if w is None else int(w) for w in shape)
            raise ValueError(f"{name} must have shape {want}, got {tuple(t.shape)}")
    return _vp(t.data_ptr())


def _fp(t):
    import torch
    return {torch.float32: False, torch.float64: True}[t.dtype]


# ------------------------------------------------------------------ entry points

def nn_dtw_build_envelopes(train, W: int, env=None, stream=None):
    """Envelopes (U, Lo) of every training series, Eq. 3-4: tensor [N, L, 2]."""
    import torch
    lib = load()
    f64 = _fp(train)
    N, L = train.shape
    if env is None:
        env = torch.empty((N, L, 2), dtype=train.dtype, device=train.device)
    fn = lib.nn_dtw_build_envelopes_f64 if f64 else lib.nn_dtw_build_envelopes
    with _on([train, env], stream):
        _check(fn(_dev(train, train.dtype, "train", 2), N, L, int(W),
                _dev(env, train.dtype, "env", shape=(N, L, 2)), _stream(stream)),
             "nn_dtw_build_envelopes")
    return env


def lb_enhanced(test, train, env, W: int, V: int, keogh: bool = False, safe: bool = False,
                out=None, stream=None, tile: int = 0):
    """LB_Enhanced^V (or LB_Keogh) for all pairs: tensor [Q, N] (``tile``:
    the bound pass's tile shape, see LB_TILE)."""
    import torch
    lib = load()
    f64 = _fp(test)
    Q, L = test.shape
    N = train.shape[0]
    if out is None:
        out = torch.empty((Q, N), dtype=test.dtype, device=test.device)
    flags = (LB_KEOGH if keogh else 0) | (LB_SAFE if safe else 0) | LB_TILE(tile)
    fn = lib.lb_enhanced_f64 if f64 else lib.lb_enhanced
    with _on([test, train, env, out], stream):
        _check(fn(_dev(test, test.dtype, "test", 2), Q,
                _dev(train, test.dtype, "train", shape=(N, L)),
                _dev(env, test.dtype, "env", shape=(N, L, 2)), N, L, int(W), int(V), flags,
                _dev(out, test.dtype, "out", shape=(Q, N)), _stream(stream)), "lb_enhanced")
    return out


def lb_new(test, train, W: int, safe: bool = False, out=None, stream=None):
    """LB_New (Sec. 2.2.5) for all pairs: tensor [Q, N]."""
    import torch
    lib = load()
    f64 = _fp(test)
    Q, L = test.shape
    N = train.shape[0]
    if out is None:
        out = torch.empty((Q, N), dtype=test.dtype, device=test.device)
    flags = LB_NEW | (LB_SAFE if safe else 0)
    fn = lib.lb_enhanced_f64 if f64 else lib.lb_enhanced
    with _on([test, train, out], stream):
        _check(fn(_dev(test, test.dtype, "test", 2), Q,
                  _dev(train, test.dtype, "train", shape=(N, L)), None, N, L, int(W), 1, flags,
                  _dev(out, test.dtype, "out", shape=(Q, N)), _stream(stream)), "lb_new")
    return out


def nn_dtw_build_second_envelopes(env, W: int, env2=None, stream=None):
    """Second envelopes (window max of Lo, window min of U) of every training
    series, from its envelopes [N, L, 2]: tensor [N, L, 2]."""
    import torch
    lib = load()
    f64 = _fp(env)
    N, L = env.shape[0], env.shape[1]
    if env2 is None:
        env2 = torch.empty_like(env)
    fn = lib.nn_dtw_build_second_envelopes_f64 if f64 else lib.nn_dtw_build_second_envelopes
    with _on([env, env2], stream):
        _check(fn(_dev(env, env.dtype, "env", shape=(N, L, 2)), N, L, int(W),
                _dev(env2, env.dtype, "env2", shape=(N, L, 2)), _stream(stream)),
             "nn_dtw_build_second_envelopes")
    return env2


def lb_enhanced_improved(test, test_env, train, env, env2, W: int, V: int, safe: bool = False,
                         out=None, stream=None):
    """LB_Enhanced^V with the LB_Improved bridge (Sec. 5) for all pairs:
    tensor [Q, N].  test_env: envelopes of the test set; env, env2: the
    training series' envelopes and second envelopes, all with the same W."""
    import torch
    lib = load()
    f64 = _fp(test)
    Q, L = test.shape
    N = train.shape[0]
    if out is None:
        out = torch.empty((Q, N), dtype=test.dtype, device=test.device)
    fn = lib.lb_enhanced_improved_f64 if f64 else lib.lb_enhanced_improved
    with _on([test, test_env, train, env, env2, out], stream):
        _check(fn(_dev(test, test.dtype, "test", 2),
                _dev(test_env, test.dtype, "test_env", shape=(Q, L, 2)), Q,
                _dev(train, test.dtype, "train", shape=(N, L)),
                _dev(env, test.dtype, "env", shape=(N, L, 2)),
                _dev(env2, test.dtype, "env2", shape=(N, L, 2)), N, L, int(W), int(V),
                LB_SAFE if safe else 0, _dev(out, test.dtype, "out", shape=(Q, N)),
                _stream(stream)), "lb_enhanced_improved")
    return out


def lb_improved(test, test_env, train, env, env2, W: int, safe: bool = False, out=None,
                stream=None):
    """LB_Improved (Sec. 2.2.4, Eq. 5) for all pairs: LB_Keogh plus the
    second pass over the whole series (lb_enhanced_improved with
    NNDTW_LB_KEOGH); tensor [Q, N]."""
    import torch
    lib = load()
    f64 = _fp(test)
    Q, L = test.shape
    N = train.shape[0]
    if out is None:
        out = torch.empty((Q, N), dtype=test.dtype, device=test.device)
    fn = lib.lb_enhanced_improved_f64 if f64 else lib.lb_enhanced_improved
    with _on([test, test_env, train, env, env2, out], stream):
        _check(fn(_dev(test, test.dtype, "test", 2),
                  _dev(test_env, test.dtype, "test_env", shape=(Q, L, 2)), Q,
                  _dev(train, test.dtype, "train", shape=(N, L)),
                  _dev(env, test.dtype, "env", shape=(N, L, 2)),
                  _dev(env2, test.dtype, "env2", shape=(N, L, 2)), N, L, int(W), 1,
                  LB_KEOGH | (LB_SAFE if safe else 0), _dev(out, test.dtype, "out", shape=(Q, N)),
                  _stream(stream)), "lb_improved")
    return out


def dtw_windowed(test, train, pairs, W: int, out=None, stream=None, flags: int = 0):
    """DTW_W for explicit (q, t) pairs (int32 tensor [P, 2]): tensor [P]."""
    import torch
    lib = load()
    f64 = _fp(test)
    L = test.shape[1]
    P = pairs.shape[0]
    if out is None:
        out = torch.empty((P,), dtype=test.dtype, device=test.device)
    args = (_dev(test, test.dtype, "test", 2), _dev(train, test.dtype, "train", shape=(None, L)),
            _dev(pairs, torch.int32, "pairs", shape=(P, 2)), P, L, int(W))
    with _on([test, train, pairs, out], stream):
        tail = (_dev(out, test.dtype, "out", shape=(P,)), _stream(stream))
        if f64:
            _check(lib.dtw_windowed_f64(*args, *tail), "dtw_windowed_f64")
        else:
            _check(lib.dtw_windowed_ex(*args, int(flags), *tail), "dtw_windowed")
    return out


def nn_dtw_workspace_size(N: int, Q: int, L: int, W: int, V: int, fp64: bool = False) -> int:
    return int(load().nn_dtw_workspace_size(N, Q, L, W, V, 1 if fp64 else 0))


@dataclass
class SearchResult:
    nn_idx: object
    nn_label: object
    nn_dist: object
    stats: dict | None = None


def nn_dtw_search(train, labels, test, W: int, V: int, env=None, flags: int = 0,
                  workspace=None, out=None, stats: bool = False, stream=None) -> SearchResult:
    """Exact 1-NN under DTW_W with LB_Enhanced^V pruning (FP32 or FP64 by dtype)."""
    import torch
    lib = load()
    f64 = _fp(train)
    N, L = train.shape
    Q = test.shape[0]
    need = lib.nn_dtw_workspace_size(N, Q, L, int(W), int(V), 1 if f64 else 0)
    if need == 0:
        raise NnDtwError(EINVAL, "nn_dtw_workspace_size")
    if workspace is None:
        workspace = torch.empty((need,), dtype=torch.uint8, device=train.device)
    if out is None:
        out = (torch.empty((Q,), dtype=torch.int32, device=train.device),
               torch.empty((Q,), dtype=torch.int32, device=train.device),
               torch.empty((Q,), dtype=torch.float64, device=train.device))
    idx, lab, dist = out
    st = Stats() if stats else None
    fn = lib.nn_dtw_search_f64 if f64 else lib.nn_dtw_search
    envp = _dev(env, train.dtype, "env", shape=(N, L, 2)) if env is not None else None
    with _on([train, labels, test, env, idx, lab, dist, workspace], stream):
        _check(fn(_dev(train, train.dtype, "train", 2), _dev(labels, torch.int32, "labels", shape=(N,)),
                N, _dev(test, train.dtype, "test", shape=(Q, L)), Q, L, int(W), int(V), envp,
                int(flags), _dev(idx, torch.int32, "nn_idx", shape=(Q,)),
                _dev(lab, torch.int32, "nn_label", shape=(Q,)),
                _dev(dist, torch.float64, "nn_dist", shape=(Q,)),
                _dev(workspace, torch.uint8, "workspace"),
                workspace.numel(), ctypes.byref(st) if st is not None else None, _stream(stream)),
             "nn_dtw_search")
    return SearchResult(idx, lab, dist, st.as_dict() if st is not None else None)


def nn_dtw_search_noalloc(train, labels, test, W: int, V: int, env=None, flags: int = 0,
                          out=None, stats: bool = False, stream=None) -> SearchResult:
    """The FP32 search with the library's fixed scratch array: no device memory
    is allocated for scratch (see include/nndtw.h; at most
    NNDTW_NOALLOC_SCRATCH_BYTES of workspace).  Outputs are the caller's
    (allocated here only when ``out`` is not given)."""
    import torch
    lib = load()
    N, L = train.shape
    Q = test.shape[0]
    if out is None:
        out = (torch.empty((Q,), dtype=torch.int32, device=train.device),
               torch.empty((Q,), dtype=torch.int32, device=train.device),
               torch.empty((Q,), dtype=torch.float64, device=train.device))
    idx, lab, dist = out
    st = Stats() if stats else None
    envp = _dev(env, torch.float32, "env", shape=(N, L, 2)) if env is not None else None
    with _on([train, labels, test, env, idx, lab, dist], stream):
        _check(lib.nn_dtw_search_noalloc(
          _dev(train, torch.float32, "train", 2), _dev(labels, torch.int32, "labels", shape=(N,)),
          N, _dev(test, torch.float32, "test", shape=(Q, L)), Q, L, int(W), int(V), envp,
          int(flags), _dev(idx, torch.int32, "nn_idx", shape=(Q,)),
          _dev(lab, torch.int32, "nn_label", shape=(Q,)),
          _dev(dist, torch.float64, "nn_dist", shape=(Q,)), ctypes.byref(st) if st is not None else None,
          _stream(stream)), "nn_dtw_search_noalloc")
    return SearchResult(idx, lab, dist, st.as_dict() if st is not None else None)


def nn_dtw_search_f64(train, labels, test, W: int, V: int, **kw) -> SearchResult:
    import torch
    if train.dtype != torch.float64:
        raise TypeError("nn_dtw_search_f64 takes float64 tensors")
    return nn_dtw_search(train, labels, test, W, V, **kw)


def _descs(sets, outs, sizing=False):
    """Descriptors of the datasets; with sizing (workspace-size queries, which
    write nothing) the output tensors may be placeholders of any size."""
    import torch
    arr = (DatasetDesc * len(sets))()
    for i, (d, o) in enumerate(zip(sets, outs)):
        train, test = d["train"], d["test"]
        N, L = train.shape
        Q = test.shape[0]
        qs = None if sizing else (Q,)
        env = d.get("env")
        arr[i] = DatasetDesc(
            _dev(train, torch.float32, "train", 2),
            _dev(d["labels"], torch.int32, "labels", shape=(N,)), N,
            _dev(test, torch.float32, "test", shape=(Q, L)), Q, L, int(d["W"]), int(d["V"]),
            _dev(env, torch.float32, "env", shape=(N, L, 2)) if env is not None else None,
            _dev(o[0], torch.int32, "nn_idx", shape=qs),
            _dev(o[1], torch.int32, "nn_label", shape=qs),
            _dev(o[2], torch.float64, "nn_dist", shape=qs), int(d.get("flags", 0)))
    return arr


def _set_tensors(sets, outs):
    """Every tensor of a batch's descriptors, for the one-device check."""
    ts = []
    for d, o in zip(sets, outs):
        ts += [d["train"], d["labels"], d["test"], d.get("env"), *o]
    return ts


def _windows_array(windows):
    w = np.ascontiguousarray(np.asarray(windows, dtype=np.int32))
    if w.ndim != 1 or w.size == 0:
        raise ValueError("windows must be a non-empty 1-D list")
    return w


def nn_dtw_learn_window_workspace_size(N: int, L: int, windows, V: int) -> int:
    w = _windows_array(windows)
    return int(load().nn_dtw_learn_window_workspace_size(N, L, w.ctypes.data, w.size, V))


def nn_dtw_learn_window(train, labels, windows, V: int, flags: int = 0, workspace=None,
                        correct=None, stream=None):
    """Window learning by leave-one-out 1-NN on a training set: for every
    candidate window, the number of training series whose leave-one-out
    nearest neighbour has the same label (int64 tensor [len(windows)])."""
    import torch
    lib = load()
    N, L = train.shape
    w = _windows_array(windows)
    if workspace is None:
        n = nn_dtw_learn_window_workspace_size(N, L, w, V)
        if n == 0:
            raise NnDtwError(EINVAL, "nn_dtw_learn_window_workspace_size")
        workspace = torch.empty(n, dtype=torch.uint8, device=train.device)
    if correct is None:
        correct = torch.empty(w.size, dtype=torch.int64, device=train.device)
    with _on([train, labels, correct, workspace], stream):
        _check(lib.nn_dtw_learn_window(_dev(train, torch.float32, "train", 2),
                                     _dev(labels, torch.int32, "labels", shape=(N,)), N, L,
                                     w.ctypes.data, w.size, int(V), int(flags),
                                     _dev(correct, torch.int64, "correct", shape=(w.size,)),
                                     _dev(workspace, torch.uint8, "workspace"), workspace.numel(),
                                     _stream(stream)),
             "nn_dtw_learn_window")
    return correct


def learn_window(train, labels, windows, V: int, flags: int = 0):
    """The learned window: the candidate with the highest leave-one-out
    accuracy, the smallest such window among equals.  Returns (W, accuracies)."""
    correct = nn_dtw_learn_window(train, labels, windows, V, flags).cpu().numpy()
    acc = correct / float(train.shape[0])
    w = _windows_array(windows)
    best = max(range(w.size), key=lambda k: (acc[k], -w[k]))
    return int(w[best]), acc


def nn_dtw_batch_workspace_size(sets) -> int:
    import torch
    dev = sets[0]["train"].device if sets else "cuda"
    dummy = [(torch.empty(0, dtype=torch.int32, device=dev),) * 2 +
             (torch.empty(0, dtype=torch.float64, device=dev),) for _ in sets]
    arr = _descs(sets, dummy, sizing=True)
    return int(load().nn_dtw_batch_workspace_size(arr, len(sets)))


def nn_dtw_search_batched(sets, workspace=None, outs=None, flags: int = 0, stream=None):
    """Search many datasets in one call.  ``sets``: list of dicts with keys
    train, labels, test, W, V (and optional env, flags).  Returns one
    SearchResult per dataset."""
    import torch
    lib = load()
    if outs is None:
        outs = [(torch.empty(d["test"].shape[0], dtype=torch.int32, device=d["test"].device),
                 torch.empty(d["test"].shape[0], dtype=torch.int32, device=d["test"].device),
                 torch.empty(d["test"].shape[0], dtype=torch.float64, device=d["test"].device))
                for d in sets]
    arr = _descs(sets, outs)
    need = lib.nn_dtw_batch_workspace_size(arr, len(sets))
    if need == 0:
        raise NnDtwError(EINVAL, "nn_dtw_batch_workspace_size")
    if workspace is None:
        workspace = torch.empty((need,), dtype=torch.uint8, device=sets[0]["train"].device)
    with _on([workspace] + _set_tensors(sets, outs), stream):
        _check(lib.nn_dtw_search_batched(arr, len(sets), _dev(workspace, torch.uint8, "workspace"),
                                       workspace.numel(), int(flags), _stream(stream)),
             "nn_dtw_search_batched")
    return [SearchResult(*o) for o in outs]


class BatchedSearch:
    """A batch of datasets searched by one CUDA graph launch.

    Allocates the outputs and the workspace once, runs the batch eagerly once
    (which also performs the library's one-time set-up outside the capture),
    captures one nn_dtw_search_batched call into a CUDA graph and replays it on
    ``run()``.  Inputs are read from the same tensors at every replay.
    """

    def __init__(self, sets, flags: int = 0, graph: bool = True):
        import torch
        self.sets = sets
        self.flags = flags
        dev = sets[0]["train"].device
        self.outs = [(torch.empty(d["test"].shape[0], dtype=torch.int32, device=dev),
                      torch.empty(d["test"].shape[0], dtype=torch.int32, device=dev),
                      torch.empty(d["test"].shape[0], dtype=torch.float64, device=dev))
                     for d in sets]
        self.workspace = torch.empty((nn_dtw_batch_workspace_size(sets),), dtype=torch.uint8,
                                     device=dev)
        self.graph = None
        with torch.cuda.device(dev):
            self._call()
            torch.cuda.synchronize()
            if graph:
                self.graph = torch.cuda.CUDAGraph()
                s = torch.cuda.Stream()
                s.wait_stream(torch.cuda.current_stream())
                with torch.cuda.stream(s):
                    with torch.cuda.graph(self.graph, stream=s):
                        self._call()
                torch.cuda.current_stream().wait_stream(s)
                torch.cuda.synchronize()

    def _call(self):
        return nn_dtw_search_batched(self.sets, workspace=self.workspace, outs=self.outs,
                                     flags=self.flags)

    def run(self):
        if self.graph is not None:
            self.graph.replay()
        else:
            self._call()
        return [SearchResult(*o) for o in self.outs]


def nn_dtw_host_buffer_size(N: int, Q: int, L: int, W: int, V: int) -> int:
    return int(load().nn_dtw_host_buffer_size(N, Q, L, W, V))


def _host(a, dtype, name, shape=None):
    """Host pointer of a C-contiguous numpy array of the given dtype and
    (with shape) shape: the library copies exactly that many elements."""
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags.c_contiguous:
        raise TypeError(f"{name} must be a C-contiguous numpy {np.dtype(dtype).name} array")
    if shape is not None and tuple(a.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {a.shape}")
    return _vp(a.ctypes.data)


def nn_dtw_search_host(train, labels, test, W: int, V: int, flags: int = 0, buffer=None,
                       out=None, stats: bool = False, stream=None) -> SearchResult:
    """The FP32 search on host (numpy) buffers; copies in and out inside the call."""
    import torch
    lib = load()
    N, L = train.shape
    Q = test.shape[0]
    if out is None:
        out = (np.empty(Q, np.int32), np.empty(Q, np.int32), np.empty(Q, np.float64))
    idx, lab, dist = out
    # host arguments first: the library copies exactly these many elements
    hp = (_host(train, np.float32, "train", (N, L)), _host(labels, np.int32, "labels", (N,)),
          _host(test, np.float32, "test", (Q, L)), _host(idx, np.int32, "nn_idx", (Q,)),
          _host(lab, np.int32, "nn_label", (Q,)), _host(dist, np.float64, "nn_dist", (Q,)))
    need = lib.nn_dtw_host_buffer_size(N, Q, L, int(W), int(V))
    if need == 0:
        raise NnDtwError(EINVAL, "nn_dtw_host_buffer_size")
    if buffer is None:
        buffer = torch.empty((need,), dtype=torch.uint8, device="cuda")
    st = Stats() if stats else None
    with _on([buffer], stream):
        _check(lib.nn_dtw_search_host(
          hp[0], hp[1], N, hp[2], Q, L, int(W), int(V), int(flags), hp[3], hp[4], hp[5],
          _dev(buffer, torch.uint8, "buffer"), buffer.numel(),
          ctypes.byref(st) if st is not None else None, _stream(stream)), "nn_dtw_search_host")
    return SearchResult(idx, lab, dist, st.as_dict() if st is not None else None)


class BatchedHostSearch:
    """The batched search end to end on host (numpy) arrays through
    nn_dtw_search_batched_host: every call copies each dataset's inputs to
    the device, searches the whole batch and copies the results back.
    ``sets``: list of dicts with numpy arrays train (float32 [N, L]), labels
    (int32 [N]), test (float32 [Q, L]) and W, V (optional flags).  The
    output arrays (one (idx, label, dist) triple per dataset, reused by every
    call) and the device buffer are allocated once here; pass pinned arrays
    (and ``outs``) for asynchronous copies."""

    def __init__(self, sets, outs=None, device=None):
        import torch
        lib = load()
        self.sets = sets
        if outs is None:
            outs = [(np.empty(d["test"].shape[0], np.int32), np.empty(d["test"].shape[0], np.int32),
                     np.empty(d["test"].shape[0], np.float64)) for d in sets]
        self.outs = outs
        self.arr = (HostDatasetDesc * len(sets))()
        for i, (d, o) in enumerate(zip(sets, outs)):
            N, L = d["train"].shape
            Q = d["test"].shape[0]
            self.arr[i] = HostDatasetDesc(
                _host(d["train"], np.float32, "train", (N, L)),
                _host(d["labels"], np.int32, "labels", (N,)), N,
                _host(d["test"], np.float32, "test", (Q, L)), Q, L, int(d["W"]), int(d["V"]),
                _host(o[0], np.int32, "nn_idx", (Q,)), _host(o[1], np.int32, "nn_label", (Q,)),
                _host(o[2], np.float64, "nn_dist", (Q,)), int(d.get("flags", 0)))
        need = lib.nn_dtw_batch_host_buffer_size(self.arr, len(sets))
        if need == 0:
            raise NnDtwError(EINVAL, "nn_dtw_batch_host_buffer_size")
        self.buffer = torch.empty((need,), dtype=torch.uint8,
                                  device=device if device is not None else "cuda")

    def run(self, flags: int = 0, stream=None):
        lib = load()
        with _on([self.buffer], stream):
            _check(lib.nn_dtw_search_batched_host(self.arr, len(self.sets),
                                                  _dev(self.buffer, self.buffer.dtype, "buffer"),
                                                  self.buffer.numel(), int(flags),
                                                  _stream(stream)),
                   "nn_dtw_search_batched_host")
        return self.outs


# ------------------------------------------------------------ unequal lengths

@dataclass
class Ragged:
    """A set of series of unequal lengths on the device: series k is
    ``values[offsets[k]:offsets[k+1]]`` (float32 values, int64 offsets with
    n+1 entries); ``max_len`` is the longest length."""
    values: object
    offsets: object
    max_len: int

    def __post_init__(self):
        # The kernels read series k at values[offsets[k] .. offsets[k+1]):
        # offsets that leave the array would make them read past it, so the
        # table is checked once here (one copy of the offsets to the host).
        import torch
        if not (isinstance(self.values, torch.Tensor) and isinstance(self.offsets, torch.Tensor)):
            raise TypeError("Ragged values and offsets must be tensors")
        if self.values.dim() != 1 or self.offsets.dim() != 1 or self.offsets.shape[0] < 1:
            raise ValueError("Ragged values must be 1-D and offsets 1-D with n+1 entries")
        off = self.offsets.detach().to("cpu", torch.int64)
        lens = off[1:] - off[:-1]
        if int(off[0]) != 0 or int(off[-1]) != int(self.values.shape[0]) or bool((lens < 0).any()):
            raise ValueError("Ragged offsets must start at 0, never decrease and end at the "
                             "number of values")
        longest = int(lens.max()) if lens.numel() else 0
        if self.max_len < longest:
            raise ValueError(f"max_len {self.max_len} is below the longest series ({longest})")

    @property
    def n(self) -> int:
        return int(self.offsets.shape[0]) - 1


def ragged(series, device="cuda") -> Ragged:
    """Pack a list of 1-D series into a Ragged set on ``device``."""
    import numpy as np
    import torch
    xs = [np.ascontiguousarray(np.asarray(x, dtype=np.float32).ravel()) for x in series]
    off = np.zeros(len(xs) + 1, np.int64)
    off[1:] = np.cumsum([x.shape[0] for x in xs])
    vals = np.concatenate(xs) if xs else np.zeros(0, np.float32)
    return Ragged(torch.from_numpy(vals).to(device), torch.from_numpy(off).to(device),
                  int(max((x.shape[0] for x in xs), default=0)))


def _ragged_ptrs(r: Ragged, name: str):
    import torch
    n = r.n
    if n < 0:
        raise ValueError(f"{name}.offsets must have at least one entry")
    return (_dev(r.values, torch.float32, f"{name}.values", 1),
            _dev(r.offsets, torch.int64, f"{name}.offsets", shape=(n + 1,)))


def nn_dtw_build_envelopes_varlen(train: Ragged, W: int, env=None, max_len: int | None = None,
                                  stream=None):
    """Envelope rows of every series of a ragged set (rows i < min(L_t + W,
    max_len) of each [max_len, 2] block): tensor [N, max_len, 2]."""
    import torch
    lib = load()
    ml = int(max_len or train.max_len)
    N = train.n
    if env is None:
        env = torch.empty((N, ml, 2), dtype=torch.float32, device=train.values.device)
    v, o = _ragged_ptrs(train, "train")
    with _on([train.values, train.offsets, env], stream):
        _check(lib.nn_dtw_build_envelopes_varlen(
            v, o, N, ml, int(W), _dev(env, torch.float32, "env", shape=(N, ml, 2)),
            _stream(stream)), "nn_dtw_build_envelopes_varlen")
    return env


def lb_enhanced_varlen(test: Ragged, train: Ragged, env, W: int, V: int, keogh: bool = False,
                       safe: bool = False, out=None, max_len: int | None = None, stream=None):
    """LB_Enhanced^V (or LB_Keogh) of every pair of two ragged sets, unequal
    lengths allowed (+inf without a warping path): tensor [Q, N]."""
    import torch
    lib = load()
    ml = int(max_len or max(test.max_len, train.max_len))
    Q, N = test.n, train.n
    if out is None:
        out = torch.empty((Q, N), dtype=torch.float32, device=test.values.device)
    flags = (LB_KEOGH if keogh else 0) | (LB_SAFE if safe else 0)
    tv, to = _ragged_ptrs(test, "test")
    bv, bo = _ragged_ptrs(train, "train")
    with _on([test.values, test.offsets, train.values, train.offsets, env, out], stream):
        _check(lib.lb_enhanced_varlen(
            tv, to, Q, bv, bo, _dev(env, torch.float32, "env", shape=(N, ml, 2)), N, ml, int(W),
            int(V), flags, _dev(out, torch.float32, "out", shape=(Q, N)), _stream(stream)),
            "lb_enhanced_varlen")
    return out


def dtw_windowed_varlen(test: Ragged, train: Ragged, pairs, W: int, out=None,
                        max_len: int | None = None, stream=None):
    """FP32 DTW_W of explicit (q, t) pairs of two ragged sets: tensor [P]."""
    import torch
    lib = load()
    ml = int(max_len or max(test.max_len, train.max_len))
    P = pairs.shape[0]
    if out is None:
        out = torch.empty((P,), dtype=torch.float32, device=test.values.device)
    tv, to = _ragged_ptrs(test, "test")
    bv, bo = _ragged_ptrs(train, "train")
    with _on([test.values, train.values, pairs, out], stream):
        _check(lib.dtw_windowed_varlen(
            tv, to, bv, bo, _dev(pairs, torch.int32, "pairs", shape=(P, 2)), P, ml, int(W),
            _dev(out, torch.float32, "out", shape=(P,)), _stream(stream)), "dtw_windowed_varlen")
    return out


def nn_dtw_varlen_workspace_size(N: int, Q: int, max_len: int, W: int, V: int) -> int:
    return int(load().nn_dtw_varlen_workspace_size(N, Q, max_len, W, V))


def nn_dtw_search_varlen(train: Ragged, labels, test: Ragged, W: int, V: int, flags: int = 0,
                         workspace=None, out=None, stats: bool = False,
                         max_len: int | None = None, stream=None) -> SearchResult:
    """Exact 1-NN under DTW_W for series of unequal lengths (index -1,
    label -1, distance +inf for a query with no training series inside the
    window)."""
    import torch
    lib = load()
    ml = int(max_len or max(test.max_len, train.max_len))
    N, Q = train.n, test.n
    need = lib.nn_dtw_varlen_workspace_size(N, Q, ml, int(W), int(V))
    if need == 0:
        raise NnDtwError(EINVAL, "nn_dtw_varlen_workspace_size")
    dev = train.values.device
    if workspace is None:
        workspace = torch.empty((need,), dtype=torch.uint8, device=dev)
    if out is None:
        out = (torch.empty((Q,), dtype=torch.int32, device=dev),
               torch.empty((Q,), dtype=torch.int32, device=dev),
               torch.empty((Q,), dtype=torch.float64, device=dev))
    idx, lab, dist = out
    st = Stats() if stats else None
    tv, to = _ragged_ptrs(test, "test")
    bv, bo = _ragged_ptrs(train, "train")
    with _on([train.values, train.offsets, labels, test.values, test.offsets, idx, lab, dist,
              workspace], stream):
        _check(lib.nn_dtw_search_varlen(
            bv, bo, _dev(labels, torch.int32, "labels", shape=(N,)), N, tv, to, Q, ml, int(W),
            int(V), int(flags), _dev(idx, torch.int32, "nn_idx", shape=(Q,)),
            _dev(lab, torch.int32, "nn_label", shape=(Q,)),
            _dev(dist, torch.float64, "nn_dist", shape=(Q,)),
            _dev(workspace, torch.uint8, "workspace"), workspace.numel(),
            ctypes.byref(st) if st is not None else None, _stream(stream)),
            "nn_dtw_search_varlen")
    return SearchResult(idx, lab, dist, st.as_dict() if st is not None else None)


class VarlenHostSearch:
    """nn_dtw_search_varlen_host with its device buffer allocated once: the
    unequal-length search end to end on host arrays (values float32,
    offsets int64 with n+1 entries, labels int32; pinned memory makes the
    copies faster).  Results go to host arrays."""

    def __init__(self, train_vals, train_off, labels, test_vals, test_off, W: int, V: int,
                 max_len: int, flags: int = 0, device=None):
        import torch
        self.lib = load()
        for a, dt, name in ((train_vals, np.float32, "train values"),
                            (train_off, np.int64, "train offsets"), (labels, np.int32, "labels"),
                            (test_vals, np.float32, "test values"),
                            (test_off, np.int64, "test offsets")):
            _host(a, dt, name)
        self.tv, self.to, self.lab, self.qv, self.qo = (train_vals, train_off, labels, test_vals,
                                                        test_off)
        self.N, self.Q = self.to.shape[0] - 1, self.qo.shape[0] - 1
        if self.lab.shape != (self.N,):
            raise ValueError(f"labels must have shape ({self.N},)")
        if self.to[-1] != self.tv.shape[0] or self.qo[-1] != self.qv.shape[0]:
            raise ValueError("offsets must end at the number of values")
        self.W, self.V, self.max_len, self.flags = int(W), int(V), int(max_len), int(flags)
        need = self.lib.nn_dtw_varlen_host_buffer_size(
            _vp(self.to.ctypes.data), self.N, _vp(self.qo.ctypes.data), self.Q, self.max_len,
            self.W, self.V)
        if need == 0:
            raise NnDtwError(EINVAL, "nn_dtw_varlen_host_buffer_size")
        self.buf = torch.empty((need,), dtype=torch.uint8, device=device or "cuda")
        self.idx = np.empty(self.Q, np.int32)
        self.nlab = np.empty(self.Q, np.int32)
        self.dist = np.empty(self.Q, np.float64)

    def bytes_per_call(self):
        """(host-to-device, device-to-host) bytes copied by one call."""
        h2d = self.tv.nbytes + self.to.nbytes + self.qv.nbytes + self.qo.nbytes + self.lab.nbytes
        return h2d, self.idx.nbytes + self.nlab.nbytes + self.dist.nbytes

    def __call__(self, stream=None):
        with _on([self.buf], stream):
            _check(self.lib.nn_dtw_search_varlen_host(
                _vp(self.tv.ctypes.data), _vp(self.to.ctypes.data), _vp(self.lab.ctypes.data),
                self.N, _vp(self.qv.ctypes.data), _vp(self.qo.ctypes.data), self.Q,
                self.max_len, self.W, self.V, self.flags, _vp(self.idx.ctypes.data),
                _vp(self.nlab.ctypes.data), _vp(self.dist.ctypes.data),
                _vp(self.buf.data_ptr()), self.buf.numel(), None, _stream(stream)),
                "nn_dtw_search_varlen_host")
        return self.idx, self.nlab, self.dist


def nn_dtw_stage_times() -> dict:
    """Stage times (ms) of this thread's last search run with TIME_STAGES."""
    lib = load()
    buf = (ctypes.c_float * 8)()
    _check(lib.nn_dtw_stage_times(buf), "nn_dtw_stage_times")
    return {name: float(buf[i]) for i, name in enumerate(STAGES)}


def nn_dtw_probe_cell_rate(iters: int = 20000, stream=None) -> float:
    """Measured FP32 DTW cell-update rate of the whole GPU (cells/s), no memory."""
    import torch
    lib = load()
    n = int(lib.nn_dtw_probe_sink_bytes())
    sink = torch.empty((n,), dtype=torch.uint8, device="cuda")
    out = ctypes.c_double(0.0)
    _check(lib.nn_dtw_probe_cell_rate(_dev(sink, torch.uint8, "sink"), n, int(iters),
                                      ctypes.byref(out), _stream(stream)), "nn_dtw_probe_cell_rate")
    return float(out.value)


def nn_dtw_last_call_launches() -> int:
    """Kernel launches issued by this thread's last FP32 search call."""
    return int(load().nn_dtw_last_call_launches())


def nn_dtw_last_call_stage_launches() -> dict:
    """Kernel launches of this thread's last FP32 search call, per stage."""
    buf = (ctypes.c_longlong * 8)()
    _check(load().nn_dtw_last_call_stage_launches(buf), "nn_dtw_last_call_stage_launches")
    return {name: int(buf[i]) for i, name in enumerate(STAGES[:7])}


def nn_dtw_strerror(code: int) -> str:
    return load().nn_dtw_strerror(int(code)).decode()


def nn_dtw_version() -> int:
    return int(load().nn_dtw_version())
