"""FP64 CPU oracle for NN-DTW with LB_Enhanced^V (arXiv 1808.09617).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
CUDA library never imports, links or calls it, and it shares no code with the
CUDA path (no kernels, headers, helpers, tables or pre/post-processing).

The arithmetic lives in ``nndtw_oracle.c`` (plain loops, double precision,
``-ffp-contract=off``); this module compiles it with gcc, loads it with ctypes
and converts numpy inputs to float64 (FP32 inputs are promoted exactly).

Functions and the passage of the paper each one follows:

=====================  ====================================================
``envelope``           Sec. 2.2.3, Eq. 3-4 (naive window scan)
``dtw``                Sec. 2.1, Eq. 1-2 with the warping window W
``ed``                 DTW_0, squared Euclidean distance (Sec. 2.1)
``lb_keogh``           Sec. 2.2.3 (LB_Keogh)
``lb_enhanced``        Sec. 3.1, Eq. 7 / Algorithm 1
``lb_improved``        Sec. 2.2.4, Eq. 5 (LB_Improved)
``lb_new``             Sec. 2.2.5 (LB_New)
``nn_brute``           1-NN by exhaustive DTW (Sec. 1, the task itself)
``nn_pruned``          the paper's lower-bound search protocol (Sec. 4)
``*_var``              the same for series of unequal lengths (Sec. 2:
                       the equal-length exposition generalises); ragged
                       sets are (values, offsets) pairs
=====================  ====================================================
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nndtw_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_d = ctypes.POINTER(ctypes.c_double)
_i32 = ctypes.POINTER(ctypes.c_int32)
_i64 = ctypes.POINTER(ctypes.c_int64)


def compile_oracle(src: str = _SRC, out: str = _LIB_PATH) -> str:
    """Compile the oracle C file into a shared library with gcc."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-std=c11", "-D_GNU_SOURCE", src, "-o", tmp, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _declare(lib):
    lib.oracle_envelope.argtypes = [_d, ctypes.c_int, ctypes.c_int, _d, _d]
    lib.oracle_envelope.restype = None
    lib.oracle_envelopes.argtypes = [_d, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _d, _d]
    lib.oracle_envelopes.restype = None
    lib.oracle_dtw.argtypes = [_d, _d, ctypes.c_int, ctypes.c_int]
    lib.oracle_dtw.restype = ctypes.c_double
    lib.oracle_dtw_abandon.argtypes = [_d, _d, ctypes.c_int, ctypes.c_int, ctypes.c_double]
    lib.oracle_dtw_abandon.restype = ctypes.c_double
    lib.oracle_ed.argtypes = [_d, _d, ctypes.c_int]
    lib.oracle_ed.restype = ctypes.c_double
    lib.oracle_lb_keogh.argtypes = [_d, _d, _d, ctypes.c_int]
    lib.oracle_lb_keogh.restype = ctypes.c_double
    lib.oracle_lb_enhanced.argtypes = [_d, _d, _d, _d, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_double]
    lib.oracle_lb_enhanced.restype = ctypes.c_double
    lib.oracle_lb_enhanced_improved.argtypes = [_d, _d, _d, _d, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_int]
    lib.oracle_lb_enhanced_improved.restype = ctypes.c_double
    lib.oracle_lb_improved.argtypes = [_d, _d, _d, _d, ctypes.c_int, ctypes.c_int]
    lib.oracle_lb_improved.restype = ctypes.c_double
    lib.oracle_lb_new.argtypes = [_d, _d, ctypes.c_int, ctypes.c_int]
    lib.oracle_lb_new.restype = ctypes.c_double
    lib.oracle_lb_matrix.argtypes = [_d, ctypes.c_int64, _d, _d, _d, ctypes.c_int64,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     _d, ctypes.c_int]
    lib.oracle_lb_matrix.restype = None
    lib.oracle_dtw_pairs.argtypes = [_d, _d, ctypes.c_int64, _i32, ctypes.c_int64,
                                     ctypes.c_int, ctypes.c_int, _d, ctypes.c_int]
    lib.oracle_dtw_pairs.restype = None
    lib.oracle_nn_brute.argtypes = [_d, _i32, ctypes.c_int64, _d, ctypes.c_int64,
                                    ctypes.c_int, ctypes.c_int, _i32, _i32, _d, ctypes.c_int]
    lib.oracle_nn_brute.restype = None
    lib.oracle_nn_loo.argtypes = [_d, _i32, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _i32,
                                  _i32, _d, ctypes.c_int]
    lib.oracle_nn_loo.restype = None
    lib.oracle_nn_pruned.argtypes = [_d, _i32, _d, _d, ctypes.c_int64, _d, ctypes.c_int64,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_int, _i32, _i32, _d,
                                     _i64, ctypes.c_int]
    lib.oracle_nn_pruned.restype = None
    lib.oracle_envelope_var.argtypes = [_d, ctypes.c_int, ctypes.c_int, ctypes.c_int, _d, _d]
    lib.oracle_envelope_var.restype = None
    lib.oracle_dtw_var.argtypes = [_d, ctypes.c_int, _d, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_double]
    lib.oracle_dtw_var.restype = ctypes.c_double
    lib.oracle_lb_keogh_var.argtypes = [_d, ctypes.c_int, ctypes.c_int, _d, _d, ctypes.c_int]
    lib.oracle_lb_keogh_var.restype = ctypes.c_double
    lib.oracle_lb_enhanced_var.argtypes = [_d, ctypes.c_int, _d, ctypes.c_int, _d, _d,
                                           ctypes.c_int, ctypes.c_int, ctypes.c_double]
    lib.oracle_lb_enhanced_var.restype = ctypes.c_double
    lib.oracle_envelopes_var.argtypes = [_d, _i64, ctypes.c_int64, ctypes.c_int, _i64, _d, _d]
    lib.oracle_envelopes_var.restype = None
    lib.oracle_lb_matrix_var.argtypes = [_d, _i64, ctypes.c_int64, _d, _i64, _d, _d, _i64,
                                         ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, _d, ctypes.c_int]
    lib.oracle_lb_matrix_var.restype = None
    lib.oracle_dtw_matrix_var.argtypes = [_d, _i64, ctypes.c_int64, _d, _i64, ctypes.c_int64,
                                          ctypes.c_int, _d, ctypes.c_int]
    lib.oracle_dtw_matrix_var.restype = None
    lib.oracle_nn_brute_var.argtypes = [_d, _i64, _i32, ctypes.c_int64, _d, _i64,
                                        ctypes.c_int64, ctypes.c_int, _i32, _i32, _d,
                                        ctypes.c_int]
    lib.oracle_nn_brute_var.restype = None
    lib.oracle_nn_pruned_var.argtypes = [_d, _i64, _i32, _d, _d, _i64, ctypes.c_int64, _d,
                                         _i64, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                         _i32, _i32, _d, _i64, ctypes.c_int]
    lib.oracle_nn_pruned_var.restype = None
    return lib


def load(path: str | None = None):
    """Load (compiling first if needed) the oracle library.  With ``path`` given,
    load that library instead (the mutation tests compile altered copies)."""
    global _lib
    if path is not None:
        return _declare(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            stale = (not os.path.exists(_LIB_PATH)
                     or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
            if stale:
                compile_oracle()
            _lib = _declare(ctypes.CDLL(_LIB_PATH))
    return _lib


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)))


def _f64(x):
    return np.ascontiguousarray(np.asarray(x), dtype=np.float64)


def _p(a, t=_d):
    return a.ctypes.data_as(t)


class Oracle:
    """Typed numpy front end over one loaded oracle library."""

    def __init__(self, lib=None):
        self.lib = lib if lib is not None else load()

    # -- single-series routines -------------------------------------------
    def envelope(self, b, W):
        b = _f64(b)
        L = b.shape[-1]
        U = np.empty(L); Lo = np.empty(L)
        self.lib.oracle_envelope(_p(b), L, int(W), _p(U), _p(Lo))
        return U, Lo

    def dtw(self, a, b, W, cutoff=np.inf):
        a = _f64(a); b = _f64(b)
        assert a.shape == b.shape and a.ndim == 1
        return self.lib.oracle_dtw_abandon(_p(a), _p(b), a.shape[0], int(W), float(cutoff))

    def ed(self, a, b):
        a = _f64(a); b = _f64(b)
        return self.lib.oracle_ed(_p(a), _p(b), a.shape[0])

    def lb_keogh(self, a, U, Lo):
        a = _f64(a); U = _f64(U); Lo = _f64(Lo)
        return self.lib.oracle_lb_keogh(_p(a), _p(U), _p(Lo), a.shape[0])

    def lb_enhanced(self, a, b, U, Lo, W, V, D=np.inf):
        a = _f64(a); b = _f64(b); U = _f64(U); Lo = _f64(Lo)
        return self.lib.oracle_lb_enhanced(_p(a), _p(b), _p(U), _p(Lo), a.shape[0],
                                           int(W), int(V), float(D))

    def lb_enhanced_improved(self, a, b, U, Lo, W, V):
        """LB_Enhanced^V with the LB_Improved bridge (Sec. 5, Sec. 2.2.4)."""
        a = _f64(a); b = _f64(b); U = _f64(U); Lo = _f64(Lo)
        return self.lib.oracle_lb_enhanced_improved(_p(a), _p(b), _p(U), _p(Lo), a.shape[0],
                                                    int(W), int(V))

    def lb_improved(self, a, b, U, Lo, W):
        """LB_Improved (Sec. 2.2.4): LB_Keogh(A, B) + LB_Keogh(B, A')."""
        a = _f64(a); b = _f64(b); U = _f64(U); Lo = _f64(Lo)
        return self.lib.oracle_lb_improved(_p(a), _p(b), _p(U), _p(Lo), a.shape[0], int(W))

    def lb_new(self, a, b, W):
        """LB_New (Sec. 2.2.5)."""
        a = _f64(a); b = _f64(b)
        assert a.shape == b.shape and a.ndim == 1 and a.shape[0] >= 2
        return self.lib.oracle_lb_new(_p(a), _p(b), a.shape[0], int(W))

    # -- batched drivers ----------------------------------------------------
    def envelopes(self, train, W):
        train = _f64(train)
        N, L = train.shape
        U = np.empty((N, L)); Lo = np.empty((N, L))
        self.lib.oracle_envelopes(_p(train), N, L, int(W), _p(U), _p(Lo))
        return U, Lo

    def lb_matrix(self, test, train, W, V, kind="enhanced", env=None, threads=None):
        test = _f64(test); train = _f64(train)
        Q, L = test.shape
        N = train.shape[0]
        U, Lo = env if env is not None else self.envelopes(train, W)
        U = _f64(U); Lo = _f64(Lo)
        out = np.empty((Q, N))
        k = {"enhanced": 0, "keogh": 1, "improved": 2, "lb_improved": 3, "new": 4}[kind]
        self.lib.oracle_lb_matrix(_p(test), Q, _p(train), _p(U), _p(Lo), N, L, int(W),
                                  int(V), k, _p(out), threads or default_threads())
        return out

    def dtw_pairs(self, test, train, W, pairs=None, threads=None):
        """DTW_W for explicit (q, t) pairs, or the full Q x N matrix."""
        test = _f64(test); train = _f64(train)
        Q, L = test.shape
        N = train.shape[0]
        if pairs is None:
            P = Q * N
            out = np.empty(P)
            self.lib.oracle_dtw_pairs(_p(test), _p(train), N, None, P, L, int(W), _p(out),
                                      threads or default_threads())
            return out.reshape(Q, N)
        pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
        P = pairs.shape[0]
        out = np.empty(P)
        self.lib.oracle_dtw_pairs(_p(test), _p(train), N, _p(pairs, _i32), P, L, int(W),
                                  _p(out), threads or default_threads())
        return out

    def nn_brute(self, train, labels, test, W, threads=None):
        train = _f64(train); test = _f64(test)
        labels = np.ascontiguousarray(labels, dtype=np.int32)
        N, L = train.shape
        Q = test.shape[0]
        idx = np.empty(Q, np.int32); lab = np.empty(Q, np.int32); dist = np.empty(Q)
        self.lib.oracle_nn_brute(_p(train), _p(labels, _i32), N, _p(test), Q, L, int(W),
                                 _p(idx, _i32), _p(lab, _i32), _p(dist),
                                 threads or default_threads())
        return idx, lab, dist

    def nn_loo(self, train, labels, W, threads=None):
        """Leave-one-out 1-NN of every training series among the others."""
        train = _f64(train)
        labels = np.ascontiguousarray(labels, dtype=np.int32)
        N, L = train.shape
        idx = np.empty(N, np.int32); lab = np.empty(N, np.int32); dist = np.empty(N)
        self.lib.oracle_nn_loo(_p(train), _p(labels, _i32), N, L, int(W), _p(idx, _i32),
                               _p(lab, _i32), _p(dist), threads or default_threads())
        return idx, lab, dist

    def loo_correct(self, train, labels, windows, threads=None):
        """Window learning: for each W, the number of training series whose
        leave-one-out nearest neighbour has the same label."""
        labels = np.ascontiguousarray(labels, dtype=np.int32)
        return np.array([int((self.nn_loo(train, labels, W, threads)[1] == labels).sum())
                         for W in windows], np.int64)

    def nn_pruned(self, train, labels, test, W, V, env=None, threads=None):
        """Returns (idx, label, dist, stats) with stats = (lb_pruned, abandoned, completed)."""
        train = _f64(train); test = _f64(test)
        labels = np.ascontiguousarray(labels, dtype=np.int32)
        N, L = train.shape
        Q = test.shape[0]
        U, Lo = env if env is not None else self.envelopes(train, W)
        U = _f64(U); Lo = _f64(Lo)
        idx = np.empty(Q, np.int32); lab = np.empty(Q, np.int32); dist = np.empty(Q)
        st = np.zeros(3, np.int64)
        self.lib.oracle_nn_pruned(_p(train), _p(labels, _i32), _p(U), _p(Lo), N, _p(test), Q,
                                  L, int(W), int(V), _p(idx, _i32), _p(lab, _i32), _p(dist),
                                  _p(st, _i64), threads or default_threads())
        return idx, lab, dist, st

    # -- unequal lengths (ragged sets: values and offsets) --------------------
    def envelope_var(self, b, W, E=None):
        """B's envelope for the rows 1..E of a series compared with it
        (default E = len(b) + W, the longest series with a path)."""
        b = _f64(b)
        E = b.shape[0] + int(W) if E is None else int(E)
        assert 1 <= E <= b.shape[0] + int(W)
        U = np.empty(E); Lo = np.empty(E)
        self.lib.oracle_envelope_var(_p(b), b.shape[0], int(W), E, _p(U), _p(Lo))
        return U, Lo

    def dtw_var(self, a, b, W, cutoff=np.inf):
        a = _f64(a); b = _f64(b)
        return self.lib.oracle_dtw_var(_p(a), a.shape[0], _p(b), b.shape[0], int(W),
                                       float(cutoff))

    def lb_keogh_var(self, a, b, W):
        a = _f64(a); b = _f64(b)
        U, Lo = self.envelope_var(b, W)
        if a.shape[0] > U.shape[0]:
            return np.inf
        return self.lib.oracle_lb_keogh_var(_p(a), a.shape[0], b.shape[0], _p(U), _p(Lo),
                                            int(W))

    def lb_enhanced_var(self, a, b, W, V, D=np.inf):
        a = _f64(a); b = _f64(b)
        assert a.shape[0] >= 2 and b.shape[0] >= 2
        U, Lo = self.envelope_var(b, W)
        if a.shape[0] > U.shape[0]:
            return np.inf
        return self.lib.oracle_lb_enhanced_var(_p(a), a.shape[0], _p(b), b.shape[0], _p(U),
                                               _p(Lo), int(W), int(V), float(D))

    @staticmethod
    def _ragged(vals, off):
        vals = _f64(vals)
        off = np.ascontiguousarray(off, dtype=np.int64)
        assert off.ndim == 1 and off[0] == 0 and off[-1] == vals.shape[0]
        return vals, off

    def envelopes_var(self, train, off, W):
        """Envelopes of a ragged set: (U, Lo, eoff), series t's L_t + W rows
        at eoff[t] = off[t] + t W."""
        train, off = self._ragged(train, off)
        N = off.shape[0] - 1
        eoff = off + np.arange(N + 1, dtype=np.int64) * int(W)
        U = np.empty(int(eoff[-1])); Lo = np.empty(int(eoff[-1]))
        self.lib.oracle_envelopes_var(_p(train), _p(off, _i64), N, int(W), _p(eoff, _i64),
                                      _p(U), _p(Lo))
        return U, Lo, eoff

    def lb_matrix_var(self, test, toff, train, off, W, V, kind="enhanced", env=None,
                      threads=None):
        test, toff = self._ragged(test, toff)
        train, off = self._ragged(train, off)
        Q, N = toff.shape[0] - 1, off.shape[0] - 1
        U, Lo, eoff = env if env is not None else self.envelopes_var(train, off, W)
        out = np.empty((Q, N))
        k = {"enhanced": 0, "keogh": 1}[kind]
        self.lib.oracle_lb_matrix_var(_p(test), _p(toff, _i64), Q, _p(train), _p(off, _i64),
                                      _p(_f64(U)), _p(_f64(Lo)), _p(eoff, _i64), N, int(W),
                                      int(V), k, _p(out), threads or default_threads())
        return out

    def dtw_matrix_var(self, test, toff, train, off, W, threads=None):
        test, toff = self._ragged(test, toff)
        train, off = self._ragged(train, off)
        Q, N = toff.shape[0] - 1, off.shape[0] - 1
        out = np.empty((Q, N))
        self.lib.oracle_dtw_matrix_var(_p(test), _p(toff, _i64), Q, _p(train), _p(off, _i64),
                                       N, int(W), _p(out), threads or default_threads())
        return out

    def nn_brute_var(self, train, off, labels, test, toff, W, threads=None):
        train, off = self._ragged(train, off)
        test, toff = self._ragged(test, toff)
        labels = np.ascontiguousarray(labels, dtype=np.int32)
        N, Q = off.shape[0] - 1, toff.shape[0] - 1
        idx = np.empty(Q, np.int32); lab = np.empty(Q, np.int32); dist = np.empty(Q)
        self.lib.oracle_nn_brute_var(_p(train), _p(off, _i64), _p(labels, _i32), N, _p(test),
                                     _p(toff, _i64), Q, int(W), _p(idx, _i32), _p(lab, _i32),
                                     _p(dist), threads or default_threads())
        return idx, lab, dist

    def nn_pruned_var(self, train, off, labels, test, toff, W, V, env=None, threads=None):
        """Returns (idx, label, dist, stats), stats = (lb_pruned, abandoned, completed)."""
        train, off = self._ragged(train, off)
        test, toff = self._ragged(test, toff)
        labels = np.ascontiguousarray(labels, dtype=np.int32)
        N, Q = off.shape[0] - 1, toff.shape[0] - 1
        U, Lo, eoff = env if env is not None else self.envelopes_var(train, off, W)
        idx = np.empty(Q, np.int32); lab = np.empty(Q, np.int32); dist = np.empty(Q)
        st = np.zeros(3, np.int64)
        self.lib.oracle_nn_pruned_var(_p(train), _p(off, _i64), _p(labels, _i32),
                                      _p(_f64(U)), _p(_f64(Lo)), _p(eoff, _i64), N, _p(test),
                                      _p(toff, _i64), Q, int(W), int(V), _p(idx, _i32),
                                      _p(lab, _i32), _p(dist), _p(st, _i64),
                                      threads or default_threads())
        return idx, lab, dist, st


_default = None


def get() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle()
    return _default
