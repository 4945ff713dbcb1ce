"""The C-ABI library loads and exports every declared symbol (CPU only: no
call here touches a GPU; argument validation happens before any CUDA call)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nndtw.h")


@pytest.fixture(scope="module")
def clib():
    from paper_1808_09617_gb300 import build, nndtw
    if not os.path.exists(nndtw.LIB_PATH):
        build.build()
    return nndtw.load()


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"NNDTW_API\s+[\w\s\*]+?\b(\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("nn_dtw_build_envelopes", "lb_enhanced", "nn_dtw_search",
                 "nn_dtw_workspace_size", "nn_dtw_strerror"):
        assert must in names


def test_every_declared_symbol_is_exported(clib):
    for name in declared_symbols():
        assert hasattr(clib, name), name
        assert ctypes.cast(getattr(clib, name), ctypes.c_void_p).value


def test_host_only_calls(clib):
    from paper_1808_09617_gb300 import nndtw
    assert clib.nn_dtw_version() >= 100
    for code in range(0, 7):
        assert clib.nn_dtw_strerror(code)
    assert nndtw.nn_dtw_workspace_size(500, 500, 256, 26, 5) > 500 * 500 * 4
    assert nndtw.nn_dtw_workspace_size(500, 500, 256, 26, 5, fp64=True) > 0
    # invalid sizes give 0 bytes
    assert nndtw.nn_dtw_workspace_size(0, 5, 256, 26, 5) == 0
    assert nndtw.nn_dtw_workspace_size(5, 5, 1, 0, 5) == 0
    assert nndtw.nn_dtw_workspace_size(5, 5, nndtw.NNDTW_MAX_L + 1, 0, 5) == 0
    assert nndtw.nn_dtw_workspace_size(5, 5, nndtw.NNDTW_MAX_L, 0, 5) > 0
    assert nndtw.nn_dtw_workspace_size(5, 5, 64, -1, 5) == 0
    assert nndtw.nn_dtw_workspace_size(5, 5, 64, 3, 0) == 0
    assert nndtw.nn_dtw_host_buffer_size(10, 4, 64, 6, 2) > nndtw.nn_dtw_workspace_size(
        10, 4, 64, 6, 2)


def test_invalid_arguments_rejected_before_cuda(clib):
    from paper_1808_09617_gb300 import nndtw
    vp = ctypes.c_void_p
    # N = 0
    assert clib.nn_dtw_search(vp(8), vp(8), 0, vp(8), 1, 16, 2, 1, None, 0, vp(8), vp(8),
                              vp(8), vp(256), 1 << 20, None, None) == nndtw.EINVAL
    # null pointers
    assert clib.nn_dtw_search(None, vp(8), 4, vp(8), 1, 16, 2, 1, None, 0, vp(8), vp(8),
                              vp(8), vp(256), 1 << 20, None, None) == nndtw.EINVAL
    # misaligned workspace
    assert clib.nn_dtw_search(vp(8), vp(8), 4, vp(8), 1, 16, 2, 1, None, 0, vp(8), vp(8),
                              vp(8), vp(257), 1 << 20, None, None) == nndtw.EINVAL
    # workspace too small
    assert clib.nn_dtw_search(vp(8), vp(8), 4, vp(8), 1, 16, 2, 1, None, 0, vp(8), vp(8),
                              vp(8), vp(256), 16, None, None) == nndtw.ENOSPACE
    # Q = 0 is a no-op
    assert clib.nn_dtw_search(vp(8), vp(8), 4, vp(8), 0, 16, 2, 1, None, 0, vp(8), vp(8),
                              vp(8), vp(256), 1 << 20, None, None) == nndtw.OK
    assert clib.lb_enhanced(vp(8), 2, vp(8), vp(8), 2, 1, 0, 1, 0, vp(8), None) == nndtw.EINVAL
    assert clib.lb_enhanced(vp(8), 2, vp(8), vp(8), 2, 8, 0, 0, 0, vp(8), None) == nndtw.EINVAL
    assert clib.nn_dtw_build_envelopes(None, 3, 8, 1, vp(8), None) == nndtw.EINVAL
    assert clib.nn_dtw_build_envelopes(vp(8), 0, 8, 1, vp(8), None) == nndtw.OK
    assert clib.dtw_windowed(vp(8), vp(8), vp(8), -1, 8, 1, vp(8), None) == nndtw.EINVAL
    assert clib.nn_dtw_search_host(None, None, 4, None, 0, 16, 2, 1, 0, None, None, None,
                                   None, 0, None, None) == nndtw.OK


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1808_09617_gb300 import nndtw
    with pytest.raises(nndtw.NativeLibraryMissing):
        saved = nndtw._lib
        nndtw._lib = None
        try:
            nndtw.load(str(tmp_path / "missing.so"))
        finally:
            nndtw._lib = saved


def test_host_entry_checks_shapes_before_any_copy():
    """The host-buffer entry point copies exactly N*L, Q*L, N and Q elements:
    the binding rejects arrays of any other shape before calling the library
    (no GPU needed to see it)."""
    import numpy as np
    import pytest

    from paper_1808_09617_gb300 import nndtw
    train = np.zeros((10, 32), np.float32)
    test = np.zeros((4, 32), np.float32)
    with pytest.raises(ValueError, match="labels"):
        nndtw.nn_dtw_search_host(train, np.zeros(9, np.int32), test, 3, 2)
    with pytest.raises(ValueError, match="test"):
        nndtw.nn_dtw_search_host(train, np.zeros(10, np.int32), np.zeros((4, 31), np.float32), 3, 2)
    out = (np.empty(3, np.int32), np.empty(4, np.int32), np.empty(4, np.float64))
    with pytest.raises(ValueError, match="nn_idx"):
        nndtw.nn_dtw_search_host(train, np.zeros(10, np.int32), test, 3, 2, out=out)
    with pytest.raises(TypeError, match="train"):
        nndtw.nn_dtw_search_host(train.astype(np.float64), np.zeros(10, np.int32), test, 3, 2)


def test_binding_requires_one_device():
    """Tensors on two GPUs, or a stream of another GPU, are refused before any
    pointer reaches the library (its kernels run on the current device)."""
    import torch
    from paper_1808_09617_gb300 import nndtw
    c0, c1 = torch.device("cuda", 0), torch.device("cuda", 1)
    assert nndtw.one_device([c1, c1, None]) == 1
    with pytest.raises(ValueError):
        nndtw.one_device([c0, c1])
    with pytest.raises(ValueError):
        nndtw.one_device([c0, c0], stream_device=c1)
    with pytest.raises(TypeError):
        nndtw.one_device([torch.device("cpu")])
    with pytest.raises(ValueError):
        nndtw.one_device([])


def test_varlen_arguments_rejected_before_cuda(clib):
    """The unequal-length entry points check sizes, pointers, flags and the
    workspace before any CUDA call."""
    from paper_1808_09617_gb300 import nndtw
    vp = ctypes.c_void_p
    ws = nndtw.nn_dtw_varlen_workspace_size(50, 20, 128, 12, 5)
    assert ws > 50 * 20 * 4
    assert nndtw.nn_dtw_varlen_workspace_size(0, 20, 128, 12, 5) == 0
    assert nndtw.nn_dtw_varlen_workspace_size(50, 20, 1, 12, 5) == 0
    assert nndtw.nn_dtw_varlen_workspace_size(50, 20, nndtw.NNDTW_MAX_L + 1, 12, 5) == 0
    assert nndtw.nn_dtw_varlen_workspace_size(50, 20, 128, -1, 5) == 0
    args = lambda **kw: [kw.get("train", vp(8)), kw.get("toff", vp(8)), vp(8),
                         kw.get("N", 50), vp(8), vp(8), kw.get("Q", 20),
                         kw.get("max_len", 128), kw.get("W", 12), kw.get("V", 5),
                         kw.get("flags", 0), vp(8), vp(8), vp(8), kw.get("ws", vp(256)),
                         kw.get("ws_bytes", ws), None, None]
    f = clib.nn_dtw_search_varlen
    assert f(*args(N=0)) == nndtw.EINVAL
    assert f(*args(train=None)) == nndtw.EINVAL
    assert f(*args(toff=None)) == nndtw.EINVAL
    assert f(*args(max_len=1)) == nndtw.EINVAL
    assert f(*args(W=-2)) == nndtw.EINVAL
    assert f(*args(V=0)) == nndtw.EINVAL
    assert f(*args(ws=vp(257))) == nndtw.EINVAL
    assert f(*args(ws_bytes=ws - 1)) == nndtw.ENOSPACE
    for bad in (nndtw.LEAVE_ONE_OUT, nndtw.REVERSE, nndtw.IMPROVED):
        assert f(*args(flags=bad)) == nndtw.EINVAL
    assert f(*args(Q=0)) == nndtw.OK
    assert clib.nn_dtw_build_envelopes_varlen(None, vp(8), 3, 16, 2, vp(8), None) == nndtw.EINVAL
    assert clib.nn_dtw_build_envelopes_varlen(vp(8), vp(8), 0, 16, 2, vp(8), None) == nndtw.OK
    assert clib.nn_dtw_build_envelopes_varlen(vp(8), vp(8), 3, 1, 2, vp(8), None) == nndtw.EINVAL
    assert clib.lb_enhanced_varlen(vp(8), vp(8), 2, vp(8), vp(8), vp(8), 2, 16, 2, 0, 0, vp(8),
                                   None) == nndtw.EINVAL
    assert clib.lb_enhanced_varlen(vp(8), vp(8), 2, vp(8), vp(8), vp(8), 2, 16, 2, 1,
                                   nndtw.LB_NEW, vp(8), None) == nndtw.EINVAL
    assert clib.dtw_windowed_varlen(vp(8), vp(8), vp(8), vp(8), vp(8), -1, 16, 2, vp(8),
                                    None) == nndtw.EINVAL
    assert clib.dtw_windowed_varlen(vp(8), vp(8), vp(8), vp(8), vp(8), 0, 16, 2, vp(8),
                                    None) == nndtw.OK


def test_varlen_host_entry_checks_offsets_before_any_copy(clib):
    """The host-buffer unequal-length search checks its offset tables on the
    host: a length outside [2, max_len] or a table not starting at 0 is
    rejected before any copy or CUDA call."""
    import numpy as np
    from paper_1808_09617_gb300 import nndtw
    vp = ctypes.c_void_p
    good = np.array([0, 5, 9, 15], np.int64)
    qgood = np.array([0, 6, 12], np.int64)
    assert clib.nn_dtw_varlen_host_buffer_size(vp(good.ctypes.data), 3, vp(qgood.ctypes.data),
                                               2, 8, 2, 2) > 0
    assert clib.nn_dtw_varlen_host_buffer_size(None, 3, vp(qgood.ctypes.data), 2, 8, 2, 2) == 0
    vals = np.zeros(64, np.float32)
    lab = np.zeros(3, np.int32)
    out_i = np.zeros(2, np.int32)
    out_d = np.zeros(2, np.float64)

    def call(off, qoff, max_len=8):
        return clib.nn_dtw_search_varlen_host(
            vp(vals.ctypes.data), vp(off.ctypes.data), vp(lab.ctypes.data), 3,
            vp(vals.ctypes.data), vp(qoff.ctypes.data), 2, max_len, 2, 2, 0,
            vp(out_i.ctypes.data), vp(out_i.ctypes.data), vp(out_d.ctypes.data), vp(256),
            1 << 30, None, None)
    assert call(np.array([0, 5, 6, 15], np.int64), qgood) == nndtw.EINVAL   # length 1
    assert call(good, np.array([0, 6, 15], np.int64)) == nndtw.EINVAL        # longer than 8
    assert call(np.array([1, 5, 9, 15], np.int64), qgood) == nndtw.EINVAL   # not from 0
    assert call(good, np.array([0, 7, 5], np.int64)) == nndtw.EINVAL         # decreasing


def test_ragged_set_checks_its_offsets():
    """A ragged set's offset table is checked when the set is built: the
    kernels would read past the values with a table that leaves them."""
    import torch
    from paper_1808_09617_gb300 import nndtw
    v = torch.zeros(10)
    ok = nndtw.Ragged(v, torch.tensor([0, 4, 10]), 6)
    assert ok.n == 2
    for off, ml in (([0, 4, 11], 7), ([1, 4, 10], 6), ([0, 6, 4, 10], 6), ([0, 4, 10], 5)):
        with pytest.raises(ValueError):
            nndtw.Ragged(v, torch.tensor(off), ml)
    with pytest.raises(ValueError):
        nndtw.Ragged(torch.zeros(2, 5), torch.tensor([0, 10]), 10)
