"""Host logic of bench.py (CPU only): the algorithmic bytes behind the HBM
figures of the envelope and bound stages."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_stage_bytes_follow_shapes_and_flags():
    import bench
    from paper_1808_09617_gb300 import nndtw
    N, Q, L = 100, 40, 64
    shape = [dict(N=N, Q=Q, L=L)]
    plain = bench.stage_bytes(shape, [0], nndtw)
    # envelopes: every training element read once, its (U, Lo) pair written
    assert plain["envelopes"] == 12 * N * L
    # bounds: the norms and the tiled pass read every series (and the
    # envelopes) once, one FP32 bound written per pair
    assert plain["lb"] == 4 * (Q + N) * L + 4 * (Q * L + 3 * N * L) + 4 * Q * N
    rev = bench.stage_bytes(shape, [nndtw.REVERSE], nndtw)
    assert rev["envelopes"] == plain["envelopes"] + 12 * Q * L
    assert rev["lb"] == plain["lb"] + 4 * Q * N          # the ends-and-bands sums
    imp = bench.stage_bytes(shape, [nndtw.IMPROVED], nndtw)
    assert imp["envelopes"] == plain["envelopes"] + 12 * Q * L + 36 * N * L
    assert imp["lb"] == plain["lb"]
    # switched off by the flags that disable the cascade's second stage
    assert bench.stage_bytes(shape, [nndtw.REVERSE | nndtw.NO_REVERSE], nndtw) == plain
    assert bench.stage_bytes(shape, [nndtw.IMPROVED | nndtw.KEOGH_BOUND], nndtw) == plain
    two = bench.stage_bytes(shape * 2, [0, nndtw.REVERSE], nndtw)
    assert two["lb"] == plain["lb"] + rev["lb"]
