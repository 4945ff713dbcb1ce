"""The FP64 oracle against the pins of ``oracle_pins`` (CPU only)."""
import pytest

import oracle_pins


@pytest.mark.parametrize("pin", oracle_pins.ALL_PINS, ids=lambda f: f.__name__)
def test_oracle_pin(orc, pin):
    pin(orc)


def test_dtw_paths_length_7(orc):
    """One larger exhaustive case: all 8,989 window-free paths at L=7."""
    import numpy as np
    from oracle import paths
    rng = np.random.default_rng(77)
    a, b = rng.standard_normal(7), rng.standard_normal(7)
    for W in (1, 3, 6):
        exact = paths.dtw_by_paths(a, b, W)
        assert abs(orc.dtw(a, b, W) - exact) <= 1e-12 * exact
