"""The library's tap tables for in-ray smoothing, called through the C ABI on the host (no
GPU): the linear-sampling fold reproduces the offsets and coefficients Algorithm 9 prints,
and the N-tap binomial filters cost Section 6's 3(N-1)/2 + 1 fetches per step."""
import ctypes as C
import json
import math
import os

import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def built_library():
    from paper_1707_00442_gb300 import build
    build.build()


def test_algorithm9_constants():
    from paper_1707_00442_gb300 import binomial_taps, linear_sampling_taps
    g = json.load(open(os.path.join(GOLD, "alg9_ninetap.json")))
    tol = 0.6 * 10.0 ** -g["printed_decimals"]
    for c0, off, w in (binomial_taps(9, drop=2),
                       linear_sampling_taps([math.comb(12, k) / 4070 for k in range(2, 11)])):
        assert len(off) == len(w) == 2
        assert c0 == pytest.approx(g["coeff_0"], abs=tol)
        assert off[0] == pytest.approx(g["offset_1"], abs=tol) and off[1] == pytest.approx(g["offset_2"], abs=tol)
        assert w[0] == pytest.approx(g["coeff_1"], abs=tol) and w[1] == pytest.approx(g["coeff_2"], abs=tol)


def test_binomial_fetch_counts():
    from paper_1707_00442_gb300 import binomial_taps
    g = json.load(open(os.path.join(GOLD, "fetch_counts.json")))
    for N, fetches in zip(g["gaussian_taps"], g["gaussian_fetches"]):
        c0, off, w = binomial_taps(N)
        assert 1 + 6 * len(off) == fetches
        assert c0 + 2 * sum(w) == pytest.approx(1.0, abs=1e-15)  # a normalised kernel


def test_fold_at_integer_points_is_the_kernel():
    """Linear interpolation of a sequence at each folded offset, weighted, equals the
    discrete kernel applied to it (exact algebra of the fold)."""
    import numpy as np
    from paper_1707_00442_gb300 import linear_sampling_taps
    rng = np.random.default_rng(3)
    w = rng.random(11)
    w = (w + w[::-1]) / 2
    c0, off, wt = linear_sampling_taps(w)
    g = rng.normal(size=41)
    x = np.arange(len(g), dtype=np.float64)
    i = 20
    folded = c0 * g[i] + sum(wj * (np.interp(i + o, x, g) + np.interp(i - o, x, g)) for o, wj in zip(off, wt))
    assert folded == pytest.approx(float(np.dot(w, g[i - 5:i + 6])), abs=1e-12)


def test_tap_tables_through_the_abi():
    """The raw C calls: Algorithm 9's printed kernel, and the errors the header states."""
    from paper_1707_00442_gb300 import _lib
    L = _lib.lib()
    c0, nf = C.c_double(), C.c_int32()
    offs, wts = (C.c_double * 4)(), (C.c_double * 4)()
    assert L.shw_binomial_taps(9, 2, C.byref(c0), offs, wts, 4, C.byref(nf)) == _lib.SHW_OK
    g = json.load(open(os.path.join(GOLD, "alg9_ninetap.json")))
    tol = 0.6 * 10.0 ** -g["printed_decimals"]
    assert nf.value == 2 and abs(c0.value - g["coeff_0"]) <= tol
    assert abs(offs[0] - g["offset_1"]) <= tol and abs(offs[1] - g["offset_2"]) <= tol
    assert abs(wts[0] - g["coeff_1"]) <= tol and abs(wts[1] - g["coeff_2"]) <= tol
    # too few output slots, an even tap count, an asymmetric kernel, a row beyond 62
    assert L.shw_binomial_taps(13, 0, C.byref(c0), offs, wts, 2, C.byref(nf)) == _lib.SHW_ENOMEM
    assert L.shw_binomial_taps(8, 0, C.byref(c0), offs, wts, 4, C.byref(nf)) == _lib.SHW_EINVAL
    w = (C.c_double * 3)(0.2, 0.5, 0.3)
    assert L.shw_linear_sampling_taps(w, 1, C.byref(c0), offs, wts, 4, C.byref(nf)) == _lib.SHW_EINVAL
    assert L.shw_binomial_taps(63, 1, C.byref(c0), offs, wts, 4, C.byref(nf)) == _lib.SHW_EUNSUPPORTED
