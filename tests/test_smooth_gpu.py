"""GPU parity of shw_smooth / shw_smooth_weights against the FP64 oracle (Section 4.2)."""
import numpy as np
import pytest

import oracle
import scene
from parity import TOL_F32, shw, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    return shw()


def _gpu_smooth(m, cube, sigma, r):
    out = m.smooth(to_dev(cube), sigma, r)
    m.sync_status()
    return out.cpu().numpy()


# (nx % 4 == 0 and 1 <= r <= 8 take the TMA pipeline; the others the staged kernel)
@pytest.mark.parametrize("dims,sigma,r", [((45, 37, 29), 1.0, 3), ((64, 64, 64), 1.0, 3), ((70, 33, 90), 2.0, 6),
                                         ((31, 40, 17), 0.8, 0), ((50, 50, 50), 5.0, 16), ((33, 65, 40), 3.0, 9),
                                         ((5, 3, 2), 1.5, 4), ((44, 37, 29), 1.0, 3), ((68, 33, 90), 2.0, 6),
                                         ((36, 70, 20), 2.7, 8), ((4, 5, 3), 0.6, 1), ((12, 64, 130), 1.7, 5),
                                         ((96, 40, 300), 2.0, 6), ((8, 8, 8), 3.0, 8)])
def test_smooth_parity(m, dims, sigma, r):
    cube = scene.tiny_cube(config_id=21, dims=dims, n_sources=2)
    g = _gpu_smooth(m, cube, sigma, r)
    o = oracle.smooth(cube, oracle.gauss_weights(sigma, r))
    rng = float(cube.max() - cube.min())
    err = np.abs(g.astype(np.float64) - o).max()
    assert err <= TOL_F32 * rng, err


def test_smooth_delta_is_kernel(m):
    c = np.zeros((15, 15, 15), np.float32)
    c[7, 7, 7] = 1.0
    g = _gpu_smooth(m, c, 1.0, 3)
    w = oracle.gauss_weights(1.0, 3)
    ref = np.zeros_like(g, dtype=np.float64)
    ref[4:11, 4:11, 4:11] = w[:, None, None] * w[None, :, None] * w[None, None, :]
    assert np.abs(g - ref).max() <= 1e-7 and abs(g.sum() - 1) < 1e-5


def test_smooth_weights_binomial(m):
    """The paper's 9-tap filter (b_12's central taps, Algorithm 9) through explicit weights."""
    b12 = oracle.binomial_weights(12)
    w = b12[2:11] / b12[2:11].sum()
    cube = scene.tiny_cube(config_id=22, dims=(40, 36, 52), n_sources=2)
    g = m.smooth_weights(to_dev(cube), w.astype(np.float32))
    m.sync_status()
    o = oracle.smooth(cube, w.astype(np.float32).astype(np.float64))
    assert np.abs(g.cpu().numpy() - o).max() <= TOL_F32 * float(cube.max() - cube.min())


def test_smooth_nan_propagates_locally(m):
    cube = scene.tiny_cube(config_id=23, dims=(32, 32, 32), n_sources=1)
    cube[16, 16, 16] = np.nan
    g = _gpu_smooth(m, cube, 1.0, 2)
    o = oracle.smooth(cube, oracle.gauss_weights(1.0, 2))
    assert np.array_equal(np.isnan(g), np.isnan(o))
    ok = ~np.isnan(o)
    assert np.abs(g[ok] - o[ok]).max() <= TOL_F32 * float(np.nanmax(cube) - np.nanmin(cube))


def test_smooth_tma_and_staged_paths_agree(m):
    cube = scene.tiny_cube(config_id=24, dims=(68, 52, 75), n_sources=2)
    a = _gpu_smooth(m, cube, 2.0, 6)
    with m.debug_flags("smooth_plain"):
        b = _gpu_smooth(m, cube, 2.0, 6)
    assert np.abs(a - b).max() <= 1e-6 * float(cube.max() - cube.min())


def test_smooth_wait_timeout_is_reported_and_recovered(m):
    """Device-side waits are bounded: with SHW_DEBUG_FAULT_TIMEOUT the smoothing leaves one
    plane's tensor copy unissued, every CTA's bounded wait for it runs out, the CTA waits for its
    own copies in flight and returns, and shw_sync_status reports SHW_ETIMEOUT.  The next
    normal call runs clean and correct (no GPU fault is involved)."""
    cube = scene.tiny_cube(config_id=26, dims=(64, 48, 40), n_sources=2)
    ct = to_dev(cube)
    with m.debug_flags("fault_timeout"):
        m.smooth(ct, 1.0, 3)
        with pytest.raises(m.ShwError) as e:
            m.sync_status()
    assert e.value.status == 5  # SHW_ETIMEOUT
    m.sync_status()  # the error word was cleared by the report
    g = _gpu_smooth(m, cube, 1.0, 3)
    o = oracle.smooth(cube, oracle.gauss_weights(1.0, 3))
    assert np.abs(g - o).max() <= TOL_F32 * float(cube.max() - cube.min())
