"""The seeded synthetic inputs match their stated recipe (layout, seeds, noise unit, source
model, ratio cube, batch sizes, benchmark cubes).  These generators hold none of the
method's arithmetic; both the oracle and the CUDA path take their inputs from them."""
import math

import numpy as np

import scene
from scene import cubes


def test_layout_dtype_and_determinism():
    a = scene.tiny_cube(config_id=3, dims=(40, 24, 16), n_sources=2)
    b = scene.tiny_cube(config_id=3, dims=(40, 24, 16), n_sources=2)
    c = scene.tiny_cube(config_id=4, dims=(40, 24, 16), n_sources=2)
    assert a.shape == (16, 24, 40) and a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_noise_is_unit_normal_away_from_sources():
    cube = scene.tiny_cube(config_id=1, dims=(64, 64, 64), n_sources=0)
    assert abs(float(cube.mean())) < 0.01 and abs(float(cube.std()) - 1.0) < 0.01


def test_source_model_peak_position_and_spectral_gradient():
    cube = np.zeros((40, 48, 48), np.float32)
    s = cubes.Source(x=24.0, y=20.0, z=18.0, peak=5.0, sig_major=4.0, sig_minor=2.0, pa=0.0, sig_z=3.0,
                     grad=0.25)
    cubes.add_source(cube, s)
    z, y, x = np.unravel_index(int(np.argmax(cube)), cube.shape)
    assert (x, y, z) == (24, 20, 18) and abs(float(cube.max()) - 5.0) < 1e-5
    # the spectral centroid moves with x (rotating disc): grad channels per voxel
    col_hi, col_lo = cube[:, 20, 32], cube[:, 20, 16]
    zc = lambda col: float((np.arange(40) * col).sum() / col.sum())  # noqa: E731
    assert abs((zc(col_hi) - zc(col_lo)) / 16.0 - 0.25) < 0.01
    # elliptical: the major axis (x, pa = 0) is wider than the minor (y)
    assert cube[18, 20, 24 + 4] > cube[18, 20 + 4, 24]


def test_ratio_cube_is_scaled_first_plus_fresh_noise():
    first = scene.tiny_cube(config_id=1, dims=(32, 32, 32), n_sources=2)
    second = scene.ratio_cube(first, config_id=1)
    resid = second - np.float32(0.3) * first
    assert abs(float(resid.std()) - 1.0) < 0.03 and abs(float(np.corrcoef(resid.ravel(), first.ravel())[0, 1])) < 0.05
    assert np.array_equal(scene.ratio_cube(first, config_id=1, noise=False), (first * np.float32(0.3)))


def test_batch_dims_and_paper_cubes():
    d = scene.batch_dims(n=2000)
    assert d.shape == (2000, 3) and d.min() >= 32 and d.max() <= 256
    logs = np.log(d.astype(np.float64) + 0.5)  # floor of a log-uniform: roughly uniform in log
    assert abs(float(np.median(logs)) - 0.5 * (math.log(32) + math.log(256))) < 0.1
    u = scene.paper_uniform_cube(32)
    assert u.shape == (32, 32, 32) and u.min() >= 0.0 and u.max() < 1.0 and abs(float(u.mean()) - 0.5) < 0.01


def test_paper_standins_follow_their_recipe():
    """The stand-ins for the paper's three cubes: shapes of Section 5.2, noise of unit sigma,
    maxima near the reported maximum / sigma, NaN outside the Antennae mosaic's footprint."""
    for kind, (lo_max, hi_max) in (("ngc2903", (12.0, 25.0)), ("antennae", (50.0, 90.0))):
        c = scene.paper_standin(kind)
        nx, ny, nz = scene.STANDIN_DIMS[kind]
        assert c.shape == (nz, ny, nx) and c.dtype == np.float32
        assert lo_max <= float(np.nanmax(c)) <= hi_max, kind
        corner = c[:, :20, :20]
        if kind == "antennae":
            assert np.isnan(corner).all() and not np.isnan(c[:, ny // 2, nx // 2]).any()
        else:
            assert abs(float(corner.std()) - 1.0) < 0.05
    ha, n2 = scene.paper_standin("gama511867")
    assert ha.shape == n2.shape == (37, 50, 50)
    assert 6.0 <= float(ha.max()) <= 12.0
