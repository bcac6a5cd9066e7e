"""Pins of the oracle's per-sample filters: intensity clipping (Algorithm 10) and intensity
domain scaling (Algorithm 11), applied to every sample before the transfer function (for
the line ratio, to each cube's sample before the quotient), and the alpha threshold of the
first-moment-inspired colourings (the remedy for faint images in the paper's discussion).
Each pin is a numpy restatement on the spectral-axis view, where every channel is sampled
twice with nearest sampling (Section 2.2)."""
import numpy as np
import pytest

import scene

LO, HI = -3.0, 8.0


@pytest.fixture(scope="module")
def O(oracle_lib):
    return oracle_lib


@pytest.fixture(scope="module")
def tiny():
    return scene.tiny_cube()


def _img(m):
    return m[::-1, :].repeat(2, 0).repeat(2, 1)


CAM = scene.ortho_axis_camera((64, 64, 64), 128, 128)


def _clip(c, tmin, tmax):
    return np.where((c < tmin) | (c > tmax), LO, c)


def _scale(c, tmin, tmax):
    return np.where((c < tmin) | (c > tmax), LO, (c - tmin) / (tmax - tmin))


@pytest.mark.parametrize("mode", ["mip", "avg"])
def test_clip_beyond_the_data_is_identity(O, tiny, mode):
    a = O.render(tiny, CAM, mode, interp="trilinear", lut=scene.linear_lut())
    b = O.render(tiny, CAM, mode, interp="trilinear", lut=scene.linear_lut(), filter="clip",
                 min_threshold=float(tiny.min()) - 1, max_threshold=float(tiny.max()) + 1)
    assert np.array_equal(a["scalar"], b["scalar"]) and np.array_equal(a["rgba"], b["rgba"])


@pytest.mark.parametrize("tmin,tmax", [(0.5, 4.0), (-1.0, 2.5), (1.5, 1.5)])
def test_clip_moment_maps(O, tiny, tmin, tmax):
    c = tiny.astype(np.float64)
    mip = O.render(tiny, CAM, "mip", interp="nearest", lut=scene.linear_lut(), filter="clip",
                   min_threshold=tmin, max_threshold=tmax)
    assert np.array_equal(mip["scalar"], _img(_clip(c, tmin, tmax).max(axis=0)))
    avg = O.render(tiny, CAM, "avg", interp="nearest", lut=scene.linear_lut(), filter="clip",
                   min_threshold=tmin, max_threshold=tmax)
    assert np.allclose(avg["scalar"], _img(_clip(c, tmin, tmax).mean(axis=0)), rtol=0, atol=1e-13)


@pytest.mark.parametrize("tmin,tmax", [(0.5, 4.0), (-1.0, 2.5)])
def test_scale_moment_maps(O, tiny, tmin, tmax):
    c = tiny.astype(np.float64)
    mip = O.render(tiny, CAM, "mip", interp="nearest", lut=scene.linear_lut(), filter="scale",
                   min_threshold=tmin, max_threshold=tmax)
    assert np.allclose(mip["scalar"], _img(_scale(c, tmin, tmax).max(axis=0)), rtol=0, atol=1e-15)
    avg = O.render(tiny, CAM, "avg", interp="nearest", lut=scene.linear_lut(), filter="scale",
                   min_threshold=tmin, max_threshold=tmax)
    assert np.allclose(avg["scalar"], _img(_scale(c, tmin, tmax).mean(axis=0)), rtol=0, atol=1e-13)
    kept = (c >= tmin) & (c <= tmax)
    assert kept.any() and (~kept).any()


def test_ratio_filters_each_cube(O, tiny):
    c1 = tiny.astype(np.float64)
    c2 = scene.ratio_cube(tiny, config_id=1).astype(np.float64)
    tmin, tmax = 0.8, 6.0
    r = O.render(tiny, CAM, "ratio", interp="nearest", lut=scene.ratio_lut(), cube2=c2.astype(np.float32),
                 lo=0.0, hi=1.0, ratio_floor=0.0, filter="clip", min_threshold=tmin, max_threshold=tmax)
    f1 = np.where((c1 < tmin) | (c1 > tmax), 0.0, c1)
    f2 = np.where((c2 < tmin) | (c2 > tmax), 0.0, c2)
    with np.errstate(divide="ignore", invalid="ignore"):
        q = np.where(f1 > 0.0, f2 / f1, 0.0)
    assert np.allclose(r["scalar"], _img(q.max(axis=0)), rtol=0, atol=1e-14)


def test_alpha_threshold(O, tiny):
    tmin = 3.0
    a = O.render(tiny, CAM, "spectral", interp="nearest", lut=scene.linear_lut(), alpha_threshold=True,
                 min_threshold=tmin)
    b = O.render(tiny, CAM, "spectral", interp="nearest", lut=scene.linear_lut())
    mx = tiny.astype(np.float64).max(axis=0)
    assert np.array_equal(a["rgba"][..., 3], _img((mx > tmin).astype(np.float64)))
    assert np.array_equal(a["rgba"][..., :3], b["rgba"][..., :3]) and np.array_equal(a["scalar"], b["scalar"])
    m1 = O.render(tiny, CAM, "moment1", interp="nearest", lut=scene.linear_lut(), alpha_threshold=True,
                  min_threshold=0.0)
    mean = tiny.astype(np.float64).mean(axis=0)
    assert np.array_equal(m1["rgba"][..., 3], _img((mean > 0.0).astype(np.float64)))


def test_filter_arguments_checked(O, tiny):
    with pytest.raises(ValueError):
        O.render(tiny, CAM, "mip", lut=scene.linear_lut(), filter="clip", min_threshold=2.0, max_threshold=1.0)
    with pytest.raises(ValueError):
        O.render(tiny, CAM, "mip", lut=scene.linear_lut(), filter="scale", min_threshold=1.0, max_threshold=1.0)
