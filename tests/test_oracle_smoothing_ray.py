"""Pins of the oracle's in-ray smoothing (Section 4.1-4.2): the box along the ray
(Algorithm 8) and the per-axis taps of Algorithm 9, applied to every sample before the
filter and the transfer function.

Readings pinned here: box neighbours lie one voxel apart along the ray's unit direction;
the 3-D taps run Algorithm 9 once per data axis, x then y then z, each pass starting from
the previous pass's value (so a sample costs 1 + 6 M fetches, the count Section 6 gives
for the N-tap kernel).  Each expected value is an independent computation: scipy's
moving average, numpy's discrete convolution with the unmerged binomial kernel, or a
closed form for linear data."""
import json
import math
import os

import numpy as np
import pytest

import scene

LO, HI = -3.0, 8.0
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def O(oracle_lib):
    return oracle_lib


@pytest.fixture(scope="module")
def tiny():
    return scene.tiny_cube(dims=(32, 32, 48))


def _alg9():
    g = json.load(open(os.path.join(GOLD, "alg9_ninetap.json")))
    return g["coeff_0"], [g["offset_1"], g["offset_2"]], [g["coeff_1"], g["coeff_2"]]


def _b12_central9():
    # Algorithm 9's coefficients are b_12 without its two outer taps on each side,
    # renormalised: C(12, k) / 4070, k = 2..10 (Section 4.2)
    w = np.array([math.comb(12, k) for k in range(2, 11)], np.float64)
    return w / w.sum()


@pytest.mark.parametrize("mode", ["mip", "avg", "composite", "spectral"])
def test_box_arm0_and_unit_taps_are_identity(O, tiny, mode):
    cam = scene.orbit_camera(tiny.shape[::-1], 30, 20, 48, 40)
    kw = dict(interp="trilinear", lut=scene.linear_lut(), opacity_scale=0.05)
    a = O.render(tiny, cam, mode, **kw)
    b = O.render(tiny, cam, mode, smooth="box", smooth_arm=0, **kw)
    c = O.render(tiny, cam, mode, smooth="taps", smooth_taps=(1.0, [1.5], [0.0]), **kw)
    for r in (b, c):
        assert np.array_equal(a["scalar"], r["scalar"]) and np.array_equal(a["rgba"], r["rgba"])
        assert np.array_equal(a["nsamples"], r["nsamples"])


@pytest.mark.parametrize("arm", [1, 2, 4])
@pytest.mark.parametrize("step", [1.0, 0.5])
def test_box_spectral_axis_is_a_moving_average(O, tiny, arm, step):
    """Down the spectral axis with nearest sampling the box is scipy's clamped moving
    average along z; MIP and AVG then take the max / mean over channels."""
    from scipy.ndimage import uniform_filter1d
    nz, ny, nx = tiny.shape
    cam = scene.ortho_axis_camera((nx, ny, nz), nx, ny)
    c = tiny.astype(np.float64)
    ma = uniform_filter1d(c, size=2 * arm + 1, axis=0, mode="nearest")
    mip = O.render(tiny, cam, "mip", interp="nearest", step=step, lut=scene.linear_lut(), smooth="box",
                   smooth_arm=arm)
    assert np.allclose(mip["scalar"], ma.max(axis=0)[::-1, :], rtol=0, atol=1e-12)
    avg = O.render(tiny, cam, "avg", interp="nearest", step=step, lut=scene.linear_lut(), smooth="box",
                   smooth_arm=arm)
    assert np.allclose(avg["scalar"], ma.mean(axis=0)[::-1, :], rtol=0, atol=1e-12)
    raw = O.render(tiny, cam, "mip", interp="nearest", step=step, lut=scene.linear_lut())
    assert not np.allclose(raw["scalar"], mip["scalar"])


@pytest.mark.parametrize("ortho", [False, True])
def test_box_oblique_linear_cube(O, ortho):
    """Trilinear interpolation with edge clamping reproduces a linear field f at the
    coordinate-wise clamped point, so the box value at p is the mean of f(clamp(p + i d)),
    d the ray's unit direction (from its sample positions)."""
    nx, ny, nz = 20, 24, 28
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    coef = np.array([0.37, -0.21, 0.13])
    cube = (coef[0] * x + coef[1] * y + coef[2] * z + 0.5).astype(np.float32)
    cam = scene.orbit_camera((nx, ny, nz), 37, -24, 24, 20, ortho=ortho)
    arm, h = 3, 0.5
    hi = np.array([nx - 1, ny - 1, nz - 1], np.float64)
    f = lambda p: np.clip(p, 0.0, hi) @ coef + 0.5  # noqa: E731
    pix = np.arange(cam.width * cam.height)
    res = O.render(cube, cam, "avg", interp="trilinear", step=h, lut=scene.linear_lut(), smooth="box",
                   smooth_arm=arm, pixels=pix)
    checked = 0
    for q in pix[::7]:
        px, py = int(q % cam.width), int(q // cam.width)
        pos, _ = O.ray_trace(cube, cam, px, py, interp="trilinear", step=h)
        if len(pos) < 2:
            continue
        d = (pos[-1] - pos[0]) / ((len(pos) - 1) * h)
        vals = [np.mean([f(p + i * d) for i in range(-arm, arm + 1)]) for p in pos]
        assert res["scalar"][q] == pytest.approx(np.mean(vals), abs=1e-6)  # float32 cube rounding
        checked += 1
    assert checked > 20


def _axis_profile_cube(axis, n=(24, 26, 28)):
    nx, ny, nz = n
    g = np.random.default_rng(11).normal(size=n[axis])
    shape = (nz, ny, nx)
    bshape = [1, 1, 1]
    bshape[2 - axis] = n[axis]
    cube = np.broadcast_to(g.reshape(bshape), shape).astype(np.float32)
    return cube, g.astype(np.float32).astype(np.float64)


def _conv_edge(g, b):
    r = (len(b) - 1) // 2
    return np.convolve(np.pad(g, r, mode="edge"), b[::-1], mode="valid")


@pytest.mark.parametrize("interp", ["nearest", "trilinear"])
def test_taps_chain_on_axis_profiles(O, interp):
    """A cube that varies along one axis only, sampled at integer positions on that axis.
    Linear sampling at +-1.3846, +-3.2308 equals the discrete 9-tap kernel there (trilinear);
    the chain x, y, z then weights the kernel's result by c0^2 (x), c0 (y) or 1 (z) and the
    raw value by the rest.  Nearest sampling instead fetches the rounded voxels +-1, +-3."""
    c0, off, w = _alg9()
    taps = (c0, off, w)
    b = _b12_central9()
    if interp == "nearest":
        b = np.zeros(9)
        b[4] = c0
        for o, wj in zip(off, w):
            k = int(math.floor(o + 0.5))
            b[4 + k] += wj
            b[4 - k] += wj
    for axis in range(3):
        cube, g = _axis_profile_cube(axis)
        nz, ny, nx = cube.shape
        conv = _conv_edge(g, b)
        if axis == 0:
            cam = scene.ortho_axis_camera((nx, ny, nz), nx, ny, axis="z")
            exp = c0 * c0 * conv + (1 - c0 * c0) * g
            img = np.broadcast_to(exp[None, :], (ny, nx))
        elif axis == 1:
            cam = scene.ortho_axis_camera((nx, ny, nz), nx, ny, axis="z")
            exp = c0 * conv + (1 - c0) * g
            img = np.broadcast_to(exp[::-1, None], (ny, nx))
        else:
            cam = scene.ortho_axis_camera((nx, ny, nz), nz, ny, axis="x")
            img = np.broadcast_to(conv[None, :], (ny, nz))
        r = O.render(cube, cam, "avg", interp=interp, lut=scene.linear_lut(), smooth="taps", smooth_taps=taps)
        assert np.allclose(r["scalar"], img, rtol=0, atol=2e-9), axis


def test_taps_x_first_differs_from_z_first(O):
    """The chain's order matters for a cube varying along x: the x pass's result is damped
    by the y and z passes (c0^2) -- not the plain kernel that an x-last order would give."""
    c0, off, w = _alg9()
    cube, g = _axis_profile_cube(0)
    nz, ny, nx = cube.shape
    cam = scene.ortho_axis_camera((nx, ny, nz), nx, ny, axis="z")
    r = O.render(cube, cam, "avg", interp="trilinear", lut=scene.linear_lut(), smooth="taps",
                 smooth_taps=(c0, off, w))
    plain = _conv_edge(g, _b12_central9())
    assert not np.allclose(r["scalar"][0], plain, atol=1e-3)


def test_fetches_per_step(O, tiny):
    """Section 6's fetch counts per ray step: N for an N-box, 3 (N - 1)/2 + 1 for the
    N-tap 3-D kernel (binomial b_{N-1}, linear-sampling merged), 1 raw."""
    gold = json.load(open(os.path.join(GOLD, "fetch_counts.json")))
    cam = scene.orbit_camera(tiny.shape[::-1], 30, 20, 24, 20)
    kw = dict(interp="trilinear", lut=scene.linear_lut())
    base, n0 = O.count_fetches(lambda: O.render(tiny, cam, "avg", **kw))
    steps = int(base["nsamples"].sum())
    assert steps > 1000 and n0 == gold["raw_fetches"] * steps
    for arm in (1, 2, 4):
        _, n = O.count_fetches(lambda: O.render(tiny, cam, "avg", smooth="box", smooth_arm=arm, **kw))
        assert n == (2 * arm + 1) * steps
    for N, fetches in zip(gold["gaussian_taps"], gold["gaussian_fetches"]):
        off, wt = O.linear_sampling_merge(O.binomial_weights(N - 1))
        taps = (wt[0], off[1:], wt[1:])
        _, n = O.count_fetches(lambda: O.render(tiny, cam, "avg", smooth="taps", smooth_taps=taps, **kw))
        assert n == fetches * steps, N


def test_smoothing_precedes_the_filter(O, tiny):
    """Algorithm 1 smooths the fetched value, then filters it: clipping the box-smoothed
    moving average on the spectral-axis view."""
    from scipy.ndimage import uniform_filter1d
    nz, ny, nx = tiny.shape
    cam = scene.ortho_axis_camera((nx, ny, nz), nx, ny)
    ma = uniform_filter1d(tiny.astype(np.float64), size=5, axis=0, mode="nearest")
    tmin, tmax = 0.3, 2.0
    clipped = np.where((ma < tmin) | (ma > tmax), LO, ma)
    r = O.render(tiny, cam, "mip", interp="nearest", step=1.0, lut=scene.linear_lut(), smooth="box",
                 smooth_arm=2, filter="clip", min_threshold=tmin, max_threshold=tmax)
    assert np.allclose(r["scalar"], clipped.max(axis=0)[::-1, :], rtol=0, atol=1e-12)


def test_ratio_smooths_each_cube(O, tiny):
    """The line ratio smooths both cubes' samples before the quotient."""
    from scipy.ndimage import uniform_filter1d
    nz, ny, nx = tiny.shape
    cam = scene.ortho_axis_camera((nx, ny, nz), nx, ny)
    c2 = scene.ratio_cube(tiny, config_id=1)
    m1 = uniform_filter1d(tiny.astype(np.float64), size=3, axis=0, mode="nearest")
    m2 = uniform_filter1d(c2.astype(np.float64), size=3, axis=0, mode="nearest")
    with np.errstate(divide="ignore", invalid="ignore"):
        v = np.where(m1 > 0.5, m2 / m1, 0.0)
    r = O.render(tiny, cam, "ratio", interp="nearest", step=1.0, lut=scene.ratio_lut(), cube2=c2, lo=0.0,
                 hi=1.0, ratio_floor=0.5, smooth="box", smooth_arm=1)
    assert np.allclose(r["scalar"], v.max(axis=0)[::-1, :], rtol=0, atol=1e-12)
