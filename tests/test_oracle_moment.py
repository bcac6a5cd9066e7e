"""Pins of the oracle's first-moment mode (Eq. 4 along each ray).

Reading taken: the weight of a sample is its intensity above DATAMIN, max(v - lo, 0)
(a NaN sample, already DATAMIN, weighs nothing), its position the sample's z (the
channel for nearest sampling, the continuous coordinate for trilinear); the scalar is
sum(z w) / sum(w), the channel its rounding, the colour the map at (M1 + 1/2) / nz and
alpha the normalised mean intensity.  A ray with no weight is transparent, channel -1.
Each pin restates the definition independently of the oracle's code: numpy reductions
over the moment-map view, a brute-force sampler, and a one-channel cube whose moment is
that channel exactly."""
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


def _img_from_map(m):
    return m[::-1, :].repeat(2, 0).repeat(2, 1)


def test_moment1_ortho_nearest_is_moment_map(O, tiny):
    """Section 2.2: on the spectral-axis view every channel is sampled twice, so the ray's
    first moment is the moment-1 map of the cube (with weights above DATAMIN)."""
    cam = scene.ortho_axis_camera((64, 64, 64), 128, 128)
    r = O.render(tiny, cam, "moment1", interp="nearest", lut=scene.linear_lut(), lo=LO, hi=HI)
    w = np.maximum(tiny.astype(np.float64) - LO, 0.0)
    z = np.arange(64, dtype=np.float64)[:, None, None]
    m1 = (z * w).sum(axis=0) / w.sum(axis=0)
    assert np.allclose(r["scalar"], _img_from_map(m1), rtol=0, atol=1e-10)
    assert np.array_equal(r["index"], _img_from_map(np.floor(m1 + 0.5).astype(np.int32)))
    mean = tiny.astype(np.float64).mean(axis=0)
    assert np.allclose(r["rgba"][..., 3], _img_from_map(np.clip((mean - LO) / (HI - LO), 0, 1)), rtol=0, atol=1e-12)
    lut = scene.linear_lut().astype(np.float64)
    u = 255 * np.clip((r["scalar"] + 0.5) / 64, 0, 1)
    i0 = np.minimum(np.floor(u).astype(int), 254)
    f = u - i0
    rgb = (1 - f)[..., None] * lut[i0, :3] + f[..., None] * lut[i0 + 1, :3]
    assert np.allclose(r["rgba"][..., :3], rgb, rtol=0, atol=1e-12)


def _bilinear(m, x, y):
    ny, nx = m.shape
    x0 = np.floor(x).astype(int); y0 = np.floor(y).astype(int)
    fx = x - x0; fy = y - y0
    cx = lambda i: np.clip(i, 0, nx - 1)
    cy = lambda j: np.clip(j, 0, ny - 1)
    a = m[cy(y0), cx(x0)] * (1 - fx) + m[cy(y0), cx(x0 + 1)] * fx
    b = m[cy(y0 + 1), cx(x0)] * (1 - fx) + m[cy(y0 + 1), cx(x0 + 1)] * fx
    return a * (1 - fy) + b * fy


def test_moment1_ortho_trilinear_brute_force(O, tiny):
    """Brute force: samples at z = -1/4 + k/2, bilinear in (x, y) per channel plane, linear
    in z with clamp-to-edge, weights max(v - lo, 0)."""
    cam = scene.ortho_axis_camera((64, 64, 64), 128, 128)
    r = O.render(tiny, cam, "moment1", interp="trilinear", lut=scene.linear_lut(), lo=LO, hi=HI)
    px = np.arange(128)
    X, Y = px / 2 - 0.25, 63.25 - px / 2
    planes = np.stack([_bilinear(tiny[c].astype(np.float64), X[None, :], Y[:, None]) for c in range(64)])
    zs = -0.25 + 0.5 * np.arange(128)
    k0 = np.floor(zs).astype(int)
    fz = (zs - k0)[:, None, None]
    lo_p = planes[np.clip(k0, 0, 63)]
    hi_p = planes[np.clip(k0 + 1, 0, 63)]
    v = lo_p + fz * (hi_p - lo_p)
    w = np.maximum(v - LO, 0.0)
    m1 = (zs[:, None, None] * w).sum(axis=0) / w.sum(axis=0)
    assert np.allclose(r["scalar"], m1, rtol=0, atol=1e-9)


def _z_span(cam, dims):
    """Heights where each pixel's ray enters and leaves the box [-1/2, n - 1/2]^3
    (Appendix A cameras, restated in numpy); rows of NaN for misses."""
    W, H = cam.width, cam.height
    px, py = np.meshgrid(np.arange(W), np.arange(H))
    xs, ys = (2 * px + 1 - W) / W, (H - 2 * py - 1) / H
    e, r, u, f = (np.asarray(v, np.float64) for v in (cam.eye, cam.right, cam.up, cam.fwd))
    if cam.ortho:
        o = e + (xs * cam.ortho_half_h * W / H)[..., None] * r + (ys * cam.ortho_half_h)[..., None] * u
        d = np.broadcast_to(f / np.linalg.norm(f), o.shape)
    else:
        d = f + (xs * cam.tan_half_fovy * W / H)[..., None] * r + (ys * cam.tan_half_fovy)[..., None] * u
        d = d / np.linalg.norm(d, axis=-1, keepdims=True)
        o = np.broadcast_to(e, d.shape)
    n = np.array(dims, np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        ta, tb = (-0.5 - o) / d, (n - 0.5 - o) / d
    t0 = np.maximum(np.minimum(ta, tb).max(axis=-1), 0.0)
    t1 = np.maximum(ta, tb).min(axis=-1)
    za, zb = o[..., 2] + t0 * d[..., 2], o[..., 2] + t1 * d[..., 2]
    lo_z, hi_z = np.minimum(za, zb), np.maximum(za, zb)
    miss = ~(t0 < t1)
    lo_z[miss] = np.nan
    hi_z[miss] = np.nan
    return lo_z, hi_z, o[..., 2] + 0 * t0, d[..., 2] + 0 * t0, t0, t1


@pytest.mark.parametrize("interp", ["nearest", "trilinear"])
def test_moment1_single_bright_channel(O, interp):
    """Everything 1 below DATAMIN but one channel c = 17 (2 above DATAMIN).  Nearest: a
    ray across it has its moment exactly at c.  Trilinear: the value along the ray is
    lo - 1 + 3 max(1 - |z - c|, 0), so the weights are max(2 - 3 |z - c|, 0) and the
    moment is their weighted mean of the sample heights z_k = z(t0 + (k + 1/2) h),
    computed here by brute force.  A ray that never comes near c has no weight at all."""
    dims = (32, 24, 40)
    cube = np.full((40, 24, 32), LO - 1.0, np.float32)
    cube[17] = LO + 2.0
    for cam in (scene.ortho_axis_camera(dims, 32, 24), scene.orbit_camera(dims, 10.0, 5.0, 40, 30),
                scene.orbit_camera(dims, 35.0, -20.0, 40, 30, ortho=True)):
        r = O.render(cube, cam, "moment1", interp=interp, lut=scene.linear_lut(), lo=LO, hi=HI)
        za, zb, oz, dz, t0, t1 = _z_span(cam, dims)
        across = (za <= 15.5) & (zb >= 18.5)
        away = (zb <= 15.5) | (za >= 18.5)
        assert across.sum() > 20
        if interp == "nearest":
            assert np.allclose(r["scalar"][across], 17.0, rtol=0, atol=1e-9)
            assert (r["index"][across] == 17).all()
        else:
            for iy, ix in zip(*np.nonzero(across)):
                n = int(np.floor((t1[iy, ix] - t0[iy, ix]) / 0.5))
                zk = oz[iy, ix] + (t0[iy, ix] + (np.arange(n) + 0.5) * 0.5) * dz[iy, ix]
                w = np.maximum(2.0 - 3.0 * np.abs(zk - 17.0), 0.0)
                assert abs(r["scalar"][iy, ix] - (zk * w).sum() / w.sum()) < 1e-6
        assert (r["index"][away] == -1).all() and (r["rgba"][away] == 0).all()


def test_moment1_nothing_above_datamin_is_transparent(O):
    cube = np.full((16, 8, 8), LO - 1.0, np.float32)
    cube[3, 2, 2] = np.nan
    cam = scene.ortho_axis_camera((8, 8, 16), 16, 16)
    r = O.render(cube, cam, "moment1", interp="trilinear", lut=scene.linear_lut(), lo=LO, hi=HI)
    assert (r["rgba"] == 0).all() and (r["index"] == -1).all() and (r["scalar"] == 0).all()
    assert (r["nsamples"] == 32).all()
