"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: numpy
reductions that restate a closed form (moment maps, Eqs. 1 and 3), brute force on
tiny cubes, invariants (affine fields, constants, homogeneity), the paper's own
printed constants (Algorithm 9) and library routines (float16 / bfloat16
rounding).  A plausible mistake in the oracle -- a dropped term, a wrong sign or
index, a transposed operand -- breaks at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import scene

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def O(oracle_lib):
    return oracle_lib


@pytest.fixture(scope="module")
def tiny():
    return scene.tiny_cube()


def _img_from_map(m, ny):
    """Map [ny][nx] -> 2x upsampled image, row 0 = y = ny-1 (the ortho-z camera's layout)."""
    return m[::-1, :].repeat(2, 0).repeat(2, 1)


# --------------------------------------------------------------------------- projections

def test_mip_ortho_nearest_is_spectral_max(O, tiny):
    """Eq. 1 + Section 2.2: an orthographic ray down the spectral axis is a moment-map line."""
    cam = scene.ortho_axis_camera((64, 64, 64), 128, 128)
    r = O.render(tiny, cam, "mip", interp="nearest", lut=scene.linear_lut())
    assert np.array_equal(r["scalar"], _img_from_map(tiny.max(axis=0).astype(np.float64), 64))
    assert (r["nsamples"] == 128).all()


def test_spectral_index_is_last_argmax(O, tiny):
    """Algorithm 4 with '>=': the channel of the LAST maximum along the ray."""
    cube = np.round(tiny * 2).astype(np.float32)  # many exact ties
    cam = scene.ortho_axis_camera((64, 64, 64), 128, 128)
    r = O.render(cube, cam, "spectral", interp="nearest", lut=scene.linear_lut())
    last = 63 - np.argmax(cube[::-1], axis=0)
    assert np.array_equal(r["index"], _img_from_map(last, 64))
    first = np.argmax(cube, axis=0)
    assert (last != first).any()  # the case actually distinguishes first from last


def test_spectral_colour_from_channel(O, tiny):
    """MIP_1: rgb = colourMap(t_z), t_z = (channel + 1/2)/nz; alpha = v_hat(max)."""
    cam = scene.ortho_axis_camera((64, 64, 64), 128, 128)
    lut = scene.linear_lut().astype(np.float64)
    r = O.render(tiny, cam, "spectral", interp="nearest", lut=lut)
    tz = (r["index"] + 0.5) / 64
    u = 255 * tz
    i0 = np.minimum(np.floor(u).astype(int), 254)
    f = u - i0
    rgb = (1 - f)[..., None] * lut[i0, :3] + f[..., None] * lut[i0 + 1, :3]
    assert np.allclose(r["rgba"][..., :3], rgb, rtol=0, atol=1e-12)
    vhat = np.clip((r["scalar"] + 3) / 11, 0, 1)
    assert np.allclose(r["rgba"][..., 3], vhat, rtol=0, atol=1e-15)


def test_avg_ortho_nearest_is_mean(O, tiny):
    """Eq. 3: the zeroth moment / N; with h = 1/2 every voxel is sampled exactly twice."""
    cam = scene.ortho_axis_camera((64, 64, 64), 128, 128)
    r = O.render(tiny, cam, "avg", interp="nearest", lut=scene.linear_lut())
    ref = _img_from_map(tiny.astype(np.float64).mean(axis=0), 64)
    assert np.allclose(r["scalar"], ref, rtol=0, atol=1e-13)


def _bilinear(m, x, y):
    ny, nx = m.shape
    x0 = np.floor(x).astype(int); y0 = np.floor(y).astype(int)
    fx = x - x0; fy = y - y0
    cx = lambda i: np.clip(i, 0, nx - 1)
    cy = lambda j: np.clip(j, 0, ny - 1)
    a = m[cy(y0), cx(x0)] * (1 - fx) + m[cy(y0), cx(x0 + 1)] * fx
    b = m[cy(y0 + 1), cx(x0)] * (1 - fx) + m[cy(y0 + 1), cx(x0 + 1)] * fx
    return a * (1 - fy) + b * fy


def test_avg_ortho_trilinear_is_interpolated_mean(O, tiny):
    """Trilinear along z with mid-point samples weights every channel by exactly 2,
    so the average equals the bilinear interpolation of the z-mean map."""
    cam = scene.ortho_axis_camera((64, 64, 64), 128, 128)
    r = O.render(tiny, cam, "avg", interp="trilinear", lut=scene.linear_lut())
    px = np.arange(128)
    X = px / 2 - 0.25
    Y = 63.25 - px / 2
    ref = _bilinear(tiny.astype(np.float64).mean(axis=0), X[None, :], Y[:, None])
    assert np.allclose(r["scalar"], ref, rtol=0, atol=1e-12)


def test_ratio_method2(O, tiny):
    """Algorithm 14: per-sample cube2/cube1 where cube1 > floor, else DATAMIN; then MIP_0."""
    c2 = scene.ratio_cube(tiny, noise=False)
    cam = scene.ortho_axis_camera((64, 64, 64), 128, 128)
    r = O.render(tiny, cam, "ratio", interp="nearest", lut=scene.linear_lut(), cube2=c2,
                 ratio_floor=1.0, lo=0.0, hi=1.0)
    c1d, c2d = tiny.astype(np.float64), c2.astype(np.float64)
    per = np.where(c1d > 1.0, c2d / np.where(c1d > 1.0, c1d, 1.0), 0.0)
    assert np.array_equal(r["scalar"], _img_from_map(per.max(axis=0), 64))
    anyhit = (c1d > 1.0).any(axis=0)
    assert np.allclose(_img_from_map(np.where(anyhit, 0.3, 0.0), 64), r["scalar"], atol=1e-7)


def test_nan_sample_is_datamin(O, tiny):
    cube = tiny.copy()
    cube[:, 10, 10] = np.nan
    cube[5:9, 20, 20] = np.nan
    cam = scene.ortho_axis_camera((64, 64, 64), 128, 128)
    r = O.render(cube, cam, "mip", interp="nearest", lut=scene.linear_lut(), lo=-3.0)
    ref = np.where(np.isnan(cube), -3.0, cube).max(axis=0)
    assert np.array_equal(r["scalar"], _img_from_map(ref, 64))
    a = O.render(cube, cam, "avg", interp="nearest", lut=scene.linear_lut(), lo=-3.0)
    assert np.isfinite(a["scalar"]).all()


# --------------------------------------------------------------------------- compositing

def test_composite_constant_cube_closed_form(O):
    """Algorithm 3 on a constant cube of opacity a: alpha = 1 - (1 - a)^n, C = rgb * alpha."""
    lut = scene.linear_lut()
    v = -3.0 + 11.0 * 100 / 255  # v_hat exactly on knot 100
    cube = np.full((16, 12, 10), v, np.float32)  # nz=16, ny=12, nx=10
    cam = scene.ortho_axis_camera((10, 12, 16), 20, 24)
    s = 0.05
    r = O.render(cube, cam, "composite", interp="trilinear", lut=lut, opacity_scale=s)
    vhat = (np.float64(np.float32(v)) + 3.0) / 11.0
    u = 255 * vhat
    i0 = int(np.floor(u)); f = u - i0
    col = (1 - f) * lut[i0].astype(np.float64) + f * lut[i0 + 1].astype(np.float64)
    a = s * col[3]
    n = 32
    A = 1 - (1 - a) ** n
    assert np.allclose(r["rgba"][..., 3], A, rtol=0, atol=1e-14)
    assert np.allclose(r["rgba"][..., :3], col[:3] * A, rtol=0, atol=1e-14)
    assert (r["nsamples"] == n).all()


def test_composite_early_exit(O):
    """Exit after the first sample that pushes alpha above 0.99 (Algorithm 3)."""
    lut = scene.linear_lut()
    cube = np.full((64, 4, 4), 8.0, np.float32)  # v_hat = 1 -> A_lut = 1
    cam = scene.ortho_axis_camera((4, 4, 64), 8, 8)
    a = 0.3
    r = O.render(cube, cam, "composite", lut=lut, opacity_scale=a)
    k = next(k for k in range(1, 200) if 1 - (1 - a) ** k > 0.99)
    assert (r["nsamples"] == k).all()
    assert np.allclose(r["rgba"][..., 3], 1 - (1 - a) ** k, atol=1e-14)


def test_composite_matches_paper_recurrence(O):
    """The premultiplied form equals Algorithm 3's straight-alpha recurrence
    (alpha_2 = a (1 - alpha_1); alpha = alpha_1 + alpha_2; frag = frag alpha_1/alpha + colour alpha_2/alpha),
    written here independently, on a cube varying only along z."""
    rng = np.random.default_rng(3)
    prof = rng.uniform(-1.0, 6.0, size=40).astype(np.float32)
    cube = np.broadcast_to(prof[:, None, None], (40, 2, 2)).copy()
    lut = scene.perturbed_lut()  # a non-trivial colour map
    s = 0.07
    cam = scene.ortho_axis_camera((2, 2, 40), 4, 4)
    r = O.render(cube, cam, "composite", interp="nearest", lut=lut, opacity_scale=s, term_alpha=1.0)
    L = lut.astype(np.float64)

    def cmap(v):
        vh = min(max((float(v) + 3) / 11, 0.0), 1.0)
        u = 255 * vh; i0 = min(int(math.floor(u)), 254); f = u - i0
        return (1 - f) * L[i0] + f * L[i0 + 1]

    frag = np.zeros(3); alpha1 = 0.0
    for v in np.repeat(prof, 2):  # h = 1/2: each channel twice
        c = cmap(v)
        a = min(max(s * c[3], 0.0), 1.0)
        alpha2 = a * (1 - alpha1)
        alpha = max(alpha1 + alpha2, 1e-300)
        frag = frag * (alpha1 / alpha) + c[:3] * (alpha2 / alpha)
        alpha1 = alpha
    assert np.allclose(r["rgba"][0, 0, 3], alpha1, atol=1e-13)
    assert np.allclose(r["rgba"][0, 0, :3], frag * alpha1, atol=1e-13)


def test_lut_linear_alpha_is_identity(O):
    """The linear colour map's alpha channel is v_hat: a (MIP) render's alpha equals v_hat(max)."""
    cube = scene.tiny_cube()
    cam = scene.orbit_camera((64, 64, 64), 30, 20, 24, 16)
    r = O.render(cube, cam, "mip", lut=scene.linear_lut())
    hit = r["nsamples"] > 0
    vhat = np.clip((r["scalar"] + 3) / 11, 0, 1)
    assert np.allclose(r["rgba"][..., 3][hit], vhat[hit], atol=2e-7)


# --------------------------------------------------------------------------- sampling & rays

def _trilinear_brute(c, p):
    nz, ny, nx = c.shape
    x, y, z = p
    i, j, k = math.floor(x), math.floor(y), math.floor(z)
    fx, fy, fz = x - i, y - j, z - k
    cl = lambda a, n: min(max(a, 0), n - 1)
    V = lambda a, b, d: float(c[cl(d, nz), cl(b, ny), cl(a, nx)])
    lerp = lambda a, b, t: a + t * (b - a)
    c00 = lerp(V(i, j, k), V(i + 1, j, k), fx)
    c10 = lerp(V(i, j + 1, k), V(i + 1, j + 1, k), fx)
    c01 = lerp(V(i, j, k + 1), V(i + 1, j, k + 1), fx)
    c11 = lerp(V(i, j + 1, k + 1), V(i + 1, j + 1, k + 1), fx)
    return lerp(lerp(c00, c10, fy), lerp(c01, c11, fy), fz)


def test_trilinear_brute_force_4cube(O):
    rng = np.random.default_rng(7)
    c = rng.standard_normal((4, 4, 4)).astype(np.float32)
    pts = rng.uniform(-0.5, 3.5, size=(500, 3))
    got = O.sample_points(c, pts)
    ref = np.array([_trilinear_brute(c, p) for p in pts])
    assert np.allclose(got, ref, rtol=0, atol=1e-13)
    near = O.sample_points(c, pts, interp="nearest")
    ix = np.clip(np.floor(pts + 0.5).astype(int), 0, 3)
    assert np.array_equal(near, c[ix[:, 2], ix[:, 1], ix[:, 0]].astype(np.float64))


def test_trilinear_reproduces_affine_and_constant(O):
    z, y, x = np.meshgrid(np.arange(6), np.arange(5), np.arange(7), indexing="ij")
    f = (0.5 + 0.25 * x - 0.125 * y + 0.375 * z).astype(np.float32)
    rng = np.random.default_rng(1)
    pts = rng.uniform([0, 0, 0], [6, 4, 5], size=(300, 3))
    got = O.sample_points(f, pts)
    assert np.allclose(got, 0.5 + 0.25 * pts[:, 0] - 0.125 * pts[:, 1] + 0.375 * pts[:, 2], atol=1e-13)
    const = np.full((5, 5, 5), 2.5, np.float32)
    assert np.allclose(O.sample_points(const, rng.uniform(-0.5, 4.5, (100, 3))), 2.5, atol=1e-15)


def _box_hit_brute(o, d, n, tmax=10000.0, steps=400000):
    t = np.linspace(0.0, tmax, steps)
    p = o[None, :] + t[:, None] * d[None, :]
    inside = np.all((p >= -0.5) & (p <= np.array(n) - 0.5), axis=1)
    if not inside.any():
        return None
    return t[inside][0], t[inside][-1]


def test_perspective_rays_geometry(O):
    """Appendix A perspective: every sample is on the line from the eye, spaced by h, and
    the clipped chord agrees with a brute-force scan of box membership."""
    dims = (40, 30, 50)
    cube = scene.tiny_cube(dims=dims, n_sources=1)
    cam = scene.orbit_camera(dims, 37, -23, 33, 21)
    eye = cam.eye.astype(np.float64)
    for px, py in [(16, 10), (0, 0), (32, 20), (5, 17)]:
        pos, _ = O.ray_trace(cube, cam, px, py)
        if len(pos) < 2:
            continue
        steps = np.diff(pos, axis=0)
        assert np.allclose(np.linalg.norm(steps, axis=1), 0.5, atol=1e-12)
        d = steps[0] / np.linalg.norm(steps[0])
        v = pos[0] - eye
        assert np.linalg.norm(v / np.linalg.norm(v) - d) < 1e-12
        t_first = np.dot(pos[0] - eye, d) - 0.25
        hit = _box_hit_brute(eye, d, dims, tmax=400.0)
        assert hit is not None
        assert abs(hit[0] - t_first) < 2e-3
        N = len(pos)
        assert math.floor((hit[1] - hit[0]) / 0.5 + 1e-9) in (N, N - 1, N + 1)
    # the centre pixel of an odd-sized image looks straight along fwd
    cam2 = scene.orbit_camera(dims, 37, -23, 33, 21)
    pos, _ = O.ray_trace(cube, cam2, 16, 10)
    d = (pos[1] - pos[0]) / 0.5
    f = cam2.fwd.astype(np.float64)
    assert np.linalg.norm(d - f / np.linalg.norm(f)) < 1e-7


def _line_distance(p, a, d):
    """Distance of point p from the line through a with unit direction d."""
    v = p - a
    return float(np.linalg.norm(v - np.dot(v, d) * d))


def test_perspective_projection_pin(O):
    """Appendix A perspective, pinned by the forward pinhole projection (not the oracle's own
    pixel -> ray formula): a point Q is taken to camera coordinates (x, y, z) = ((Q - eye).right,
    (Q - eye).up, (Q - eye).fwd) and divided by depth; it lands in pixel
    u = W/2 (1 + x / (z tan(fov/2) W/H)), v = H/2 (1 - y / (z tan(fov/2))) (row 0 at the top).
    The oracle's ray of that pixel must pass closer to Q than the rays of its 8 neighbours,
    within one pixel's footprint at Q's depth.  A wrong aspect axis, a flipped row direction or
    a wrong field-of-view scale each moves the nearest ray to another pixel."""
    dims = (40, 30, 50)
    cube = scene.tiny_cube(dims=dims, n_sources=1)
    W, H = 64, 36  # not square: the aspect ratio matters
    cam = scene.orbit_camera(dims, 37, -23, W, H)
    eye = cam.eye.astype(np.float64)
    R, U, F = (np.asarray(v, np.float64) for v in (cam.right, cam.up, cam.fwd))
    th = float(cam.tan_half_fovy)
    rng = np.random.default_rng(17)
    checked = 0

    def ray(px, py):
        pos, _ = O.ray_trace(cube, cam, px, py)
        if len(pos) < 2:
            return None
        return pos[0], (pos[1] - pos[0]) / np.linalg.norm(pos[1] - pos[0])

    for _ in range(60):
        Q = np.array([rng.uniform(3, n - 4) for n in dims])
        q = Q - eye
        x, y, z = np.dot(q, R), np.dot(q, U), np.dot(q, F)
        u = W / 2 * (1 + x / (z * th * W / H))
        v = H / 2 * (1 - y / (z * th))
        fu, fv = u - math.floor(u), v - math.floor(v)
        if min(fu, 1 - fu, fv, 1 - fv) < 0.05 or not (1 <= u < W - 1 and 1 <= v < H - 1):
            continue  # near a pixel border, or at the image edge
        px, py = int(math.floor(u)), int(math.floor(v))
        centre = ray(px, py)
        assert centre is not None
        d0 = _line_distance(Q, *centre)
        assert d0 <= 2 * z * th / H, (Q, d0)  # within one pixel's footprint at depth z
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                if dx == dy == 0:
                    continue
                nb = ray(px + dx, py + dy)
                if nb is not None:
                    assert _line_distance(Q, *nb) > d0, (Q, px, py, dx, dy)
        checked += 1
    assert checked >= 30
    # the row direction: a point above the cube centre lands in a smaller row than one below
    c = np.array([(n - 1) / 2 for n in dims])
    rows = []
    for k in (-6.0, 6.0):
        q = c + k * U - eye
        rows.append(H / 2 * (1 - np.dot(q, U) / (np.dot(q, F) * th)))
    assert rows[1] < rows[0]


def test_ortho_sample_count_is_depth(O):
    cam = scene.ortho_axis_camera((64, 64, 64), 128, 128)
    tot, per = O.count_samples((64, 64, 64), cam)
    assert tot == 128 * 128 * 128 and (per == 128).all()
    cam = scene.ortho_axis_camera((20, 30, 40), 40, 60, axis="z")
    tot, per = O.count_samples((20, 30, 40), cam, step=0.25)
    assert (per == 160).all()


# --------------------------------------------------------------------------- smoothing

def test_gauss_weights_closed_form_and_fwhm(O):
    """Eq. 5 sampled on integer taps; Eq. 6: at half the FWHM the weight is half the peak."""
    for sigma, r in [(1.0, 3), (2.0, 6), (0.7, 2)]:
        w = O.gauss_weights(sigma, r)
        k = np.arange(-r, r + 1)
        assert abs(w.sum() - 1) < 1e-15 and np.allclose(w, w[::-1], atol=0)
        assert np.allclose(w / w[r], np.exp(-k ** 2 / (2 * sigma ** 2)), rtol=1e-14)
    sigma = 3.0 / math.sqrt(2 * math.log(2))  # FWHM/2 = 3 taps
    w = O.gauss_weights(sigma, 9)
    assert abs(w[9 + 3] / w[9] - 0.5) < 1e-14
    assert abs(2 * 3.0 - 2 * math.sqrt(2 * math.log(2)) * sigma) < 1e-12


def test_binomial_is_repeated_autoconvolution(O):
    """b_n = [1,1]^{*n}: compare with numpy's convolution chain."""
    for n in (4, 8, 12):
        ref = np.array([1.0])
        for _ in range(n):
            ref = np.convolve(ref, [1.0, 1.0])
        assert np.array_equal(O.binomial_weights(n) * 2.0 ** n, ref)


def test_ninetap_constants_from_paper(O):
    """Algorithm 9's printed offsets and coefficients: the 9 central taps of b_12,
    renormalised, merged pairwise for linear sampling."""
    g = json.load(open(os.path.join(GOLD, "alg9_ninetap.json")))
    b12 = O.binomial_weights(12)
    w9 = b12[2:11] / b12[2:11].sum()
    off, wt = O.linear_sampling_merge(w9)
    tol = 0.6 * 10.0 ** -g["printed_decimals"]
    assert abs(wt[0] - g["coeff_0"]) < tol
    assert abs(wt[1] - g["coeff_1"]) < tol and abs(wt[2] - g["coeff_2"]) < tol
    assert abs(off[1] - g["offset_1"]) < tol and abs(off[2] - g["offset_2"]) < tol
    # the printed coefficients cover both sides: c0 + 2 (c1 + c2) = 1
    assert abs(g["coeff_0"] + 2 * (g["coeff_1"] + g["coeff_2"]) - 1) < 1e-9


def test_linear_sampling_reproduces_discrete_kernel(O):
    """Fetching at the merged fractional offsets with linear interpolation equals the discrete taps."""
    rng = np.random.default_rng(5)
    sig = rng.standard_normal(200)
    for w in (O.binomial_weights(4), O.binomial_weights(12)[2:11] / O.binomial_weights(12)[2:11].sum(),
              O.binomial_weights(12)):
        r = (len(w) - 1) // 2
        off, wt = O.linear_sampling_merge(w)
        i = np.arange(20, 180)
        ref = sum(w[k + r] * sig[i + k] for k in range(-r, r + 1))
        lin = lambda x: np.interp(x, np.arange(200), sig)
        got = wt[0] * sig[i] + sum(wt[m] * (lin(i + off[m]) + lin(i - off[m])) for m in range(1, len(off)))
        assert np.allclose(got, ref, atol=1e-13)


def test_fetch_count_formula(O):
    """Section 6: an N-tap 3-D Gaussian needs 3(N-1)/2 + 1 fetches per step, i.e. the merged
    one-sided fetch count x 2 sides x 3 axes + the centre."""
    g = json.load(open(os.path.join(GOLD, "fetch_counts.json")))
    b12 = O.binomial_weights(12)
    kernels = {5: O.binomial_weights(4), 9: b12[2:11] / b12[2:11].sum(), 13: b12}
    for n, fetches in zip(g["gaussian_taps"], g["gaussian_fetches"]):
        off, _ = O.linear_sampling_merge(kernels[n])
        assert 3 * 2 * (len(off) - 1) + 1 == fetches


def test_smooth_delta_is_kernel(O):
    n = 15
    c = np.zeros((n, n, n), np.float32)
    c[7, 7, 7] = 1.0
    w = O.gauss_weights(1.0, 3)
    out = O.smooth(c, w)
    ref = np.zeros((n, n, n))
    ref[4:11, 4:11, 4:11] = w[:, None, None] * w[None, :, None] * w[None, None, :]
    assert np.allclose(out, ref, atol=1e-17) and abs(out.sum() - 1) < 1e-14


def test_smooth_constant_and_affine(O):
    w = O.gauss_weights(2.0, 6)
    c = np.full((9, 10, 11), 3.25, np.float32)
    assert np.allclose(O.smooth(c, w), 3.25, atol=1e-14)
    z, y, x = np.meshgrid(np.arange(30), np.arange(30), np.arange(30), indexing="ij")
    f = (1.0 + 0.5 * x - 0.25 * y + 0.125 * z).astype(np.float32)
    out = O.smooth(f, w)
    sl = slice(6, 24)
    assert np.allclose(out[sl, sl, sl], f[sl, sl, sl], atol=1e-12)


def test_smooth_separable_equals_direct_triple_sum(O):
    rng = np.random.default_rng(11)
    c = rng.standard_normal((16, 17, 18)).astype(np.float32)
    w = O.gauss_weights(1.3, 4)
    out = O.smooth(c, w)
    ids = np.arange(c.size)
    direct = O.smooth_points(c, w, ids).reshape(c.shape)
    assert np.allclose(out, direct, atol=1e-13)
    # clamp-to-edge: brute force on a corner voxel in plain numpy
    cp = np.pad(c.astype(np.float64), 4, mode="edge")
    K = w[:, None, None] * w[None, :, None] * w[None, None, :]
    assert abs((cp[0:9, 0:9, 0:9] * K).sum() - out[0, 0, 0]) < 1e-13


# --------------------------------------------------------------------------- reduced precision

def test_round_bf16_matches_torch(O):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.standard_normal(20000).astype(np.float32) * 10,
                        np.array([0.0, -0.0, 1.0, 65504, 1e-40, 3.4e38, np.inf, -np.inf], np.float32),
                        (1 + np.arange(256) / 128.0).astype(np.float32)])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(O.round_bf16(x).view(np.uint32), ref.view(np.uint32))


def test_round_f16_matches_numpy(O):
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.standard_normal(20000).astype(np.float32) * 100,
                        rng.standard_normal(2000).astype(np.float32) * 1e-5,
                        np.array([0.0, -0.0, 65504, 65519.9, 65520, 7e4, 6e-8, 3e-8, np.inf], np.float32)])
    with np.errstate(over="ignore"):
        ref = x.astype(np.float16).astype(np.float32)
    assert np.array_equal(O.round_f16(x).view(np.uint32), ref.view(np.uint32))
