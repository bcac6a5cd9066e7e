"""Pins of the oracle's reverse-mode gradient of the compositing render.

(1) FP64 central finite differences of the oracle's own forward render, for
voxels, colour-map entries and the opacity scale; (2) the homogeneity invariant:
the loss sees s and the colour map's alphas only through s * L[j].a, so
s dL/ds = sum_j L[j].a dL/dL[j].a.
"""
import numpy as np
import pytest

import scene

DIMS = (32, 32, 32)
W = H = 64
LO, HI = -3.0, 8.0


@pytest.fixture(scope="module")
def setup(oracle_lib):
    O = oracle_lib
    cube = scene.diff_cube(dims=DIMS, n_sources=3).astype(np.float64)
    cam = scene.orbit_camera(DIMS, 30, 20, W, H)
    lut = scene.linear_lut().astype(np.float64)
    s = 0.02
    target = O.render(cube, cam, "composite", lut=scene.perturbed_lut(), opacity_scale=s * 1.2,
                      lo=LO, hi=HI, term_alpha=0.99)["rgba"]
    return O, cube, cam, lut, s, target


def _loss(O, cube, cam, lut, s, target):
    r = O.render(cube, cam, "composite", lut=lut, opacity_scale=s, lo=LO, hi=HI, term_alpha=0.99)
    d = r["rgba"] - target
    return 0.5 * float((d * d).sum()), d


def test_grad_matches_central_differences(setup):
    O, cube, cam, lut, s, target = setup
    L0, d = _loss(O, cube, cam, lut, s, target)
    _, gv, gl, gs = O.render_grad(cube, cam, d, lut=lut, opacity_scale=s, lo=LO, hi=HI, term_alpha=0.99)
    rng = np.random.default_rng(0)
    h = 1e-6

    # voxels with a non-trivial gradient
    cand = np.flatnonzero(np.abs(gv) > 1e-6 * np.abs(gv).max())
    ids = rng.choice(cand, size=48, replace=False)
    bad = 0
    for vid in ids:
        cp = cube.copy().reshape(-1); cp[vid] += h
        cm = cube.copy().reshape(-1); cm[vid] -= h
        fd = (_loss(O, cp.reshape(cube.shape), cam, lut, s, target)[0]
              - _loss(O, cm.reshape(cube.shape), cam, lut, s, target)[0]) / (2 * h)
        g = gv.reshape(-1)[vid]
        if abs(fd - g) > 1e-5 * max(abs(g), 1e-3 * np.abs(gv).max()):
            bad += 1
    assert bad <= 1, bad  # a knot of the colour map can fall inside +-h

    # colour-map entries: the used ones and a few unused (gradient zero)
    used = np.flatnonzero(np.abs(gl).reshape(-1) > 0)
    ids = np.concatenate([rng.choice(used, size=min(40, len(used)), replace=False),
                          np.flatnonzero(np.abs(gl).reshape(-1) == 0)[:4]])
    bad = 0
    for j in ids:
        lp = lut.copy().reshape(-1); lp[j] += h
        lm = lut.copy().reshape(-1); lm[j] -= h
        fd = (_loss(O, cube, cam, lp.reshape(256, 4), s, target)[0]
              - _loss(O, cube, cam, lm.reshape(256, 4), s, target)[0]) / (2 * h)
        g = gl.reshape(-1)[j]
        if abs(fd - g) > 1e-5 * max(abs(g), 1e-3 * np.abs(gl).max()):
            bad += 1
    assert bad == 0

    fd = (_loss(O, cube, cam, lut, s + h, target)[0] - _loss(O, cube, cam, lut, s - h, target)[0]) / (2 * h)
    assert abs(fd - gs) <= 1e-6 * abs(gs)


def test_grad_homogeneity(setup):
    O, cube, cam, lut, s, target = setup
    _, d = _loss(O, cube, cam, lut, s, target)
    _, gv, gl, gs = O.render_grad(cube, cam, d, lut=lut, opacity_scale=s, lo=LO, hi=HI, term_alpha=0.99)
    lhs = s * gs
    rhs = float((lut[:, 3] * gl[:, 3]).sum())
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)
    assert abs(lhs) > 1e-6  # the identity is not trivially 0 = 0


def test_grad_forward_equals_render(setup):
    O, cube, cam, lut, s, target = setup
    r = O.render(cube, cam, "composite", lut=lut, opacity_scale=s, lo=LO, hi=HI, term_alpha=0.99)
    rgba, *_ = O.render_grad(cube, cam, np.zeros((H, W, 4)), lut=lut, opacity_scale=s, lo=LO, hi=HI,
                             term_alpha=0.99)
    assert np.array_equal(rgba, r["rgba"])
