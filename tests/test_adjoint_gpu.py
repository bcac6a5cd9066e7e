"""GPU adjoint of the compositing render (shw_render_backward) against the oracle's reverse mode.

Both sides get the same upstream gradient g = dL/dRGBA (computed from the oracle's FP64
forward and a target image, L = 1/2 ||rgba - target||^2) and return J^T g for the voxels,
the colour map and the opacity scale.  The oracle's gradient is itself pinned to FP64
central differences and the homogeneity invariant (CPU tests).

Tolerance: max |g_gpu - g_oracle| <= 1e-4 x max |g_oracle| per gradient array (FP32
transmittance and atomics summing up to ~1e8 terms: ~K eps with K <= 1e3 samples and
eps = 6e-8 gives <= 6e-5); 1e-3 at the full 256^3 size, where per-entry colour-map sums
run over ~1e8 FP32 atomic additions.
"""
import numpy as np
import pytest
import torch

import oracle
import scene
from parity import shw, to_dev
from scene import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    return shw()


def _case(dims, width, height, s, interp="trilinear", ckpt_interval=64, yaw=30, pitch=20, n_sources=3):
    cube = scene.diff_cube(dims=dims, n_sources=n_sources)
    cam = scene.orbit_camera(dims, yaw, pitch, width, height)
    lut = scene.linear_lut()
    target = oracle.render(cube, cam, "composite", interp=interp, lut=scene.perturbed_lut(),
                           opacity_scale=s * 1.2)["rgba"]
    o = oracle.render(cube, cam, "composite", interp=interp, lut=lut, opacity_scale=s)
    g = (o["rgba"] - target).astype(np.float32).astype(np.float64)  # the GPU receives it in float32
    return cube, cam, lut, g


def _gpu_grad(m, cube, cam, lut, g, s, interp="trilinear", ckpt_interval=64, term_alpha=0.99):
    ct, lt = to_dev(cube), to_dev(lut)
    out = m.render(ct, cam, "composite", lut=lt, opacity_scale=s, interp=interp, ckpt=True,
                   ckpt_interval=ckpt_interval, term_alpha=term_alpha)
    gv = torch.zeros_like(ct)
    gl = torch.zeros_like(lt)
    gs = torch.zeros(1, device="cuda")
    m.render_backward(ct, cam, to_dev(g.astype(np.float32)), out["ckpt"], lut=lt, opacity_scale=s, interp=interp,
                      ckpt_interval=ckpt_interval, term_alpha=term_alpha, grad_vol=gv, grad_lut=gl, grad_scale=gs)
    m.sync_status()
    return out, gv.cpu().numpy(), gl.cpu().numpy(), float(gs.item())


def _check(gpu, ref, rtol, what):
    gv, gl, gs = gpu
    _, rv, rl, rs = ref
    ev = np.abs(gv - rv).max() / np.abs(rv).max()
    el = np.abs(gl - rl).max() / np.abs(rl).max()
    es = abs(gs - rs) / abs(rs)
    assert ev <= rtol and el <= rtol and es <= rtol, (what, ev, el, es)
    return ev, el, es


@pytest.mark.parametrize("interp", ["trilinear", "nearest"])
@pytest.mark.parametrize("ckpt_interval", [1, 7, 64])
def test_adjoint_matches_oracle_small(m, interp, ckpt_interval):
    s = 0.02
    cube, cam, lut, g = _case((32, 32, 32), 64, 64, s, interp=interp)
    out, gv, gl, gs = _gpu_grad(m, cube, cam, lut, g, s, interp=interp, ckpt_interval=ckpt_interval)
    ref = oracle.render_grad(cube, cam, g, interp=interp, lut=lut, opacity_scale=s)
    _check((gv, gl, gs), ref, 1e-4, f"{interp}/I={ckpt_interval}")


def test_adjoint_with_early_exit(m):
    """Large opacity: most rays terminate early; the exit sample is held fixed on both sides."""
    s = 0.6
    cube, cam, lut, g = _case((40, 36, 44), 72, 60, s, yaw=-40, pitch=15)
    out, gv, gl, gs = _gpu_grad(m, cube, cam, lut, g, s)
    o = oracle.render(cube, cam, "composite", lut=lut, opacity_scale=s, eps_pos=1e-6, eps_val=1e-4)
    ns = out["nsamples"].cpu().numpy()
    assert (ns < o["nsamples"].max()).mean() > 0.3 or (o["rgba"][..., 3] > 0.99).mean() > 0.2
    # rays whose exit decision is fragile would differ in K: zero their upstream gradient on both sides
    frag = o["fragile"] != 0
    g = g.copy()
    g[frag] = 0
    out, gv, gl, gs = _gpu_grad(m, cube, cam, lut, g, s)
    ref = oracle.render_grad(cube, cam, g, lut=lut, opacity_scale=s)
    _check((gv, gl, gs), ref, 1e-4, "early exit")


def test_adjoint_full_size(m):
    """The differentiation workload: 256^3 cube, 512 x 512 perspective, checkpoints every 64."""
    w = W.DIFF
    cube, cam, lut, g = _case(w["dims"], w["width"], w["height"], w["opacity_scale"], n_sources=10)
    out, gv, gl, gs = _gpu_grad(m, cube, cam, lut, g, w["opacity_scale"], ckpt_interval=w["ckpt_interval"])
    ref = oracle.render_grad(cube, cam, g, lut=lut, opacity_scale=w["opacity_scale"])
    _check((gv, gl, gs), ref, 1e-3, "256^3")


def test_autograd_function(m):
    """Through torch.autograd: a loss linear in the image, L = sum(G * rgba), so dL/dRGBA = G is a
    fixed input that the oracle receives as well."""
    s = 0.02
    cube, cam, lut, g = _case((32, 32, 32), 64, 64, s)
    G = to_dev(g.astype(np.float32))
    ct = to_dev(cube).requires_grad_(True)
    lt = to_dev(lut).requires_grad_(True)
    st = torch.tensor(s, device="cuda", requires_grad=True)
    rgba = m.composite_render(ct, lt, st, cam)
    (rgba * G).sum().backward()
    ref = oracle.render_grad(cube, cam, g.astype(np.float32).astype(np.float64), lut=lut, opacity_scale=s)
    _check((ct.grad.cpu().numpy(), lt.grad.cpu().numpy(), float(st.grad.item())), ref, 1e-4, "autograd")
