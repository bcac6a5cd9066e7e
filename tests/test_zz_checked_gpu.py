"""The bounds-checked build (-DSHW_CHECKED) on the GPU.

That build checks, on the device, every index a kernel takes without clamping: the
samplers' interior paths (gather and staged marchers, bricks, pairs, linear 16-bit cubes),
the staged marcher's shared-memory reads, the plane sweep's offsets and planes and the
smoothing's output planes; a violating index is clamped into its array and recorded, and
shw_sync_status reports SHW_EBOUNDS.  Here the test builds that library and runs every
kernel family through it -- views of every class, both marchers, each storage, the sweep,
both smoothings, batch plans (one on its own 16^3 bricks), the adjoint -- requiring no violation and outputs
bit-identical to the normal library's (the checks change no result)."""
import numpy as np
import pytest
import torch

import scene
from parity import shw, to_dev

pytestmark = pytest.mark.gpu

VIEWS = [
    dict(dims=(68, 45, 66), yaw=30, pitch=20, W=100, H=75),               # z-major, oblique
    dict(dims=(68, 45, 66), yaw=80, pitch=10, W=90, H=61),                # x-major
    dict(dims=(68, 45, 66), yaw=15, pitch=75, W=70, H=83),                # y-major, looking down
    dict(dims=(68, 45, 66), yaw=200, pitch=-35, W=77, H=77),              # negative directions
    dict(dims=(64, 40, 96), yaw=30, pitch=20, W=160, H=90, ortho=True),   # parallel, oblique
    dict(dims=(64, 40, 96), yaw=-135, pitch=40, W=49, H=33, dist_scale=0.3),  # eye inside the cube
]


@pytest.fixture(scope="module")
def libs():
    m = shw()
    from paper_1707_00442_gb300 import _lib, build
    normal = _lib.LIB_PATH
    checked = build.build_checked()
    yield m, normal, checked
    _lib._lib = None
    _lib.LIB_PATH = normal


def _use(path):
    from paper_1707_00442_gb300 import _lib
    _lib._lib = None
    _lib.LIB_PATH = path


def _host(out):
    if isinstance(out, torch.Tensor):
        return {"out": out.cpu()}
    if isinstance(out, (list, tuple)):
        return {str(i): o.cpu() for i, o in enumerate(out)}
    return {k: v.cpu() for k, v in out.items()}


def _both(libs, fn):
    """fn() under the normal and the checked library: the checked run reports no violation
    (sync_status would raise SHW_EBOUNDS) and every output is bit-identical."""
    m, normal, checked = libs
    res = []
    for path in (normal, checked):
        _use(path)
        out = _host(fn())
        torch.cuda.synchronize()
        m.sync_status()
        res.append(out)
    _use(normal)
    a, b = res
    assert set(a) == set(b)
    for k in a:
        assert torch.equal(a[k], b[k]), k


def _cam(v):
    return scene.orbit_camera(v["dims"], v["yaw"], v["pitch"], v["W"], v["H"], ortho=v.get("ortho", False),
                              dist_scale=v.get("dist_scale", 1.0))


def _cube(i, dims):
    cube = scene.tiny_cube(config_id=110 + i, dims=dims, n_sources=3)
    cube[dims[2] // 3, dims[1] // 2, dims[0] // 4] = np.nan
    return cube


@pytest.mark.parametrize("view", range(len(VIEWS)))
def test_checked_marchers(libs, view):
    m = libs[0]
    v = VIEWS[view]
    ct = to_dev(_cube(view, v["dims"]))
    lut = to_dev(scene.linear_lut())
    cam = _cam(v)
    for mode in ("mip", "avg", "composite", "spectral", "moment1"):
        kw = dict(opacity_scale=0.05) if mode == "composite" else {}
        for flags in (("require_staging",), ("no_staging",)):
            def run(flags=flags, mode=mode, kw=kw):
                with m.debug_flags(*flags):
                    return m.render(ct, cam, mode, lut=lut, **kw)
            _both(libs, run)
    _both(libs, lambda: m.render(ct, cam, "mip", lut=lut, interp="nearest"))
    _both(libs, lambda: m.render(ct, cam, "mip", lut=lut, smooth="box", smooth_arm=1))


@pytest.mark.parametrize("view", [0, 1, 4])
def test_checked_storages_and_pairs(libs, view):
    m = libs[0]
    v = dict(VIEWS[view], dims=(72, 45, 66))
    cube = _cube(view, v["dims"])
    ct = to_dev(cube)
    c2 = to_dev(scene.ratio_cube(cube, config_id=view))
    pair = torch.stack([ct, c2], dim=-1).contiguous()
    lut, rlut = to_dev(scene.linear_lut()), to_dev(scene.ratio_lut())
    cam = _cam(v)
    kw = dict(lo=0.0, hi=1.0, ratio_floor=1.0)
    for storage in ("bf16", "f16", "bf16_linear", "f16_linear"):
        _both(libs, lambda storage=storage: m.render(m.pack_bricks(ct, storage), cam, "composite", lut=lut,
                                                     opacity_scale=0.05))
        _both(libs, lambda storage=storage: m.render(m.pack_bricks(pair, storage), cam, "ratio", lut=rlut, **kw))
    _both(libs, lambda: m.render(pair, cam, "ratio", lut=rlut, **kw))
    _both(libs, lambda: m.render(ct, cam, "ratio", lut=rlut, vol2=c2, **kw))


def test_checked_plane_sweep(libs):
    m = libs[0]
    from scene.camera import ortho_axis_camera
    dims = (64, 48, 80)
    ct = to_dev(_cube(7, dims))
    lut = to_dev(scene.linear_lut())
    for W, H in ((64, 48), (32, 24), (128, 96)):  # one voxel per pixel, zoomed out, zoomed in
        cam = ortho_axis_camera(dims, W, H)
        for mode in ("mip", "avg", "composite", "spectral", "moment1"):
            kw = dict(opacity_scale=0.05) if mode == "composite" else {}
            _both(libs, lambda mode=mode, kw=kw, cam=cam: m.render(ct, cam, mode, lut=lut, **kw))
            _both(libs, lambda mode=mode, kw=kw, cam=cam: m.render(ct, cam, mode, lut=lut, interp="nearest", **kw))


def test_checked_smoothing(libs):
    m = libs[0]
    for dims in ((72, 45, 66), (70, 33, 41)):  # the TMA pipeline, and rows it does not take
        ct = to_dev(scene.tiny_cube(config_id=120, dims=dims, n_sources=2))
        first = to_dev(scene.tiny_cube(config_id=121, dims=dims, n_sources=2))
        for r in (1, 6):
            _both(libs, lambda ct=ct, r=r: m.smooth(ct, 2.0, r))
            _both(libs, lambda ct=ct, first=first, r=r: m.smooth_zip(ct, first, 2.0, r))


def test_checked_batch_and_adjoint(libs):
    m = libs[0]
    lut = to_dev(scene.linear_lut())
    items = []
    for i, d in enumerate(((40, 36, 30), (33, 50, 27), (64, 20, 45))):
        ct = to_dev(scene.batch_subcube(i, d))
        vol = ct if i != 1 else m.pack_bricks(ct, "bf16")
        items.append((vol, scene.orbit_camera(d, 40 * i, 15, 48 + 5 * i, 40), ("mip", "composite", "avg")[i]))

    def batch():
        plan = m.BatchPlan(items, lut=lut, opacity_scale=0.05, tune=False)
        try:
            return [o.clone() for o in plan.render()]
        finally:
            plan.close()
    _both(libs, batch)

    own = [(to_dev(scene.batch_subcube(i, d)), scene.orbit_camera(d, 25 * i, -20, 44, 36), ("avg", "spectral")[i % 2])
           for i, d in enumerate(((17, 40, 33), (48, 16, 21), (1, 5, 9)))]

    def own_bricks():
        # the plan's own 16^3 bricks (the kernel without the float32 path)
        plan = m.BatchPlan(own, lut=lut, pack="bf16", brick=16, tune=False)
        try:
            return [o.clone() for o in plan.render()]
        finally:
            plan.close()
    _both(libs, own_bricks)

    dims = (40, 36, 44)
    ct = to_dev(scene.diff_cube(dims=dims, n_sources=2))
    cam = scene.orbit_camera(dims, 30, 20, 48, 40)

    def adjoint():
        # (the gradients accumulate with float atomics in no fixed order, so only the
        # forward image is compared bit for bit; the backward must record no violation)
        out = m.render(ct, cam, "composite", lut=lut, opacity_scale=0.05, ckpt=True, ckpt_interval=7)
        gv, gl, gs = torch.zeros_like(ct), torch.zeros_like(lut), torch.zeros(1, device="cuda")
        m.render_backward(ct, cam, torch.full_like(out["rgba"], 0.1), out["ckpt"], lut=lut, opacity_scale=0.05,
                          ckpt_interval=7, grad_vol=gv, grad_lut=gl, grad_scale=gs)
        assert bool(torch.isfinite(gv).all()) and float(gv.abs().sum()) > 0
        return {"rgba": out["rgba"]}
    _both(libs, adjoint)
