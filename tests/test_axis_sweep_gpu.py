"""The plane sweep for orthographic spectral-axis views must reproduce the general marcher
bit for bit (same interpolation arithmetic, same transfer-function state)."""
import math

import numpy as np
import pytest
import torch

import oracle
import scene
from parity import TOL_F32, compare, shw, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    return shw()


# Nearest sampling: the eye moves off the half-voxel grid in the image plane so that no pixel
# centre lies on a voxel-rounding tie (with the centred eye, whole images of the ragged and
# two-voxel cases would be ties, which the oracle flags and the comparison must skip).
NEAREST_SHIFT = (0.137, 0.071)


def _cam_z(dims, W, H, *, down=False, angle_deg=0.0, spacing=1.0, shift=(0.0, 0.0)):
    nx, ny, nz = dims
    c = math.cos(math.radians(angle_deg)); s = math.sin(math.radians(angle_deg))
    right = np.array([c, s, 0.0]); up = np.array([-s, c, 0.0]); fwd = np.array([0.0, 0.0, 1.0])
    eye = np.array([(nx - 1) / 2, (ny - 1) / 2, -8.0])
    if down:
        fwd = -fwd; right = -right; eye[2] = nz + 8.0
    eye = eye + shift[0] * right + shift[1] * up
    half_h = spacing * H / 2
    cam = scene.Camera(eye.astype(np.float32), right.astype(np.float32), up.astype(np.float32),
                       fwd.astype(np.float32), 0.0, float(half_h), True, W, H)
    return cam


CASES = [
    dict(dims=(64, 48, 40), W=64, H=48),                       # 1 voxel per pixel
    dict(dims=(64, 48, 40), W=128, H=96),                      # half a voxel per pixel
    dict(dims=(64, 48, 40), W=37, H=29, spacing=2.0),          # ragged image, two voxels per pixel
    dict(dims=(60, 50, 33), W=70, H=61, angle_deg=23.0),       # rotated in the image plane
    dict(dims=(60, 50, 33), W=70, H=61, down=True),            # looking down -z
    dict(dims=(60, 50, 33), W=53, H=77, down=True, angle_deg=-71.0, spacing=0.7),
    dict(dims=(64, 48, 40), W=64, H=48, step=0.25),           # four samples per cell
    dict(dims=(60, 50, 33), W=70, H=61, down=True, step=1.0),  # one sample per cell
    dict(dims=(60, 50, 33), W=53, H=40, step=0.3),             # no fixed pattern of samples per cell
]


def _both(m, monkeypatch, cube_t, cam, mode, lut_t, **kw):
    a = m.render(cube_t, cam, mode, lut=lut_t, **kw)
    torch.cuda.synchronize()
    with m.debug_flags("no_axis_sweep"):
        b = m.render(cube_t, cam, mode, lut=lut_t, **kw)
        torch.cuda.synchronize()
    m.sync_status()
    return a, b


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("mode", ["mip", "avg", "composite", "spectral", "moment1"])
@pytest.mark.parametrize("interp", ["trilinear", "nearest"])
def test_sweep_equals_general_marcher(m, monkeypatch, case, mode, interp):
    c = CASES[case]
    dims = c["dims"]
    cube = scene.tiny_cube(config_id=50 + case, dims=dims, n_sources=2)
    cube[3, 5, 7] = np.nan
    cam = _cam_z(dims, c["W"], c["H"], down=c.get("down", False), angle_deg=c.get("angle_deg", 0.0),
                 spacing=c.get("spacing", 1.0), shift=NEAREST_SHIFT if interp == "nearest" else (0.0, 0.0))
    lut = to_dev(scene.linear_lut())
    kw = dict(interp=interp, opacity_scale=0.05, step=c.get("step", 0.5))
    if mode == "composite":
        kw["ckpt"] = True
        kw["ckpt_interval"] = 7
    a, b = _both(m, monkeypatch, to_dev(cube), cam, mode, lut, **kw)
    for k in a:
        if k == "ckpt":
            continue
        assert torch.equal(a[k], b[k]), (k, mode, interp, case)
    if mode == "composite":
        # defined part of the checkpoint buffer: the per-ray count K, then slot m < ceil(K / I) of each ray
        H, W = cam.height, cam.width
        ka = a["ckpt"][:4 * H * W].view(torch.int32).reshape(H, W)
        kb = b["ckpt"][:4 * H * W].view(torch.int32).reshape(H, W)
        assert torch.equal(ka, kb)
        ta = a["ckpt"][4 * H * W:].view(torch.float32).reshape(-1, H, W)
        tb = b["ckpt"][4 * H * W:].view(torch.float32).reshape(-1, H, W)
        used = torch.arange(ta.shape[0], device="cuda")[:, None, None] < (ka[None] + 6) // 7
        assert torch.equal(ta[used], tb[used])
        assert int(ka.max()) > 0
    if mode != "composite":
        # the oracle takes the step the library received: the float32 nearest to it
        o = oracle.render(cube, cam, mode, interp=interp, lut=scene.linear_lut(), opacity_scale=0.05,
                          step=float(np.float32(c.get("step", 0.5))), eps_pos=1e-6, eps_val=1e-4)
        g = {k: v.cpu().numpy() for k, v in a.items()}
        compare(g, o, mode, scale=float(dims[2]) if mode == "moment1" else float(np.nanmax(cube) - np.nanmin(cube)),
                max_fragile=0.15 if interp == "trilinear" else 0.01,
                what=f"sweep/{mode}/{interp}/{case}")


def test_sweep_early_exit(m, monkeypatch):
    cube = np.full((40, 16, 32), 8.0, np.float32)
    cam = _cam_z((32, 16, 40), 32, 16)
    lut = to_dev(scene.linear_lut())
    a, b = _both(m, monkeypatch, to_dev(cube), cam, "composite", lut, opacity_scale=0.3)
    for k in a:
        assert torch.equal(a[k], b[k])
    k = next(k for k in range(1, 200) if 1 - 0.7 ** k > 0.99)
    assert (a["nsamples"].cpu().numpy() == k).all()


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("interp", ["trilinear", "nearest"])
def test_sweep_mip_without_index(m, monkeypatch, case, interp):
    """MIP with no argmax output keeps the running maximum alone; values match the marcher."""
    c = CASES[case]
    dims = c["dims"]
    cube = scene.tiny_cube(config_id=70 + case, dims=dims, n_sources=2)
    cube[5, 9, 11] = np.nan
    cube[2, 3, 4] = 0.0
    cam = _cam_z(dims, c["W"], c["H"], down=c.get("down", False), angle_deg=c.get("angle_deg", 0.0),
                 spacing=c.get("spacing", 1.0), shift=NEAREST_SHIFT if interp == "nearest" else (0.0, 0.0))
    lut = to_dev(scene.linear_lut())
    a, b = _both(m, monkeypatch, to_dev(cube), cam, "mip", lut, interp=interp, step=c.get("step", 0.5),
                 index=False)
    assert set(a) == set(b) and "index" not in a
    for k in a:
        assert torch.equal(a[k], b[k]), (k, interp, case)

