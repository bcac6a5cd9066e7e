"""Cubes of 2^31 voxels or more take the marcher's 64-bit-index instances (float32 and 16-bit
bricks).  A 2048 x 1024 x 1024 cube (8 GiB) that grows strictly along x, built on the device,
viewed along +x with parallel rays through the voxel centres: every ray's maximum is its last
voxel (nearest) or the clamped sample past it (trilinear), so MIP and its channel are exact."""
import numpy as np
import pytest
import torch

import scene
from parity import shw, to_dev

pytestmark = pytest.mark.gpu

DIMS = (2048, 1024, 1024)  # nx, ny, nz: 2^31 voxels


@pytest.fixture(scope="module")
def m():
    return shw()


@pytest.fixture(scope="module")
def big():
    nx, ny, nz = DIMS
    dev = torch.device("cuda")
    x = torch.arange(nx, device=dev, dtype=torch.float32) * 1e-3
    y = torch.arange(ny, device=dev, dtype=torch.float32) * 1e-4
    z = torch.arange(nz, device=dev, dtype=torch.float32) * 1e-4
    cube = torch.empty((nz, ny, nx), device=dev, dtype=torch.float32)
    for k in range(nz):  # one plane at a time: no 8 GiB temporaries
        cube[k] = x[None, :] + y[:, None] + z[k]
    yield cube
    del cube
    torch.cuda.empty_cache()


def _expected(last):  # last: [nz, ny] values at x = nx - 1 -> image [ny rows (y down), nz columns]
    return torch.flip(last.t(), dims=[0]).cpu().numpy()


@pytest.mark.parametrize("interp", ["nearest", "trilinear"])
def test_big_f32_mip_exact(m, big, interp):
    nx, ny, nz = DIMS
    cam = scene.ortho_axis_camera(DIMS, nz, ny, axis="x")
    lut = to_dev(scene.linear_lut())
    out = m.render(big, cam, "mip", lut=lut, interp=interp, lo=0.0, hi=3.0)
    m.sync_status()
    assert np.array_equal(out["scalar"].cpu().numpy(), _expected(big[:, :, -1]))
    assert (out["nsamples"].cpu().numpy() == 2 * nx).all()


@pytest.mark.parametrize("storage,dtype", [("bf16", torch.bfloat16), ("f16", torch.float16)])
def test_big_bricks_mip_exact(m, big, storage, dtype):
    nx, ny, nz = DIMS
    cam = scene.ortho_axis_camera(DIMS, nz, ny, axis="x")
    lut = to_dev(scene.linear_lut())
    b = m.pack_bricks(big, storage)
    assert b.data.numel() * 2 >= 2 ** 32  # 2^31 or more 16-bit elements: the 64-bit instances
    out = m.render(b, cam, "mip", lut=lut, interp="nearest", lo=0.0, hi=3.0)
    m.sync_status()
    want = _expected(big[:, :, -1].to(dtype).to(torch.float32))
    got = out["scalar"].cpu().numpy()
    del b
    torch.cuda.empty_cache()
    # rounding is monotonic, so the rounded last voxel is a maximum of the rounded row (ties
    # with the voxel before it leave the same value)
    assert np.array_equal(got, want)
