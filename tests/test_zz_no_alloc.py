"""shw_render_batch_noalloc: the batch render for callers that cannot let a library allocate
device memory (a host program that owns the whole GPU through its own pool or budget, or an
interactive loop that must not stall in an allocator).  Its scratch is a fixed device array
inside the library.

Called through the C ABI twice in a row; each time every image must match the existing
batch-plan entry point within the FP32 parity tolerance.  A request larger than the fixed
scratch must be refused with SHW_EUNSUPPORTED.  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest
import torch

import scene
from parity import TOL_F32, shw, to_dev

pytestmark = pytest.mark.gpu


def _items(m, n=10):
    dims = scene.batch_dims(n=n, lo=16, hi=64, config_id=44)
    rng = np.random.default_rng(44)
    modes = ("mip", "composite", "avg", "spectral")
    out = []
    for i, d in enumerate(dims):
        d = tuple(int(x) for x in d)
        ct = to_dev(scene.batch_subcube(i, d, config_id=44))
        vol = ct if i % 2 == 0 else m.pack_bricks(ct, "bf16")
        cam = scene.orbit_camera(d, rng.uniform(0, 360), rng.uniform(-60, 60), 40 + 5 * (i % 3), 36)
        out.append((vol, cam, modes[i % len(modes)]))
    return out


def test_noalloc_matches_batch_plan_on_two_calls():
    m = shw()
    from paper_1707_00442_gb300 import _lib
    from paper_1707_00442_gb300.api import camera_struct, params_struct, volume_struct
    lut = to_dev(scene.linear_lut())
    items = _items(m)
    plan = m.BatchPlan(items, lut=lut, opacity_scale=0.05, tune=False)
    ref = [o.clone() for o in plan.render()]
    m.sync_status()
    plan.close()

    outs = [torch.full_like(r, -1.0) for r in ref]
    arr = (_lib.BatchItem * len(items))()
    for i, (vol, cam, mode) in enumerate(items):
        arr[i].vol = volume_struct(vol)
        arr[i].cam = camera_struct(cam)
        arr[i].out_rgba = outs[i].data_ptr()
        arr[i].mode = _lib.MODES[mode]
    p = params_struct("mip", lut, opacity_scale=0.05)
    L = _lib.lib()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        for o in outs:
            o.fill_(-1.0)
        assert L.shw_render_batch_noalloc(arr, len(items), C.byref(p), stream) == _lib.SHW_OK
        assert L.shw_sync_status(stream) == _lib.SHW_OK
        for o, r in zip(outs, ref):
            assert float((o - r).abs().max()) <= TOL_F32, call


def test_noalloc_refuses_requests_beyond_its_scratch():
    m = shw()
    from paper_1707_00442_gb300 import _lib
    from paper_1707_00442_gb300.api import camera_struct, params_struct, volume_struct
    lut = to_dev(scene.linear_lut())
    cube = to_dev(scene.batch_subcube(0, (32, 32, 32), config_id=44))
    out = torch.zeros((8, 8, 4), device="cuda")
    cam = scene.orbit_camera((32, 32, 32), 10, 10, 2048, 2048)  # 16384 tiles per image
    n = 1 + _lib.NOALLOC_SCRATCH_BYTES // (16384 * 8)
    arr = (_lib.BatchItem * n)()
    for i in range(n):
        arr[i].vol = volume_struct(cube)
        arr[i].cam = camera_struct(cam)
        arr[i].out_rgba = out.data_ptr()  # never written: the request is refused on the host
        arr[i].mode = _lib.MODES["mip"]
    p = params_struct("mip", lut)
    L = _lib.lib()
    assert L.shw_render_batch_noalloc(arr, n, C.byref(p), torch.cuda.current_stream().cuda_stream) == \
        _lib.SHW_EUNSUPPORTED
    assert float(out.abs().max()) == 0.0
