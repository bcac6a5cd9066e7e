"""shw_render_batch_noalloc: the batch render for callers that cannot let a library allocate
device memory (a host program that owns the whole GPU through its own pool or budget, or an
interactive loop that must not stall in an allocator).  Its scratch is a fixed device array
inside the library, shared by every call.

Called through the C ABI: two calls in a row must give the existing batch-plan entry point's
images bit for bit (the same kernel, tiles and per-ray code); a later call with a different,
smaller item set must not consume the earlier call's table (its images match the batch plan
and the FP64 oracle, and the earlier call's outputs stay untouched); a request that fills the
scratch exactly is accepted, one tile more is refused with SHW_EUNSUPPORTED, and a call
during stream capture is refused.  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
import scene
from parity import TOL_F32, shw, to_dev

pytestmark = pytest.mark.gpu


def _items(m, n=10, config_id=44, lo=16, hi=64, W=40, H=36):
    dims = scene.batch_dims(n=n, lo=lo, hi=hi, config_id=config_id)
    rng = np.random.default_rng(config_id)
    modes = ("mip", "composite", "avg", "spectral")
    out, cubes = [], []
    for i, d in enumerate(dims):
        d = tuple(int(x) for x in d)
        cube = scene.batch_subcube(i, d, config_id=config_id)
        ct = to_dev(cube)
        vol = ct if i % 2 == 0 else m.pack_bricks(ct, "bf16")
        cam = scene.orbit_camera(d, rng.uniform(0, 360), rng.uniform(-60, 60), W + 5 * (i % 3), H)
        out.append((vol, cam, modes[i % len(modes)]))
        cubes.append(cube)
    return out, cubes


def _table(items, outs):
    from paper_1707_00442_gb300 import _lib
    from paper_1707_00442_gb300.api import camera_struct, volume_struct
    arr = (_lib.BatchItem * len(items))()
    for i, (vol, cam, mode) in enumerate(items):
        arr[i].vol = volume_struct(vol)
        arr[i].cam = camera_struct(cam)
        arr[i].out_rgba = outs[i].data_ptr()
        arr[i].mode = _lib.MODES[mode]
    return arr


def _call(arr, n, lut, stream=None, **kw):
    from paper_1707_00442_gb300 import _lib
    from paper_1707_00442_gb300.api import params_struct
    p = params_struct("mip", lut, **kw)
    s = torch.cuda.current_stream().cuda_stream if stream is None else stream
    return _lib.lib().shw_render_batch_noalloc(arr, n, C.byref(p), s)


def _plan_images(m, items, lut):
    plan = m.BatchPlan(items, lut=lut, opacity_scale=0.05, tune=False)
    ref = [o.clone() for o in plan.render()]
    m.sync_status()
    plan.close()
    return ref


def test_noalloc_matches_batch_plan_on_two_calls():
    m = shw()
    from paper_1707_00442_gb300 import _lib
    lut = to_dev(scene.linear_lut())
    items, _ = _items(m)
    ref = _plan_images(m, items, lut)
    outs = [torch.full_like(r, -1.0) for r in ref]
    arr = _table(items, outs)
    L = _lib.lib()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        for o in outs:
            o.fill_(-1.0)
        assert _call(arr, len(items), lut, opacity_scale=0.05) == _lib.SHW_OK
        assert L.shw_sync_status(stream) == _lib.SHW_OK
        for i, (o, r) in enumerate(zip(outs, ref)):
            assert torch.equal(o, r), (call, i)


def test_noalloc_bricks_only_matches_single_renders():
    """Items that are all bricks take the kernel without the float32 path: the images are those
    of single renders of the same bricks."""
    m = shw()
    from paper_1707_00442_gb300 import _lib
    lut = to_dev(scene.linear_lut())
    items, _ = _items(m, n=8, config_id=45)
    items = [(v if not isinstance(v, torch.Tensor) else m.pack_bricks(v, "f16"), c, md) for v, c, md in items]
    outs = [torch.full((int(c.height), int(c.width), 4), -1.0, device="cuda") for _, c, _ in items]
    arr = _table(items, outs)
    stream = torch.cuda.current_stream().cuda_stream
    assert _call(arr, len(items), lut, opacity_scale=0.05) == _lib.SHW_OK
    assert _lib.lib().shw_sync_status(stream) == _lib.SHW_OK
    for i, ((vol, cam, mode), o) in enumerate(zip(items, outs)):
        assert torch.equal(o, m.render(vol, cam, mode, lut=lut, opacity_scale=0.05)["rgba"]), i


def test_noalloc_smaller_second_call_uses_only_its_own_table():
    """A large call, then a smaller call with other cubes: the second must not consume the
    first call's (longer) work list or item table left in the shared scratch."""
    m = shw()
    from paper_1707_00442_gb300 import _lib
    lut = to_dev(scene.linear_lut())
    big, _ = _items(m, n=12)
    small, small_cubes = _items(m, n=3, config_id=45, lo=20, hi=40, W=33, H=29)
    big_outs = [torch.zeros((c.height, c.width, 4), device="cuda") for _, c, _ in big]
    assert _call(_table(big, big_outs), len(big), lut, opacity_scale=0.05) == _lib.SHW_OK
    torch.cuda.synchronize()
    for o in big_outs:
        o.fill_(-7.0)  # sentinel: the second call must not write here
    ref = _plan_images(m, small, lut)
    outs = [torch.full_like(r, -1.0) for r in ref]
    assert _call(_table(small, outs), len(small), lut, opacity_scale=0.05) == _lib.SHW_OK
    m.sync_status()
    for i, (o, r) in enumerate(zip(outs, ref)):
        assert torch.equal(o, r), i
    for o in big_outs:
        assert bool((o == -7.0).all())
    # the float32 items against the FP64 oracle (the batch-plan tolerance)
    for (vol, cam, mode), cube, o in zip(small, small_cubes, outs):
        if not isinstance(vol, torch.Tensor):
            continue  # the bfloat16 bricks: compared with the batch plan above
        orc = oracle.render(cube, cam, mode, lut=scene.linear_lut(), opacity_scale=0.05, eps_pos=1e-6,
                            eps_val=1e-4)
        ok = orc["fragile"] == 0
        assert ok.mean() >= 0.98
        assert np.abs(o.cpu().numpy() - orc["rgba"])[ok].max() <= TOL_F32, mode


def _limit_items(m, n_items):
    """n_items identical items of 3 x 5 tiles (48 x 80 pixels) on one small cube, all writing
    one output (the same values each time)."""
    cube = to_dev(scene.batch_subcube(0, (24, 20, 16), config_id=46))
    out = torch.zeros((80, 48, 4), device="cuda")
    cam = scene.orbit_camera((24, 20, 16), 35, 25, 48, 80)
    return [(cube, cam, "mip")] * n_items, out, cube, cam


def test_noalloc_accepts_a_request_that_fills_the_scratch_exactly():
    m = shw()
    from paper_1707_00442_gb300 import _lib
    lut = to_dev(scene.linear_lut())
    # 256 + 128 n + 8 * 15 n = 8 MiB exactly for n = 33824
    n = 33824
    assert 256 + 128 * n + 8 * 15 * n == _lib.NOALLOC_SCRATCH_BYTES
    items, out, cube, cam = _limit_items(m, n)
    arr = _table(items, [out] * n)
    assert _call(arr, n, lut) == _lib.SHW_OK
    m.sync_status()
    single = m.render(cube, cam, "mip", lut=lut)["rgba"]
    assert torch.equal(out, single)
    # one more item of one tile no longer fits
    items2 = items + [(cube, scene.orbit_camera((24, 20, 16), 35, 25, 16, 16), "mip")]
    out2 = torch.zeros((16, 16, 4), device="cuda")
    arr2 = _table(items2, [out] * n + [out2])
    assert _call(arr2, n + 1, lut) == _lib.SHW_EUNSUPPORTED
    torch.cuda.synchronize()
    assert float(out2.abs().max()) == 0.0


def test_noalloc_refuses_requests_beyond_its_scratch():
    m = shw()
    from paper_1707_00442_gb300 import _lib
    lut = to_dev(scene.linear_lut())
    cube = to_dev(scene.batch_subcube(0, (32, 32, 32), config_id=44))
    out = torch.zeros((8, 8, 4), device="cuda")
    cam = scene.orbit_camera((32, 32, 32), 10, 10, 2048, 2048)  # 16384 tiles per image
    n = 1 + _lib.NOALLOC_SCRATCH_BYTES // (16384 * 8)
    arr = _table([(cube, cam, "mip")] * n, [out] * n)  # never written: refused on the host
    assert _call(arr, n, lut) == _lib.SHW_EUNSUPPORTED
    assert float(out.abs().max()) == 0.0


def test_noalloc_refuses_a_capturing_stream():
    """The table is copied from host memory the call owns only while it runs, so a graph
    capture (whose replays would read it later) is refused before anything is enqueued."""
    m = shw()
    from paper_1707_00442_gb300 import _lib
    lut = to_dev(scene.linear_lut())
    items, _ = _items(m, n=2)
    outs = [torch.zeros((c.height, c.width, 4), device="cuda") for _, c, _ in items]
    arr = _table(items, outs)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    status = []
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        status.append(_call(arr, len(items), lut, stream=s.cuda_stream))
    assert status == [_lib.SHW_EUNSUPPORTED]
    m.sync_status()
