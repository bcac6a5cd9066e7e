"""The C ABI on the host: the library loads, exports every symbol include/*.h declares,
its struct layouts match the binding, and invalid calls are rejected on the host
before any GPU work (these tests need no GPU and make no compute call)."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1707_00442_gb300 import build
    build.build()
    from paper_1707_00442_gb300 import _lib
    return _lib.lib()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(shw_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_header(L):
    from paper_1707_00442_gb300 import _lib
    assert set(_lib.SIGNATURES) == set(declared_functions())


def header_defines():
    src = "".join(open(h).read() for h in glob.glob(os.path.join(ROOT, "include", "*.h")))
    return {m.group(1): int(m.group(2), 0) for m in re.finditer(r"#define\s+(SHW_[A-Z0-9_]+)\s+\(?(0x[0-9a-fA-F]+|\d+)",
                                                                  src)}


def test_binding_flags_match_header():
    """The binding's flag and switch values are the header's #defines."""
    from paper_1707_00442_gb300 import _lib
    d = header_defines()
    assert (_lib.BATCH_NO_TUNE, _lib.BATCH_RETUNE) == (d["SHW_BATCH_NO_TUNE"], d["SHW_BATCH_RETUNE"])
    assert _lib.BATCH_PACK == {None: 0, "bf16": d["SHW_BATCH_PACK_BF16"], "f16": d["SHW_BATCH_PACK_F16"]}
    assert _lib.BATCH_BRICK == {None: 0, 16: d["SHW_BATCH_BRICK_16"], 32: d["SHW_BATCH_BRICK_32"]}
    for name, value in _lib.DEBUG.items():
        assert d["SHW_DEBUG_" + name.upper()] == value, name
    assert _lib.ABI_VERSION == d["SHW_ABI_VERSION"]
    assert _lib.NOALLOC_SCRATCH_BYTES == 8 << 20


def test_struct_layout(L):
    from paper_1707_00442_gb300 import _lib
    assert L.shw_struct_size(0) == C.sizeof(_lib.Volume) == 24
    assert L.shw_struct_size(1) == C.sizeof(_lib.Camera) == 68
    assert L.shw_struct_size(2) == C.sizeof(_lib.RenderParams) == 112
    assert L.shw_struct_size(3) == C.sizeof(_lib.BatchItem) == 112
    assert L.shw_struct_size(4) == C.sizeof(_lib.BatchInfo) == 296
    assert L.shw_struct_size(9) == 0
    assert L.shw_abi_version() == 5


def test_status_strings(L):
    for s in range(8):  # SHW_OK .. SHW_EBOUNDS
        assert L.shw_status_string(s)
    assert L.shw_status_string(99) == b"unknown status"


def _vol(data=0x1000, n=(8, 8, 8), storage=0):
    from paper_1707_00442_gb300 import _lib
    return _lib.Volume(data, *n, storage)


def _cam(W=16, H=16, ortho=1):
    from paper_1707_00442_gb300 import _lib
    c = _lib.Camera()
    c.eye[:] = [3.5, 3.5, -8]
    c.right[:] = [1, 0, 0]
    c.up[:] = [0, 1, 0]
    c.fwd[:] = [0, 0, 1]
    c.tan_half_fovy, c.ortho_half_h, c.ortho, c.width, c.height = 0.4, 4.0, ortho, W, H
    return c


def _params(mode=0, step=0.5, lut=0x2000, lo=-3.0, hi=8.0, smooth=0, arm=0, ntaps=0, c0=1.0, off=0.0, w=0.0):
    from paper_1707_00442_gb300 import _lib
    p = _lib.RenderParams(mode, 1, step, lo, hi, lut, 1.0, 0.99, 0.0, 64)
    p.smooth, p.smooth_arm, p.smooth_ntaps, p.smooth_c0 = smooth, arm, ntaps, c0
    for j in range(4):
        p.smooth_offset[j], p.smooth_weight[j] = off, w
    return p


def test_render_rejects_invalid_arguments_on_host(L):
    """Every case must fail validation (EINVAL) before the library touches a device."""
    EINVAL = 1
    out = 0x4000
    ok_v, ok_c, ok_p = _vol(), _cam(), _params()
    b = C.byref
    cases = [
        (None, ok_c, ok_p, out),
        (_vol(data=0), ok_c, ok_p, out),
        (_vol(n=(0, 8, 8)), ok_c, ok_p, out),
        (_vol(storage=10), ok_c, ok_p, out),          # no such storage
        (_vol(data=0x1002, storage=8), ok_c, ok_p, out),  # linear 16-bit pairs need 4-byte alignment
        (_vol(data=0x1001), ok_c, ok_p, out),       # misaligned float32 cube
        (ok_v, _cam(W=0), ok_p, out),
        (ok_v, _cam(H=-3), ok_p, out),
        (ok_v, ok_c, _params(mode=10), out),
        (ok_v, ok_c, _params(step=0.0), out),
        (ok_v, ok_c, _params(step=-1.0), out),
        (ok_v, ok_c, _params(step=float("nan")), out),
        (ok_v, ok_c, _params(lut=0), out),
        (ok_v, ok_c, _params(lut=0x2004), out),      # colour map not 16-byte aligned
        (ok_v, ok_c, _params(lo=1.0, hi=1.0), out),
        (ok_v, ok_c, _params(mode=4), out),          # RATIO without a second cube
        (ok_v, ok_c, _params(smooth=3), out),        # unknown smoothing kind
        (ok_v, ok_c, _params(smooth=1, arm=-1), out),
        (ok_v, ok_c, _params(smooth=1, arm=17), out),  # box arm beyond SHW_MAX_SMOOTH_ARM
        (ok_v, ok_c, _params(smooth=2, ntaps=5, off=1.5, w=0.1), out),  # beyond SHW_MAX_SMOOTH_TAPS
        (ok_v, ok_c, _params(smooth=2, ntaps=2, off=65.0, w=0.1), out),  # offset beyond 64 voxels
        (ok_v, ok_c, _params(smooth=2, ntaps=2, off=1.5, w=float("inf")), out),
        (ok_v, ok_c, _params(smooth=2, ntaps=1, c0=float("nan"), off=1.5, w=0.1), out),
        (ok_v, ok_c, ok_p, 0),                       # no rgba output
        (ok_v, ok_c, ok_p, 0x4008),                  # rgba not 16-byte aligned
    ]
    for v, c, p, o in cases:
        st = L.shw_render(b(v) if v is not None else None, None, b(c), b(p), o, None, None, None, None, 0, None)
        assert st == EINVAL, (v, p)
    # ratio with mismatched second cube
    v2 = _vol(n=(8, 8, 9))
    assert L.shw_render(b(ok_v), b(v2), b(ok_c), b(_params(mode=4)), out, None, None, None, None, 0, None) == EINVAL
    # checkpoints only for compositing, and big enough
    assert L.shw_render(b(ok_v), None, b(ok_c), b(ok_p), out, None, None, None, 0x8000, 1 << 30, None) == EINVAL
    p2 = _params(mode=2)
    need = L.shw_ckpt_bytes(b(ok_v), b(ok_c), b(p2))
    assert need == 16 * 16 * 4 * (1 + -(-(int((8 * 8 * 3) ** 0.5 / 0.5) + 1) // 64))
    assert L.shw_render(b(ok_v), None, b(ok_c), b(p2), out, None, None, None, 0x8000, need - 4, None) == 4  # ENOMEM


def test_pair_storage_rules_on_host(L):
    """The interleaved pair storage: line ratios only, no second volume, no in-ray smoothing,
    8-byte alignment, not in batch plans; shw_smooth_zip's argument checks."""
    EINVAL, EUNSUP = 1, 2
    b = C.byref
    pv, ok_c, out = _vol(storage=3), _cam(), 0x4000
    for mode, want in ((4, None), (9, None), (0, EUNSUP), (2, EUNSUP), (7, EUNSUP)):
        if want is not None:
            assert L.shw_render(b(pv), None, b(ok_c), b(_params(mode=mode)), out, None, None, None, None, 0,
                                None) == want, mode
    assert L.shw_render(b(pv), b(_vol()), b(ok_c), b(_params(mode=4)), out, None, None, None, None, 0,
                        None) == EINVAL  # a second volume with the pair storage
    assert L.shw_render(b(pv), None, b(ok_c), b(_params(mode=4, smooth=1, arm=2)), out, None, None, None, None,
                        0, None) == EUNSUP
    assert L.shw_render(b(_vol(storage=3, data=0x1004)), None, b(ok_c), b(_params(mode=4)), out, None, None, None,
                        None, 0, None) == EINVAL  # not 8-byte aligned
    n = 8 * 8 * 8 * 4
    assert L.shw_smooth_zip(0, 0x100000, 0x200000, 8, 8, 8, 1.0, 3, None) == EINVAL
    assert L.shw_smooth_zip(0x100000, 0, 0x200000, 8, 8, 8, 1.0, 3, None) == EINVAL
    assert L.shw_smooth_zip(0x100000, 0x100000, 0x200004, 8, 8, 8, 1.0, 3, None) == EINVAL  # out misaligned
    assert L.shw_smooth_zip(0x100000, 0x200000, 0x100000 + n // 2, 8, 8, 8, 1.0, 3, None) == EINVAL  # overlap
    assert L.shw_smooth_zip(0x100000, 0x200000 - 8, 0x200000, 8, 8, 8, 1.0, 3, None) == EINVAL  # overlap
    assert L.shw_smooth_zip(0x100000, 0x100000, 0x200000, 8, 8, 8, 0.0, 3, None) == EINVAL  # sigma
    assert L.shw_smooth_zip(0x100000, 0x100000, 0x200000, 8, 8, 8, 1.0, 17, None) == EUNSUP
    # pair bricks: 4-byte elements, an 8-byte aligned float32 pair buffer in, line ratios only
    assert L.shw_bricked_bytes(64, 64, 64, 4) == L.shw_bricked_bytes(64, 64, 64, 5) == 8 * 34 ** 3 * 4
    assert L.shw_bricked_bytes(64, 64, 64, 10) == 0
    # linear 16-bit storages: 2 bytes per voxel, 4 for the pairs
    assert L.shw_bricked_bytes(64, 64, 64, 6) == L.shw_bricked_bytes(64, 64, 64, 7) == 2 * 64 ** 3
    assert L.shw_bricked_bytes(64, 64, 64, 8) == L.shw_bricked_bytes(64, 64, 64, 9) == 4 * 64 ** 3
    assert L.shw_pack_bricks(0x100004, 64, 64, 64, 8, 0x800000, 1 << 30, None) == EINVAL  # pair input 8-aligned
    assert L.shw_pack_bricks(0x100000, 64, 64, 64, 6, 0x800000, 1000, None) == 4          # ENOMEM
    assert L.shw_pack_bricks(0x100004, 64, 64, 64, 4, 0x800000, 1 << 30, None) == EINVAL  # pair input 8-aligned
    assert L.shw_pack_bricks(0x100000, 64, 64, 64, 4, 0x800002, 1 << 30, None) == EINVAL  # 4-byte elements
    assert L.shw_pack_bricks(0x100000, 64, 64, 64, 5, 0x800000, 1000, None) == 4          # ENOMEM
    for st in (4, 5):
        assert L.shw_render(b(_vol(storage=st)), None, b(ok_c), b(_params(mode=0)), out, None, None, None, None, 0,
                            None) == EUNSUP
        assert L.shw_render(b(_vol(storage=st, data=0x1002)), None, b(ok_c), b(_params(mode=4)), out, None, None,
                            None, None, 0, None) == EINVAL
    assert L.shw_render(b(_vol(storage=10)), None, b(ok_c), b(_params(mode=4)), out, None, None, None, None, 0,
                        None) == EINVAL
    # linear 16-bit pairs: the line ratios only; linear 16-bit cubes: the staged marcher only
    # (trilinear, no in-ray smoothing), refused before any launch
    for st in (8, 9):
        assert L.shw_render(b(_vol(storage=st)), None, b(ok_c), b(_params(mode=0)), out, None, None, None, None, 0,
                            None) == EUNSUP


def test_smooth_and_pack_reject_invalid_arguments_on_host(L):
    EINVAL, EUNSUP, ENOMEM = 1, 2, 4
    assert L.shw_smooth(0, 0x1000, 8, 8, 8, 1.0, 3, None) == EINVAL
    assert L.shw_smooth(0x1000, 0x1000, 8, 8, 8, 1.0, 3, None) == EINVAL            # in place
    assert L.shw_smooth(0x1000, 0x1000 + 100, 8, 8, 8, 1.0, 3, None) == EINVAL      # overlapping
    assert L.shw_smooth(0x1000, 0x100000, 8, 8, 8, 0.0, 3, None) == EINVAL          # sigma
    assert L.shw_smooth(0x1000, 0x100000, 8, 8, 8, 1.0, -1, None) == EINVAL
    assert L.shw_smooth(0x1000, 0x100000, 8, 8, 8, 1.0, 17, None) == EUNSUP
    assert L.shw_smooth(0x1000, 0x100000, 8, 0, 8, 1.0, 3, None) == EINVAL
    assert L.shw_smooth_weights(0x1000, 0x100000, 8, 8, 8, None, 3, None) == EINVAL
    assert L.shw_bricked_bytes(64, 64, 64, 1) == 8 * 34 ** 3 * 2
    assert L.shw_bricked_bytes(65, 64, 64, 2) == 12 * 34 ** 3 * 2
    assert L.shw_bricked_bytes(64, 64, 64, 0) == 0
    assert L.shw_pack_bricks(0x1000, 64, 64, 64, 0, 0x100000, 1 << 30, None) == EINVAL
    assert L.shw_pack_bricks(0x1000, 64, 64, 64, 1, 0x100000, 1000, None) == ENOMEM


def test_no_device_is_reported(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    assert L.shw_sync_status(None) == 6  # SHW_EDEVICE


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1707_00442_gb300 import _lib
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libshw.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(ImportError):
        _lib.lib()


def test_batch_plan_rejects_invalid_arguments_on_host(L):
    from paper_1707_00442_gb300 import _lib
    b = C.byref
    h = C.c_void_p()
    items = (_lib.BatchItem * 2)()
    for it in items:
        it.vol = _vol()
        it.cam = _cam()
        it.out_rgba = 0x4000
        it.mode = 0
    p = _params()
    assert L.shw_batch_plan_create(None, items, 2, b(p), 0, None) == 1
    assert L.shw_batch_plan_create(b(h), items, 0, b(p), 0, None) == 1
    assert L.shw_batch_plan_create(b(h), items, 2, b(_params(lut=0)), 0, None) == 1
    assert L.shw_batch_plan_create(b(h), items, 2, b(_params(step=0.0)), 0, None) == 1
    assert L.shw_batch_plan_create(b(h), items, 2, b(_params(smooth=1, arm=2)), 0, None) == 2  # no in-ray smoothing
    items[1].vol = _vol(storage=3)
    assert L.shw_batch_plan_create(b(h), items, 2, b(p), 0, None) == 2      # no pair storage
    items[1].vol = _vol()
    items[1].mode = 4
    assert L.shw_batch_plan_create(b(h), items, 2, b(p), 0, None) == 2      # ratio: unsupported in a batch
    items[1].mode = 7
    assert L.shw_batch_plan_create(b(h), items, 2, b(p), 0, None) == 2      # MIP_RGB: unsupported in a batch
    items[1].mode = 10
    assert L.shw_batch_plan_create(b(h), items, 2, b(p), 0, None) == 1      # not a mode
    items[1].mode = 2
    items[1].out_rgba = 0x4004
    assert L.shw_batch_plan_create(b(h), items, 2, b(p), 0, None) == 1
    items[1].out_rgba = 0x4000
    # the plan's own bricks: one pack storage, at most one fixed edge, an edge only with packing,
    # and edge 16 only when the plan packs every item (the caller's bricks are 32^3)
    PB, PF, B16, B32 = 4, 8, 16, 32
    assert L.shw_batch_plan_create(b(h), items, 2, b(p), PB | PF, None) == 1
    assert L.shw_batch_plan_create(b(h), items, 2, b(p), PB | B16 | B32, None) == 1
    assert L.shw_batch_plan_create(b(h), items, 2, b(p), B16, None) == 1
    assert L.shw_batch_plan_create(b(h), items, 2, b(p), B32, None) == 1
    items[1].vol = _vol(storage=1)
    assert L.shw_batch_plan_create(b(h), items, 2, b(p), PF | B16, None) == 2
    # brick items are addressed with 32-bit offsets: a 1281^3 cube (< 2^31 voxels) as 32^3
    # bricks holds 41^3 * 34^3 > 2^31 elements, and is refused as bricks, plain or packed
    items[1].vol = _vol(n=(1281, 1281, 1281), storage=1)
    assert L.shw_batch_plan_create(b(h), items, 2, b(p), 0, None) == 2
    assert L.shw_render_batch_noalloc(items, 2, b(p), None) == 2
    items[1].vol = _vol(n=(1281, 1281, 1281), storage=0)
    assert L.shw_batch_plan_create(b(h), items, 2, b(p), PB, None) == 2
    assert h.value is None
    assert L.shw_render_batch(None, None) == 1
    assert L.shw_batch_plan_destroy(None) == 1
