"""The batched persistent render (shw_batch_plan_create / shw_render_batch) on the GPU.

Every image of a batch must equal shw_render of that item (same per-ray code, so
bit-identical), match the oracle, survive repeated graph launches, and the plan's
autotuner and host-side fault injection must behave as documented."""
import os

import numpy as np
import pytest
import torch

import oracle
import scene
from parity import compare, shw, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    return shw()


def _batch(n=24, lo=16, hi=64, storage_cycle=("f32", "bf16", "f16"), modes=("mip", "composite", "avg", "spectral"),
           W=48, H=40):
    dims = scene.batch_dims(n=n, lo=lo, hi=hi)
    rng = np.random.default_rng(5)
    items = []
    for i, d in enumerate(dims):
        d = tuple(int(x) for x in d)
        cube = scene.batch_subcube(i, d)
        cam = scene.orbit_camera(d, rng.uniform(0, 360), rng.uniform(-60, 60), W + (i % 3) * 7, H + (i % 2) * 5)
        items.append((cube, cam, modes[i % len(modes)], storage_cycle[i % len(storage_cycle)]))
    return items


def _dev_items(m, items):
    out = []
    for cube, cam, mode, st in items:
        ct = to_dev(cube)
        vol = ct if st == "f32" else m.pack_bricks(ct, st)
        out.append((vol, cam, mode))
    return out


def test_batch_equals_single_renders_and_oracle(m):
    items = _batch()
    lut = to_dev(scene.linear_lut())
    dev = _dev_items(m, items)
    plan = m.BatchPlan(dev, lut=lut, opacity_scale=0.05, retune=True)
    outs = [o.cpu().numpy() for o in plan.render()]
    m.sync_status()
    info = plan.info
    assert info["n_items"] == len(items) and info["tuned"]
    assert all(t > 0 for (*_, t) in info["candidates"])
    for (vol, cam, mode), img, (cube, _, _, st) in zip(dev, outs, items):
        single = m.render(vol, cam, mode, lut=lut, opacity_scale=0.05)["rgba"].cpu().numpy()
        assert np.array_equal(img, single), (mode, st)
    # oracle parity on the float32 items
    for (cube, cam, mode, st), img in zip(items, outs):
        if st != "f32":
            continue
        o = oracle.render(cube, cam, mode, lut=scene.linear_lut(), opacity_scale=0.05, eps_pos=1e-6, eps_val=1e-4)
        ok = o["fragile"] == 0  # includes near-ties of the maximum (spectral hue)
        err = np.abs(img - o["rgba"])[ok].max()
        assert err <= 1e-5, (mode, err)
    plan.close()


def test_batch_relaunch_and_cache(m):
    items = _batch(n=12, storage_cycle=("f32",), modes=("mip", "composite"))
    lut = to_dev(scene.linear_lut())
    dev = _dev_items(m, items)
    p1 = m.BatchPlan(dev, lut=lut, opacity_scale=0.05)
    a = [o.clone() for o in p1.render()]
    for _ in range(3):
        b = p1.render()
    m.sync_status()
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    # same signature: the cached choice is reused without re-timing
    p2 = m.BatchPlan(dev, lut=lut, opacity_scale=0.05)
    assert not p2.info["tuned"]
    assert (p2.info["tile"], p2.info["ctas_per_sm"]) == (p1.info["tile"], p1.info["ctas_per_sm"])
    p3 = m.BatchPlan(dev, lut=lut, opacity_scale=0.05, tune=False)
    assert (p3.info["tile"], p3.info["ctas_per_sm"]) == (16, 4)
    for p in (p1, p2, p3):
        p.close()


def test_batch_fault_injection(m):
    """Host-side faults: allocation and graph capture failures are reported, nothing leaks a plan."""
    items = _batch(n=4, storage_cycle=("f32",))
    lut = to_dev(scene.linear_lut())
    dev = _dev_items(m, items)
    with m.debug_flags("fault_alloc"), pytest.raises(m.ShwError) as e:
        m.BatchPlan(dev, lut=lut, tune=False)
    assert e.value.status == 4  # SHW_ENOMEM
    with m.debug_flags("fault_graph"), pytest.raises(m.ShwError) as e:
        m.BatchPlan(dev, lut=lut, tune=False)
    assert e.value.status == 3  # SHW_ECUDA
    p = m.BatchPlan(dev, lut=lut, tune=False)
    p.render()
    m.sync_status()
    p.close()


@pytest.mark.parametrize("mode", ["ratio", "moment1"])
def test_batch_rejects_ratio_and_moment(m, mode):
    items = _batch(n=2, storage_cycle=("f32",))
    dev = _dev_items(m, items)
    dev[1] = (dev[1][0], dev[1][1], mode)
    with pytest.raises(m.ShwError) as e:
        m.BatchPlan(dev, lut=to_dev(scene.linear_lut()), tune=False)
    assert e.value.status == 2


def test_batch_survey_shaped(m):
    """Sub-cubes with each axis log-uniform in [32, 256] (the batch workload's size law), fewer of them."""
    items = _batch(n=30, lo=32, hi=256, storage_cycle=("f32", "bf16"), modes=("mip", "composite"), W=96, H=96)
    lut = to_dev(scene.linear_lut())
    dev = _dev_items(m, items)
    plan = m.BatchPlan(dev, lut=lut, opacity_scale=0.02)
    outs = plan.render()
    m.sync_status()
    rng = np.random.default_rng(1)
    for j in rng.choice(len(items), size=6, replace=False):
        vol, cam, mode = dev[j]
        single = m.render(vol, cam, mode, lut=lut, opacity_scale=0.02)["rgba"]
        assert torch.equal(outs[j], single)
    plan.close()


def test_render_items_equals_plan(m):
    """One launch per item from the library's own loop (shw_render_items), the path a plan is
    measured against, gives the plan's images bit for bit."""
    items = _batch(n=10, storage_cycle=("f32", "bf16"), modes=("mip", "composite"))
    lut = to_dev(scene.linear_lut())
    dev = _dev_items(m, items)
    plan = m.BatchPlan(dev, lut=lut, opacity_scale=0.05, tune=False)
    a = [o.clone() for o in plan.render()]
    for o in plan.outputs:
        o.fill_(-1.0)
    b = plan.render_one_by_one()
    m.sync_status()
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    plan.close()


ROUND = {"bf16": oracle.round_bf16, "f16": oracle.round_f16}


def _own_brick_bytes(dims, edge):
    """Bytes of one cube as 16-bit bricks of this edge (layout of shw_pack_bricks with 32 replaced
    by the edge and 34 by edge + 2), rounded up to the plan's 256-byte item alignment."""
    nb = np.prod([-(-int(n) // edge) for n in dims])
    return -(-int(nb) * (edge + 2) ** 3 * 2 // 256) * 256


@pytest.mark.parametrize("pack", ["bf16", "f16"])
@pytest.mark.parametrize("brick", [16, 32])
def test_batch_packs_its_own_bricks(m, pack, brick):
    """A plan that rounds its float32 items into 16-bit bricks of its own, at a fixed edge: every
    image equals shw_render of shw_pack_bricks of the item (32^3 bricks; the values and the
    arithmetic do not depend on the edge), and matches the oracle run on the rounded cube."""
    items = _batch(n=14, lo=1, hi=70, storage_cycle=("f32",), modes=("mip", "composite", "avg", "spectral"))
    items[0] = (scene.batch_subcube(90, (1, 1, 1)), scene.orbit_camera((1, 1, 1), 20, 10, 24, 16), "mip", "f32")
    items[1] = (scene.batch_subcube(91, (16, 17, 33)), scene.orbit_camera((16, 17, 33), 70, -30, 40, 36), "avg", "f32")
    lut = to_dev(scene.linear_lut())
    dev = _dev_items(m, items)
    for interp in ("trilinear", "nearest"):
        plan = m.BatchPlan(dev, lut=lut, opacity_scale=0.05, interp=interp, tune=False, pack=pack, brick=brick)
        outs = [o.clone() for o in plan.render()]
        m.sync_status()
        info = plan.info
        assert info["brick"] == brick and not info["tuned"]
        want = sum(_own_brick_bytes(cube.shape[::-1], brick) for cube, *_ in items)
        assert info["packed_bytes"] == want
        assert [c[2] for c in info["candidates"]] == [brick] * 6
        for (vol, cam, mode), img in zip(dev, outs):
            single = m.render(m.pack_bricks(vol, pack), cam, mode, lut=lut, opacity_scale=0.05, interp=interp)["rgba"]
            assert torch.equal(img, single), (mode, interp)
        plan.close()
    for (cube, cam, mode, _), img in list(zip(items, outs))[:6]:
        o = oracle.render(ROUND[pack](cube), cam, mode, lut=scene.linear_lut(), opacity_scale=0.05, interp="nearest",
                          eps_pos=1e-6, eps_val=1e-4)
        ok = o["fragile"] == 0
        err = np.abs(img.cpu().numpy() - o["rgba"])[ok].max()
        assert err <= 1e-5, (mode, err)


def test_batch_tunes_the_brick_edge(m):
    """Packing plans time every tile / CTAs-per-SM choice at both brick edges, keep the fastest
    and cache it; the images do not depend on the choice."""
    items = _batch(n=16, lo=16, hi=96, storage_cycle=("f32",), modes=("mip", "composite"))
    lut = to_dev(scene.linear_lut())
    dev = _dev_items(m, items)
    p1 = m.BatchPlan(dev, lut=lut, opacity_scale=0.05, pack="bf16", retune=True)
    a = [o.clone() for o in p1.render()]
    m.sync_status()
    info = p1.info
    assert info["tuned"] and len(info["candidates"]) == 12
    assert sorted({c[2] for c in info["candidates"]}) == [16, 32]
    assert all(t > 0 for (*_, t) in info["candidates"])
    best = min(info["candidates"], key=lambda c: c[3])
    assert (info["tile"], info["ctas_per_sm"], info["brick"]) == best[:3]
    for (vol, cam, mode), img in zip(dev, a):
        assert torch.equal(img, m.render(m.pack_bricks(vol, "bf16"), cam, mode, lut=lut, opacity_scale=0.05)["rgba"])
    p2 = m.BatchPlan(dev, lut=lut, opacity_scale=0.05, pack="bf16")
    assert not p2.info["tuned"] and p2.info["brick"] == info["brick"]
    b = p2.render()
    m.sync_status()
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    for p in (p1, p2):
        p.close()


def test_batch_pack_beside_callers_bricks(m):
    """Items the caller packed (32^3) beside float32 items the plan packs: the edge stays 32
    (16 is refused), and every image still equals its single render."""
    items = _batch(n=9, storage_cycle=("f32", "bf16", "f16"), modes=("mip", "composite", "avg"))
    lut = to_dev(scene.linear_lut())
    dev = _dev_items(m, items)
    plan = m.BatchPlan(dev, lut=lut, opacity_scale=0.05, pack="f16", retune=True)
    outs = plan.render()
    m.sync_status()
    info = plan.info
    assert info["brick"] == 32 and [c[2] for c in info["candidates"]] == [32] * 6
    for (vol, cam, mode), img, (_, _, _, st) in zip(dev, outs, items):
        v = m.pack_bricks(vol, "f16") if st == "f32" else vol
        assert torch.equal(img, m.render(v, cam, mode, lut=lut, opacity_scale=0.05)["rgba"]), (mode, st)
    plan.close()
    with pytest.raises(m.ShwError) as e:
        m.BatchPlan(dev, lut=lut, pack="f16", brick=16, tune=False)
    assert e.value.status == 2  # SHW_EUNSUPPORTED
    with pytest.raises(m.ShwError) as e:
        m.BatchPlan(dev, lut=lut, brick=16, tune=False)  # an edge without a pack storage
    assert e.value.status == 1  # SHW_EINVAL


def test_batch_of_bricks_only(m):
    """A plan whose items are all the caller's bricks takes the kernel without the float32 path;
    the images are unchanged."""
    items = _batch(n=8, storage_cycle=("bf16", "f16"), modes=("mip", "composite", "spectral", "avg"))
    lut = to_dev(scene.linear_lut())
    dev = _dev_items(m, items)
    plan = m.BatchPlan(dev, lut=lut, opacity_scale=0.05, tune=False)
    outs = [o.clone() for o in plan.render()]
    m.sync_status()
    assert plan.info["brick"] == 0
    for (vol, cam, mode), img in zip(dev, outs):
        assert torch.equal(img, m.render(vol, cam, mode, lut=lut, opacity_scale=0.05)["rgba"]), mode
    plan.close()


def test_batch_runs_one_kernel_per_kind(m):
    """Float32 cubes and bricks in one plan run as two kernels in the plan's graph (one
    work list each); a plan of one kind runs one.  The images equal the single renders."""
    lut = to_dev(scene.linear_lut())
    for cycle, kernels in ((("f32", "bf16", "f16"), 2), (("f32",), 1), (("bf16", "f16"), 1)):
        items = _batch(n=7, storage_cycle=cycle, modes=("mip", "composite", "avg", "spectral"))
        dev = _dev_items(m, items)
        plan = m.BatchPlan(dev, lut=lut, opacity_scale=0.05, tune=False)
        before = m.launch_count()
        outs = plan.render()
        assert m.launch_count() == before + kernels, cycle
        m.sync_status()
        for (vol, cam, mode), img in zip(dev, outs):
            assert torch.equal(img, m.render(vol, cam, mode, lut=lut, opacity_scale=0.05)["rgba"]), (cycle, mode)
        plan.close()
