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
    assert all(t > 0 for (_, _, t) in info["candidates"])
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
