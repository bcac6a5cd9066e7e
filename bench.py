"""Benchmark of the spectral-cube ray caster on the survey-sized workload.

One step = the whole hot path over the survey input (512 x 512 x 1024 float32 cube
and its co-registered second line): separable Gaussian smoothing (sigma 2, radius 6)
of both cubes (the second straight into the line ratio's interleaved pair storage),
then one 1920 x 1080 perspective render (yaw 30, pitch 20, fov 45,
step 0.5, trilinear) per transfer function -- MIP, average, compositing,
spectral-position colouring, line ratio -- on the smoothed cubes.

value   = ray-cast Gsamples/s over the whole job (samples of all renders of all ranks / time)
e2e     = the same metric through the public API with host buffers: the two cubes copied
          host->device and the five RGBA images copied back every step
Launch: python bench.py [--gpus N --steps K --warmup W]; N > 1 under torchrun, one rank
per GPU, each rank an independent replica (weak scaling, no collective on the data path).
--impl reference times the FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import scene  # noqa: E402
from scene import workloads as WL  # noqa: E402

WORKLOADS = {"survey": WL.SURVEY, "survey-small": WL.SURVEY_SMALL}
METRIC = "ray-cast Gsamples/s and fps vs plain FP32 path; fraction of HBM roofline"
UNIT = "Gsamples/s"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def load_peaks():
    try:
        with open(PEAKS_PATH) as f:
            p = json.load(f)
        return p, "measured"
    except (OSError, ValueError):
        return dict(FALLBACK_PEAKS), "fallback"


# --------------------------------------------------------------------------- clocks

def _pci_key(pci: str):
    """(domain, bus, device, function) of a PCI id string, or the string itself."""
    try:
        dom, bus, rest = pci.strip().lower().split(":")
        dev, fn = rest.split(".")
        return (int(dom, 16), int(bus, 16), int(dev, 16), int(fn, 16))
    except ValueError:
        return pci


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples taken while the timed region runs."""
    Q = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.bus_id = bus_id
        self.lines: list[str] = []
        self.proc = None
        self.thread = None

    def start(self):
        # every GPU the tool lists; stop() keeps the rows of this one (by PCI bus id)
        cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        return self.summary()

    def summary(self):
        """Median SM clock, maximum clock and throttle reasons of this GPU's samples."""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = [[x.strip() for x in ln.split(",")] for ln in self.lines]
        rows = [f for f in rows if len(f) >= 10]
        matched = False
        if self.bus_id:  # this GPU's rows, the PCI ids compared field by field (domain widths differ)
            mine = [f for f in rows if _pci_key(f[1]) == _pci_key(self.bus_id)]
            matched = bool(mine)
            rows = mine if mine else rows
        for f in rows:
            try:
                sm.append(float(f[2]))
                mx.append(float(f[3]))
            except ValueError:
                continue
            for name, val in zip(names, f[6:10]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "gpu_pci": self.bus_id if matched else "all listed GPUs"}


# --------------------------------------------------------------------------- workload

def make_inputs(w=None):
    w = WL.SURVEY if w is None else w
    t = time.time()
    cube = scene.survey_cube(dims=w["dims"], n_sources=w["n_sources"])
    cube2 = scene.ratio_cube(cube)
    log(f"inputs generated in {time.time() - t:.1f}s")
    return cube, cube2


class Step:
    """The survey step on one GPU: 2 smooths + 5 renders, all launches on one stream.

    The first cube is smoothed into s1 (read by the four single-cube renders); the second is
    smoothed into the line ratio's interleaved pair storage next to s1 (shw_smooth_zip), so
    the ratio render fetches both cubes' corners with one load."""

    def __init__(self, shw, torch, cube_t, cube2_t, w):
        self.shw, self.torch, self.w = shw, torch, w
        self.cam = WL.survey_camera(w=w)
        dev = cube_t.device
        self.cube, self.cube2 = cube_t, cube2_t
        self.s1 = torch.empty_like(cube_t)
        self.pair = torch.empty(tuple(cube2_t.shape) + (2,), dtype=torch.float32, device=dev)
        self.lut = torch.from_numpy(scene.linear_lut()).to(dev)
        self.rlut = torch.from_numpy(scene.ratio_lut()).to(dev)
        H, W = self.cam.height, self.cam.width
        self.outs = {m: {"rgba": torch.empty((H, W, 4), dtype=torch.float32, device=dev)} for m in WL.MODES}
        self.names = ["smooth", "smooth2"] + [f"render_{m}" for m in WL.MODES]

    def launches(self):
        shw, w = self.shw, self.w
        yield "smooth", lambda: shw.smooth(self.cube, w["sigma"], w["radius"], out=self.s1)
        yield "smooth2", lambda: shw.smooth_zip(self.cube2, self.s1, w["sigma"], w["radius"], out=self.pair)
        for m in WL.MODES:
            kw = dict(WL.MODE_PARAMS[m])
            lut = self.rlut if m == "ratio" else self.lut
            yield f"render_{m}", (lambda m=m, kw=kw, lut=lut: shw.render(
                self.vol_of(m), self.cam, m, lut=lut, step=w["step"], scalar=False, index=False, nsamples=False,
                out=self.outs[m], **kw))

    def vol_of(self, m):
        return self.pair if m == "ratio" else self.s1

    def run(self, events=None):
        for name, fn in self.launches():
            if events is not None:
                e0 = self.torch.cuda.Event(enable_timing=True)
                e1 = self.torch.cuda.Event(enable_timing=True)
                e0.record()
                fn()
                e1.record()
                events.setdefault(name, []).append((e0, e1))
            else:
                fn()

    def count_samples(self):
        """Samples per render (untimed pass with the per-ray sample-count output)."""
        shw, w = self.shw, self.w
        per = {}
        shw.smooth(self.cube, w["sigma"], w["radius"], out=self.s1)
        shw.smooth_zip(self.cube2, self.s1, w["sigma"], w["radius"], out=self.pair)
        for m in WL.MODES:
            kw = dict(WL.MODE_PARAMS[m])
            lut = self.rlut if m == "ratio" else self.lut
            o = shw.render(self.vol_of(m), self.cam, m, lut=lut, step=w["step"], scalar=False, index=False,
                           nsamples=True, **kw)
            per[m] = int(o["nsamples"].sum(dtype=self.torch.int64).item())
        return per


def pci_id(torch, dev):
    """The device's PCI location as domain:bus:device.function (lower-case hex), or None.
    Some PyTorch versions give the fields as numbers, others the whole string."""
    try:
        pr = torch.cuda.get_device_properties(dev)
        bus = pr.pci_bus_id
        if isinstance(bus, int):
            return f"{getattr(pr, 'pci_domain_id', 0):04x}:{bus:02x}:{getattr(pr, 'pci_device_id', 0):02x}.0"
        return str(bus).lower()
    except Exception:  # noqa: BLE001 -- optional information
        return None


def bind_to_gpu_node(torch, dev):
    """Run this process on the host cores next to the GPU (its PCI device's local CPU list),
    so that the pinned input buffers are placed in the memory attached to them.  Best
    effort; returns the NUMA node, or None where the system does not say."""
    try:
        bus = pci_id(torch, dev)
        base = f"/sys/bus/pci/devices/{bus}"
        if not os.path.exists(base) and len(bus.split(":")[0]) > 4:  # an 8-digit domain
            base = f"/sys/bus/pci/devices/{bus[len(bus.split(':')[0]) - 4:]}"
        cpus = open(os.path.join(base, "local_cpulist")).read().strip()
        node = int(open(os.path.join(base, "numa_node")).read().strip())
        sel = set()
        for part in cpus.split(","):
            a, _, b = part.partition("-")
            sel.update(range(int(a), int(b or a) + 1))
        if sel:
            os.sched_setaffinity(0, sel)
        log(f"host: bound to the GPU's local cores {cpus} (NUMA node {node})")
        return node
    except Exception as e:  # noqa: BLE001 -- a hint only
        log(f"host: GPU-local cores unknown ({e}); running unbound")
        return None


def copy_bandwidth(torch, dst, src, reps=3):
    """Host-to-device copy rate of one pinned buffer (GB/s), for the end-to-end record."""
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        dst.copy_(src, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return src.numel() * src.element_size() / (statistics.median(ts) * 1e-3) / 1e9


class E2EPipeline:
    """The step fed from and drained to host memory, as a stream of frames would run it:
    uploads on one stream, kernels on the current stream, downloads on a third.  A cube's
    upload for the next step starts once this step's smoothing has consumed it, so it
    overlaps the renders; each image's download overlaps the renders after it.  The renders
    that need only the first cube run before the second cube's smoothing, so the second
    upload overlaps them too.  Every step still moves both cubes in and all images out."""

    def __init__(self, step, cube_h, cube2_h, rgba_h):
        import torch
        self.torch, self.step = torch, step
        self.cube_h, self.cube2_h, self.rgba_h = cube_h, cube2_h, rgba_h
        dev = step.cube.device
        self.cin, self.cout = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
        # two sets of device images, alternating by step, so no render waits for the previous
        # step's download of its image
        self.outs = [step.outs, {m: {"rgba": torch.empty_like(o["rgba"])} for m, o in step.outs.items()}]

    def _ev(self, stream):
        e = self.torch.cuda.Event()
        e.record(stream)
        return e

    def run(self, steps):
        torch, st, shw, w = self.torch, self.step, self.step.shw, self.step.w
        main = torch.cuda.current_stream()
        free1 = free2 = self._ev(main)
        out_free = [{m: free1 for m in WL.MODES}, {m: free1 for m in WL.MODES}]
        first = [m for m in WL.MODES if m != "ratio"]
        for i in range(steps):
            outs, ofree = self.outs[i & 1], out_free[i & 1]
            self.cin.wait_event(free1)
            with torch.cuda.stream(self.cin):
                st.cube.copy_(self.cube_h, non_blocking=True)
            in1 = self._ev(self.cin)
            self.cin.wait_event(free2)
            with torch.cuda.stream(self.cin):
                st.cube2.copy_(self.cube2_h, non_blocking=True)
            in2 = self._ev(self.cin)
            main.wait_event(in1)
            shw.smooth(st.cube, w["sigma"], w["radius"], out=st.s1)
            free1 = self._ev(main)
            for m in first + ["ratio"]:
                if m == "ratio":
                    main.wait_event(in2)
                    shw.smooth_zip(st.cube2, st.s1, w["sigma"], w["radius"], out=st.pair)
                    free2 = self._ev(main)
                main.wait_event(ofree[m])
                kw = dict(WL.MODE_PARAMS[m])
                shw.render(st.vol_of(m), st.cam, m, lut=st.rlut if m == "ratio" else st.lut, step=w["step"],
                           scalar=False, index=False, nsamples=False, out=outs[m], **kw)
                self.cout.wait_event(self._ev(main))
                with torch.cuda.stream(self.cout):
                    self.rgba_h[m].copy_(outs[m]["rgba"], non_blocking=True)
                ofree[m] = self._ev(self.cout)
        main.wait_stream(self.cin)
        main.wait_stream(self.cout)

    def copies_only(self, steps):
        """CUDA-event time (ms) of `steps` steps' uploads and downloads alone, on the same streams."""
        torch, st = self.torch, self.step
        main = torch.cuda.current_stream()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(main)
        self.cin.wait_stream(main)
        self.cout.wait_stream(main)
        for _ in range(steps):
            with torch.cuda.stream(self.cin):
                st.cube.copy_(self.cube_h, non_blocking=True)
                st.cube2.copy_(self.cube2_h, non_blocking=True)
            with torch.cuda.stream(self.cout):
                for m in WL.MODES:
                    self.rgba_h[m].copy_(st.outs[m]["rgba"], non_blocking=True)
        main.wait_stream(self.cin)
        main.wait_stream(self.cout)
        e1.record(main)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)


# --------------------------------------------------------------------------- roofline

def kernel_roofline(name, t_ms, nvox, samples_per, peaks, sm_mhz, image_bytes=0, sms=152):
    """Algorithmic work per launch / measured duration, against the bound of that kernel.

    Smoothing: HBM bytes.  The method moves 8 B per voxel (read the cube, write its smoothed
    copy); the second smoothing also re-reads the first result and writes both into the line
    ratio's interleaved pair storage (16 B per voxel moved), reported beside as frac_moved.
    Renders: instruction issue.  Their loops run out of shared memory and are bound by the
    schedulers, so the roofline is warp instructions issued per second (the ncu count per
    sample of this build times the samples, over the time) against SMs x 4 schedulers x SM
    clock; the HBM fraction of the cube bytes read once and the image written, and the FP32
    fraction of the method's flops, are reported beside."""
    hbm = float(peaks["hbm_gbs"])
    traffic = TRAFFIC_PER_LAUNCH.get(name)
    if name.startswith("smooth"):
        bytes_ = 8 * nvox
        ach = bytes_ / (t_ms * 1e-3) / 1e9
        rec = {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
               "frac": round(ach / hbm, 4), "algorithmic_bytes": bytes_,
               # the three 1-D passes as separate sweeps would move 24 B per voxel: the rate
               # that form would need to match this time
               "three_pass_bytes": 24 * nvox,
               "three_pass_equiv_frac": round(24 * nvox / (t_ms * 1e-3) / 1e9 / hbm, 4)}
        if name == "smooth2":
            moved = 16 * nvox
            rec["moved_bytes"] = moved
            rec["frac_moved"] = round(moved / (t_ms * 1e-3) / 1e9 / hbm, 4)
    else:
        mode = name[len("render_"):]
        ns = samples_per[mode]
        cube_bytes = (8 if mode == "ratio" else 4) * nvox  # the ratio reads both cubes
        alg_bytes = cube_bytes + image_bytes
        flops = ALG_FLOPS_PER_SAMPLE[mode] * ns
        fp32_peak = FP32_LANES_PER_SM * 2 * sms * float(sm_mhz) * 1e6 / 1e12  # TFLOP/s (FMA = 2)
        rec = {"samples": ns, "gsamples_per_s": round(ns / (t_ms * 1e-3) / 1e9, 2),
               "hbm_frac": round(alg_bytes / (t_ms * 1e-3) / 1e9 / hbm, 4), "algorithmic_bytes": alg_bytes,
               "fp32_frac_alg_flops": round(flops / (t_ms * 1e-3) / 1e12 / fp32_peak, 4)}
        ips = WARP_INST_PER_SAMPLE.get(mode)
        loaded = peaks.get("clocks_under_load", {}).get("sm_mhz_median")
        if ips:
            peak = sms * SCHEDULERS_PER_SM * float(sm_mhz) * 1e6 / 1e9  # G warp instructions / s
            ach = ips * ns / (t_ms * 1e-3) / 1e9
            rec = {"bound": "alu", "achieved": round(ach, 1), "peak": round(peak, 1), "unit": "Gwarp-inst/s",
                   "frac": round(ach / peak, 4), "warp_inst_per_sample": ips, **rec}
            if loaded:  # against the loaded median clock recorded with the peaks as well
                rec["frac_at_peaks_loaded_clock"] = round(ach / (sms * SCHEDULERS_PER_SM * float(loaded) * 1e-3), 4)
        else:  # no instruction count for this build: the FP32 roofline of the method's flops
            ach = flops / (t_ms * 1e-3) / 1e12
            rec = {"bound": "alu", "achieved": round(ach, 3), "peak": round(fp32_peak, 2), "unit": "TFLOP/s",
                   "frac": round(ach / fp32_peak, 4), **rec}
    if traffic:
        rec["dram_frac_ncu_bytes"] = round(traffic / (t_ms * 1e-3) / 1e9 / hbm, 4)
    return rec


FP32_LANES_PER_SM = 128
SCHEDULERS_PER_SM = 4  # each issues at most one warp instruction per cycle
# FP32 flops the method needs per trilinear sample: 3 fraction weights,
# 7 lerps (sub + FMA = 3 flops), plus the transfer function's own arithmetic.
_TRI = 3 + 7 * 3
ALG_FLOPS_PER_SAMPLE = {"mip": _TRI + 1, "spectral": _TRI + 1, "avg": _TRI + 4,
                        "ratio": 2 * _TRI + 2, "composite": _TRI + 2 + 8 + 6 + 3 + 2}


def step_config(W, world):
    """The workload of one step, identical for both arms of the benchmark."""
    return {"workload": W["name"], "cube": "x".join(map(str, W["dims"])) + " f32 + ratio cube",
            "image": f"{W['width']}x{W['height']} perspective yaw30 pitch20 fov45", "step_vox": W["step"],
            "modes": WL.MODES, "smooth": "sigma 2, radius 6, both cubes (the second into the line ratio's pair storage)",
            "interp": "trilinear", "l2": "inputs larger than L2 (1 GiB cubes vs 129 MB L2)",
            "parallelism": f"replicas x{world}"}


# --------------------------------------------------------------------------- multi-rank timing

def max_over_ranks(ms_local: float, world: int, device=None) -> float:
    """The job's time: the slowest rank's (all ranks hold the value afterwards)."""
    if world <= 1:
        return ms_local
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank_step: float, steps: int, ms_job: float) -> float:
    """Units processed by all ranks (weak scaling: each rank its own replica) per second, in G."""
    return world * units_per_rank_step * steps / (ms_job * 1e-3) / 1e9


# --------------------------------------------------------------------------- our arm

def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_1707_00442_gb300 as shw
    shw._lib.lib()  # the CUDA library must load: there is no fallback

    W = WORKLOADS[args.workload]
    host_node = bind_to_gpu_node(torch, dev)
    cube, cube2 = make_inputs(W)
    nvox = cube.size
    cube_h = torch.from_numpy(cube).pin_memory()
    cube2_h = torch.from_numpy(cube2).pin_memory()
    cube_t, cube2_t = cube_h.to(dev), cube2_h.to(dev)
    h2d_gbs = copy_bandwidth(torch, cube_t, cube_h)
    step = Step(shw, torch, cube_t, cube2_t, W)
    samples_per = step.count_samples()
    samples_step = sum(samples_per.values())
    log("samples per render:", samples_per)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step.run()
    barrier()

    clocks = ClockSampler(bus_id=pci_id(torch, dev))
    clocks.start()

    events = {}
    launches0 = shw.launch_count()
    barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(args.steps):
        step.run(events)
    t1.record()
    barrier()
    launches = shw.launch_count() - launches0
    clk = clocks.stop()
    ms_total = max_over_ranks(t0.elapsed_time(t1), world, dev)
    per_kernel = {k: statistics.mean(a.elapsed_time(b) for a, b in v) for k, v in events.items()}

    # end to end through the public API with host buffers: every step uploads both cubes
    # and downloads the five images, pipelined over three streams
    rgba_h = {m: torch.empty(step.outs[m]["rgba"].shape, dtype=torch.float32).pin_memory() for m in WL.MODES}
    e2e = E2EPipeline(step, cube_h, cube2_h, rgba_h)
    e2e.run(1)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    e2e.run(args.steps)
    e1.record()
    barrier()
    ms_e2e = max_over_ranks(e0.elapsed_time(e1), world, dev)
    ms_copies = e2e.copies_only(args.steps)  # the same uploads and downloads without kernels
    h2d = 2 * nvox * 4
    d2h = sum(int(np.prod(rgba_h[m].shape)) * 4 for m in WL.MODES)

    peaks, peaks_src = load_peaks()
    sm_mhz = (clk or {}).get("sm_mhz") or peaks.get("clocks_under_load", {}).get("sm_mhz_median") or 1485.0
    img_bytes = step.cam.width * step.cam.height * 16  # the RGBA float32 image each render writes
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    roof = {k: kernel_roofline(k, t, nvox, samples_per, peaks, sm_mhz, img_bytes, sms) for k, t in per_kernel.items()}
    total_by_kind = {k: per_kernel[k] for k in per_kernel}
    dom = max(total_by_kind, key=total_by_kind.get)

    value = whole_job_rate(world, samples_step, args.steps, ms_total)
    e2e_value = whole_job_rate(world, samples_step, args.steps, ms_e2e)
    res = None
    if rank == 0:
        dr = dict(roof[dom])
        dr["kernel"] = dom
        if dr["bound"] == "hbm":
            dr["peak_source"] = f"{peaks_src} (MEASURED_PEAKS.json hbm_gbs)"
        elif dr["unit"] == "Gwarp-inst/s":
            dr["peak_source"] = "SMs x 4 schedulers x median SM clock under load (one warp instruction per cycle each)"
        else:
            dr["peak_source"] = "SMs x 128 FP32 lanes x 2 x median SM clock under load"
        dr["traffic"] = TRAFFIC_PER_LAUNCH.get(dom)
        res = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_total / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": step_config(W, world),
            "samples_per_step": samples_step,
            "fps": {m: round(1000.0 / per_kernel[f"render_{m}"], 1) for m in WL.MODES},
            "steps_per_s": round(1000.0 * args.steps / ms_total, 2),
            "per_kernel_ms": {k: round(v, 4) for k, v in per_kernel.items()},
            "roofline": dr,
            "roofline_kernels": roof,
            "e2e": {"value": round(e2e_value, 3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": round(ms_e2e / args.steps, 3),
                    "h2d_gbs": round(h2d_gbs, 1), "host_numa_node": host_node,
                    "copies_only_ms_per_step": round(ms_copies / args.steps, 3)},
            "gpu_launches": int(launches),
            "clocks": clk,
        }
        if not args.no_variants:
            res["variants"] = run_variants(shw, torch, step, W, per_kernel, samples_per, peaks)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return res, samples_per


# ncu counters of the step's kernels in the current build, per launch of the full-size step
# (one capture each, recorded under profiles/ with its command); an entry is removed when its
# kernel changes, and the JSON line then reports traffic null (or the flop roofline).
# DRAM bytes (read + write) per launch (profiles/survey_step_dram_traffic.md):
TRAFFIC_PER_LAUNCH: dict = {
    "smooth": 1386283008 + 1036524288,
    "smooth2": 2387365376 + 2102186240,
    "render_mip": 1850765056 + 19937024,
    "render_avg": 1862723328 + 16973568,
    "render_composite": 1763378944 + 17127424,
    "render_spectral": 1877628928 + 17221376,
    "render_ratio": 3900478720 + 24024064,
}
# warp instructions executed per sample of each render (same file: smsp__inst_executed.sum
# over the render's samples, 371,839,071; compositing 359,686,584):
WARP_INST_PER_SAMPLE: dict = {
    "mip": 2.322,
    "avg": 2.455,
    "composite": 3.283,
    "spectral": 2.423,
    "ratio": 3.079,
}


# --------------------------------------------------------------------------- variants

def _timeit(torch, fn, reps=5, warm=2):
    """Median CUDA-event time (ms) of one call of fn on the current stream.  Each measurement
    brackets enough back-to-back calls to last about 2 ms and divides by their number: with a
    single call between the events, the host's own time to enqueue it (argument checks, the
    tensor-map encoding) would count as GPU time while the device sits idle."""
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    fn()
    e1.record()
    torch.cuda.synchronize()
    inner = max(1, min(20, int(math.ceil(2.0 / max(e0.elapsed_time(e1), 1e-3)))))
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(inner):
            fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) / inner)
    return statistics.median(ts)


def _hbm_roof(bytes_, t_ms, hbm):
    ach = bytes_ / (t_ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s", "frac": round(ach / hbm, 4),
            "algorithmic_bytes": int(bytes_)}


def variant_moment_map(shw, torch, step, W, hbm):
    """The moment-map view (Section 2.2): orthographic down the spectral axis of the smoothed
    survey cube, one pixel per voxel column -- the plane sweep, bound by HBM."""
    dev = step.s1.device
    nvox = step.s1.numel()
    ocam = WL.survey_ortho_camera()
    mm = {}
    for m in ("mip", "avg", "spectral", "composite", "moment1"):
        kw = dict(WL.MODE_PARAMS.get(m, {}))
        o = {"rgba": torch.empty((ocam.height, ocam.width, 4), dtype=torch.float32, device=dev)}
        ns = int(shw.render(step.s1, ocam, m, lut=step.lut, step=W["step"], scalar=False, index=False, **kw)
                 ["nsamples"].sum(dtype=torch.int64).item())
        t = _timeit(torch, lambda: shw.render(step.s1, ocam, m, lut=step.lut, step=W["step"], scalar=False,
                                              index=False, nsamples=False, out=o, **kw))
        mm[m] = {"ms": round(t, 4), "gsamples_per_s": round(ns / (t * 1e-3) / 1e9, 2),
                 "roofline": _hbm_roof(4 * nvox, t, hbm)}
    return {"view": "orthographic down z, 512x512, step 0.5, trilinear; algorithmic bytes = one read of the "
                    "float32 cube per render", "modes": mm}


def variant_precision(shw, torch, step, W, per_kernel, samples_per):
    """Reduced-precision storages of the same smoothed cubes, same full-HD renders: linear
    bfloat16 / binary16 cubes (the staged marcher) and 32^3 bricks (the gather marcher).
    Speed-up against the float32 path of the step, and the image error against that float32
    render (max-abs and RMS, the scalar as a fraction of the cube's range; RGBA absolute).
    The error against the FP64 oracle is asserted by the full-size tests."""
    rng_cube = float(step.s1.max() - step.s1.min())
    out = {}
    ref = {}
    for m in WL.MODES:
        kw = dict(WL.MODE_PARAMS[m])
        lut = step.rlut if m == "ratio" else step.lut
        ref[m] = shw.render(step.vol_of(m), step.cam, m, lut=lut, step=W["step"], index=False, nsamples=False, **kw)
    for storage in ("bf16_linear", "f16_linear", "bf16", "f16"):
        v1, vp = shw.pack_bricks(step.s1, storage), shw.pack_bricks(step.pair, storage)
        per = {}
        for m in WL.MODES:
            kw = dict(WL.MODE_PARAMS[m])
            lut = step.rlut if m == "ratio" else step.lut
            vol = vp if m == "ratio" else v1
            g = shw.render(vol, step.cam, m, lut=lut, step=W["step"], index=False, nsamples=False, **kw)
            r = ref[m]
            scale = rng_cube if m != "ratio" else float(r["scalar"].max() - r["scalar"].min()) or 1.0
            es = (g["scalar"].double() - r["scalar"].double()).abs()
            er = (g["rgba"].double() - r["rgba"].double()).abs()
            o = {"rgba": g["rgba"]}
            t = _timeit(torch, lambda: shw.render(vol, step.cam, m, lut=lut, step=W["step"], scalar=False,
                                                  index=False, nsamples=False, out=o, **kw), reps=3)
            f32 = per_kernel[f"render_{m}"]
            per[m] = {"ms": round(t, 4), "fp32_ms": round(f32, 4), "speedup_vs_fp32": round(f32 / t, 3),
                      "gsamples_per_s": round(samples_per[m] / (t * 1e-3) / 1e9, 2),
                      "scalar_err_vs_fp32": {"max": float(es.max() / scale), "rms": float(es.pow(2).mean().sqrt() / scale),
                                             "p999": float(torch.quantile(es.flatten()[::16].float(), 0.999) / scale),
                                             "scale": "ratio image range" if m == "ratio" else "cube range"},
                      "rgba_err_vs_fp32": {"max": float(er.max()), "rms": float(er.pow(2).mean().sqrt())}}
            del g
        out[storage] = per
        del v1, vp
    del ref
    return {"storages": out, "note": "linear 16-bit cubes render through the staged marcher, bricks through the "
                                     "gather marcher; both hold the same rounded values"}


def best_by_brick_edge(candidates):
    """The fastest (tile, CTAs per SM, time) of each brick edge among a plan's tuned candidates
    (tile, ctas_per_sm, edge, ms); ties keep the earlier candidate, as the autotuner does."""
    best = {}
    for tile, ctas, edge, ms in candidates:
        if edge not in best or ms < best[edge][2]:
            best[edge] = (tile, ctas, ms)
    return {str(e): {"tile": t, "ctas_per_sm": c, "tune_ms": round(ms, 3)} for e, (t, c, ms) in sorted(best.items())}


def variant_batch(shw, torch, step, B):
    """2,000 sub-cubes (axes log-uniform in [32, 256]; float32 and BF16 bricks alternating; MIP and
    compositing alternating; 256x256 random views): one graph-captured persistent launch
    against one launch per sub-cube issued by the library's own loop.  Then the same
    sub-cubes all as float32, in a plan that renders them as they are and in one that rounds
    them into bfloat16 bricks of its own, the autotuner choosing the brick edge (16 or 32)
    with the tile and CTAs per SM."""
    import concurrent.futures as cf
    dev = step.s1.device
    dims = scene.batch_dims(n=B["n"], lo=B["lo"], hi=B["hi"])
    rng = np.random.default_rng(11)
    views = [(rng.uniform(0, 360), rng.uniform(-60, 60)) for _ in range(len(dims))]
    t0 = time.time()
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        cubes = list(ex.map(lambda i: scene.batch_subcube(i, tuple(int(x) for x in dims[i])), range(len(dims))))
    log(f"batch sub-cubes generated in {time.time() - t0:.1f}s")
    items, f32_items = [], []
    nvox = 0
    for i, cube in enumerate(cubes):
        d = tuple(int(x) for x in dims[i])
        ct = torch.from_numpy(cube).to(dev)
        nvox += ct.numel()
        vol = ct if i % 2 == 0 else shw.pack_bricks(ct, "bf16")
        cam = scene.orbit_camera(d, views[i][0], views[i][1], B["width"], B["height"])
        items.append((vol, cam, B["modes"][(i // 2) % 2]))
        f32_items.append((ct, cam, B["modes"][(i // 2) % 2]))
    del cubes
    plan = shw.BatchPlan(items, lut=step.lut, step=B["step"], opacity_scale=B["opacity_scale"])
    t_plan = _timeit(torch, plan.render, reps=3)
    t_loop = _timeit(torch, plan.render_one_by_one, reps=3, warm=1)
    ns = 0
    for vol, cam, mode in items:
        ns += int(shw.render(vol, cam, mode, lut=step.lut, step=B["step"], opacity_scale=B["opacity_scale"],
                             scalar=False, index=False)["nsamples"].sum(dtype=torch.int64).item())
    info = plan.info
    plan.close()
    del items
    # every sub-cube as float32, rendered as it is
    f32_plan = shw.BatchPlan(f32_items, lut=step.lut, step=B["step"], opacity_scale=B["opacity_scale"], retune=True)
    t_f32 = _timeit(torch, f32_plan.render, reps=3)
    finf = f32_plan.info
    f32_plan.close()
    # every sub-cube as float32, rounded by the plan into bfloat16 bricks of the edge it tunes
    t0 = time.time()
    own = shw.BatchPlan(f32_items, lut=step.lut, step=B["step"], opacity_scale=B["opacity_scale"], pack="bf16",
                        retune=True)
    t_create = time.time() - t0
    t_own = _timeit(torch, own.render, reps=3)
    oinf = own.info
    own.close()
    del f32_items
    by_edge = best_by_brick_edge(oinf["candidates"])
    own_bricks = {"persistent_graph_ms": round(t_own, 3), "subcubes_per_s": round(len(dims) / (t_own * 1e-3), 1),
                  "brick": oinf["brick"], "tile": oinf["tile"], "ctas_per_sm": oinf["ctas_per_sm"],
                  "packed_gb": round(oinf["packed_bytes"] / 1e9, 3), "plan_create_s": round(t_create, 2),
                  "best_by_brick_edge": by_edge, "speedup_vs_all_float32_plan": round(t_f32 / t_own, 3)}
    all_f32 = {"persistent_graph_ms": round(t_f32, 3), "subcubes_per_s": round(len(dims) / (t_f32 * 1e-3), 1),
               "tile": finf["tile"], "ctas_per_sm": finf["ctas_per_sm"]}
    return {"n": int(len(dims)), "voxels": int(nvox), "samples": ns,
            "persistent_graph_ms": round(t_plan, 3), "one_launch_per_cube_ms": round(t_loop, 3),
            "subcubes_per_s": round(len(dims) / (t_plan * 1e-3), 1),
            "subcubes_per_s_one_launch_per_cube": round(len(dims) / (t_loop * 1e-3), 1),
            "speedup": round(t_loop / t_plan, 3), "gsamples_per_s": round(ns / (t_plan * 1e-3) / 1e9, 2),
            "tile": info["tile"], "ctas_per_sm": info["ctas_per_sm"],
            "baseline": "one shw_render launch per sub-cube from the library's loop (shw_render_items)",
            "all_float32": all_f32, "own_bf16_bricks": own_bricks}


def variant_adjoint(shw, torch, step):
    """Forward with transmittance checkpoints every 64 samples and the adjoint of compositing
    (256^3 cube, 512x512 perspective)."""
    dev = step.s1.device
    D = WL.DIFF
    cube = torch.from_numpy(scene.diff_cube(dims=D["dims"])).to(dev)
    cam = scene.orbit_camera(D["dims"], D["yaw"], D["pitch"], D["width"], D["height"])
    kw = dict(lut=step.lut, step=D["step"], opacity_scale=D["opacity_scale"], ckpt_interval=D["ckpt_interval"])
    fw = shw.render(cube, cam, "composite", scalar=False, index=False, ckpt=True, **kw)
    ns = int(fw["nsamples"].sum(dtype=torch.int64).item())
    fw.pop("nsamples")
    g_rgba = torch.ones_like(fw["rgba"])
    g_vol, g_lut, g_s = torch.zeros_like(cube), torch.zeros_like(step.lut), torch.zeros(1, device=dev)
    t_fw = _timeit(torch, lambda: shw.render(cube, cam, "composite", scalar=False, index=False, nsamples=False,
                                             ckpt=True, out=fw, **kw))
    t_bw = _timeit(torch, lambda: shw.render_backward(cube, cam, g_rgba, fw["ckpt"], grad_vol=g_vol, grad_lut=g_lut,
                                                      grad_scale=g_s, **kw))
    del cube, fw, g_rgba, g_vol
    return {"workload": D["name"], "samples": ns, "forward_ms": round(t_fw, 4), "backward_ms": round(t_bw, 4),
            "forward_gsamples_per_s": round(ns / (t_fw * 1e-3) / 1e9, 2),
            "backward_gsamples_per_s": round(ns / (t_bw * 1e-3) / 1e9, 2)}


def _rotation_ms(shw, torch, vol, dims, mode, lut, width, height, pitch, nviews, kw, reps=3):
    """Median over `reps` of one full rotation's render time (nviews yaws, CUDA events) and
    the samples of one rotation."""
    cams = [scene.orbit_camera(dims, 360.0 * i / nviews, pitch, width, height) for i in range(nviews)]
    o = {"rgba": torch.empty((height, width, 4), dtype=torch.float32, device=lut.device)}
    ns = 0
    for c in cams:
        ns += int(shw.render(vol, c, mode, lut=lut, scalar=False, index=False, **kw)["nsamples"].sum(
            dtype=torch.int64).item())

    def rot():
        for c in cams:
            shw.render(vol, c, mode, lut=lut, scalar=False, index=False, nsamples=False, out=o, **kw)
    return _timeit(torch, rot, reps=reps, warm=1), ns


def variant_paper_shape(shw, torch, dev):
    """The paper's benchmark shapes (Section 6, Appendix B): U[0,1] cubes 128^3 .. 1024^3, a full
    rotation of 36 views, median of 3 rotations; MIP on canvases 500^2 .. 2000^2 (the canvas
    sweep) and compositing with k = 0.22 and a minimum threshold of 0.9 on 1000^2; and the
    stand-ins for the paper's three real cubes on 1000^2.  Frame rates here are GB300 ones;
    the paper's are OpenGL frame rates on 2013-2015 GPUs (context only)."""
    P = WL.PAPER_SHAPE
    lut = torch.from_numpy(scene.linear_lut()).to(dev)
    grid = {}
    for n in P["cubes"]:
        cube = torch.from_numpy(scene.paper_uniform_cube(n)).to(dev)
        row = {}
        for canvas in P["canvases"]:
            t, ns = _rotation_ms(shw, torch, cube, (n, n, n), "mip", lut, canvas, canvas, P["pitch"], P["views"],
                                 dict(lo=0.0, hi=1.0, step=P["step"]))
            row[f"mip_{canvas}"] = {"fps": round(1e3 * P["views"] / t, 1), "gsamples_per_s": round(ns / (t * 1e-3) / 1e9, 2)}
        t, ns = _rotation_ms(shw, torch, cube, (n, n, n), "composite", lut, 1000, 1000, P["pitch"], P["views"],
                             dict(lo=0.0, hi=1.0, step=P["step"], opacity_scale=P["opacity_scale"], filter="clip",
                                  min_threshold=P["clip"][0], max_threshold=P["clip"][1]))
        row["composite_1000"] = {"fps": round(1e3 * P["views"] / t, 1), "gsamples_per_s": round(ns / (t * 1e-3) / 1e9, 2)}
        grid[f"{n}^3"] = row
        del cube
    stand = {}
    for kind in ("ngc2903", "antennae", "gama511867"):
        c = scene.paper_standin(kind)
        dims = scene.STANDIN_DIMS[kind]
        if kind == "gama511867":
            pair = torch.stack([torch.from_numpy(c[0]), torch.from_numpy(c[1])], dim=-1).contiguous().to(dev)
            rl = torch.from_numpy(scene.ratio_lut()).to(dev)
            t, ns = _rotation_ms(shw, torch, pair, dims, "ratio", rl, 1000, 1000, P["pitch"], P["views"],
                                 dict(lo=0.0, hi=1.0, step=P["step"], ratio_floor=1.0))
            stand[kind] = {"mode": "ratio (line ratio of the two sub-cubes)", "fps": round(1e3 * P["views"] / t, 1),
                           "gsamples_per_s": round(ns / (t * 1e-3) / 1e9, 2)}
            del pair
            continue
        ct = torch.from_numpy(c).to(dev)
        r = {}
        for m in ("mip", "composite"):
            kw = dict(lo=-3.0, hi=8.0, step=P["step"])
            if m == "composite":
                kw.update(opacity_scale=0.05)
            t, ns = _rotation_ms(shw, torch, ct, dims, m, lut, 1000, 1000, P["pitch"], P["views"], kw)
            r[m] = {"fps": round(1e3 * P["views"] / t, 1), "gsamples_per_s": round(ns / (t * 1e-3) / 1e9, 2)}
        stand[kind] = r
        del ct
    return {"workload": P["name"], "rotation": f"{P['views']} views (yaw 0..350, pitch {P['pitch']}), median of 3",
            "uniform_cubes": grid, "standins_1000x1000": stand,
            "paper_context": "the paper reports up to 94 fps (MIP, 128^3, 1000^2, GTX TITAN X) and about 2 fps "
                             "for 1024^3 on a GT 750M / GRID K1 (OpenGL; not measured here)"}


def run_variants(shw, torch, step, W, per_kernel, samples_per, peaks):
    """The method's variants on the same GPU, reported beside the headline step: the moment-map
    view (the HBM-bound sweep), the reduced-precision storages against float32, the batched
    persistent launch against one launch per sub-cube, the adjoint, the paper's benchmark
    shapes and the in-ray smoothing kernels."""
    dev = step.s1.device
    hbm = float(peaks["hbm_gbs"])
    res = {}
    for name, fn in (("moment_map", lambda: variant_moment_map(shw, torch, step, W, hbm)),
                     ("precision", lambda: variant_precision(shw, torch, step, W, per_kernel, samples_per)),
                     ("batch", lambda: variant_batch(shw, torch, step, WL.BATCH)),
                     ("adjoint", lambda: variant_adjoint(shw, torch, step)),
                     ("paper_shape", lambda: variant_paper_shape(shw, torch, dev)),
                     ("in_ray_smoothing", lambda: run_in_ray_smoothing(shw, torch, dev))):
        t = time.time()
        res[name] = fn()
        shw.sync_status()
        torch.cuda.empty_cache()
        log(f"variant {name}: {time.time() - t:.1f}s")
    return res


def run_in_ray_smoothing(shw, torch, dev):
    """In-ray smoothing (Algorithms 8-9) on the paper's benchmark shape: frame time and
    fetch rate of MIP and clipped compositing for raw sampling, the N-box filters and the
    N-tap Gaussians (the 9-tap is Algorithm 9's printed kernel), median over the views."""
    P = WL.PAPER_SMOOTH
    n = P["n"]
    cube = torch.from_numpy(scene.paper_uniform_cube(n)).to(dev)
    lut = torch.from_numpy(scene.linear_lut()).to(dev)
    kernels = [("raw", {}, 1)]
    kernels += [(f"box{2 * a + 1}", dict(smooth="box", smooth_arm=a), 2 * a + 1) for a in P["box_arms"]]
    for N in P["gauss_taps"]:
        taps = shw.binomial_taps(9, drop=2) if N == 9 else shw.binomial_taps(N)
        kernels.append((f"gauss{N}", dict(smooth="taps", smooth_taps=taps), 1 + 6 * len(taps[1])))
    modes = {"mip": dict(lo=P["lo"], hi=P["hi"]),
             "composite": dict(lo=P["lo"], hi=P["hi"], opacity_scale=P["opacity_scale"], filter="clip",
                               min_threshold=P["clip"][0], max_threshold=P["clip"][1])}
    out = {}
    for m, mkw in modes.items():
        rows = {}
        for name, skw, fetches in kernels:
            ts, ss = [], []
            for yaw in P["yaws"]:
                cam = scene.orbit_camera((n, n, n), yaw, P["pitch"], P["width"], P["height"])
                o = shw.render(cube, cam, m, lut=lut, step=P["step"], scalar=False, index=False, **mkw, **skw)
                ss.append(int(o["nsamples"].sum(dtype=torch.int64).item()))
                o = {"rgba": o["rgba"]}
                ts.append(_timeit(torch, lambda: shw.render(cube, cam, m, lut=lut, step=P["step"], scalar=False,
                                                            index=False, nsamples=False, out=o, **mkw, **skw),
                                  reps=3, warm=1))
            k = int(np.argsort(ts)[len(ts) // 2])
            t, ns = ts[k], ss[k]
            rows[name] = {"fetches_per_step": fetches, "ms": round(t, 3), "fps": round(1e3 / t, 1),
                          "gsamples_per_s": round(ns / (t * 1e-3) / 1e9, 2),
                          "gfetches_per_s": round(fetches * ns / (t * 1e-3) / 1e9, 1)}
            if name.startswith("box") and P["step"] in (0.5, 1.0):
                rows[name]["note"] = "lattice running sums: about 2 fetches per step done"
        out[m] = rows
    del cube
    return {"workload": P["name"], "views": f"yaw {list(P['yaws'])}, pitch {P['pitch']}; median view",
            "fetches": "fetches_per_step is Section 6's count for the kernel (N for an N-box, "
                       "3(N-1)/2+1 for an N-tap Gaussian); gfetches_per_s counts those",
            "compositing": f"opacity scale {P['opacity_scale']}, clip [{P['clip'][0]}, {P['clip'][1]}]",
            "modes": out}


# --------------------------------------------------------------------------- oracle (CPU) arm

def oracle_sample(budget_s: float, samples_per_frame=None):
    """Time the FP64 oracle on a bounded sample of the survey step on the host cores.

    Sample: a random subset of pixels of each of the five renders (on the raw cubes; the
    oracle's cost per sample does not depend on the values) and the smoothing of a
    z-slab of both cubes; each part is scaled to the full step by its share of the work.
    Returns (Gsamples/s of the whole step, description, cores)."""
    import oracle
    cube, cube2 = make_inputs()
    cubed, cube2d = cube.astype(np.float64), cube2.astype(np.float64)
    cam = WL.survey_camera()
    npix = cam.width * cam.height
    tot, per_ray = oracle.count_samples(WL.SURVEY["dims"], cam, step=WL.SURVEY["step"])
    rng = np.random.default_rng(0)
    # calibrate: a small pixel subset first
    frac = 1.0 / 4096
    t_render = 0.0
    for it in range(3):
        npx = max(64, int(npix * frac))
        pix = rng.choice(npix, size=npx, replace=False)
        t = time.time()
        for m in WL.MODES:
            kw = dict(WL.MODE_PARAMS[m])
            lut = scene.ratio_lut() if m == "ratio" else scene.linear_lut()
            oracle.render(cubed, cam, m, lut=lut, cube2=cube2d if m == "ratio" else None, pixels=pix,
                          step=WL.SURVEY["step"], **kw)
        dt = time.time() - t
        t_render = dt / frac
        if dt > 0.5 * budget_s or it == 2:
            break
        frac = min(0.25, frac * max(2.0, 0.6 * budget_s / max(dt, 1e-3)))
    nz_s = 16
    t = time.time()
    w = oracle.gauss_weights(WL.SURVEY["sigma"], WL.SURVEY["radius"])
    oracle.smooth(cubed[:nz_s], w)
    oracle.smooth(cube2d[:nz_s], w)
    t_smooth = (time.time() - t) * cube.shape[0] / nz_s
    samples_step = 5 * tot if samples_per_frame is None else sum(samples_per_frame.values())
    step_s = t_render + t_smooth
    desc = (f"FP64 oracle: {npx} random pixels of each of the 5 renders ({frac:.2e} of 1920x1080) and "
            f"the smoothing of {nz_s} of 1024 z-planes of both cubes, each scaled to the full step")
    return samples_step / step_s / 1e9, desc, step_s


def omp_cores():
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n else os.cpu_count()


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    vals = []
    desc = ""
    for _ in range(args.warmup):
        pass  # the oracle has no warm-up state; every step is timed the same way
    for k in range(args.steps):
        v, desc, _ = oracle_sample(budget_s=max(2.0, 60.0 / max(args.steps, 1)))
        vals.append(v)
    v = statistics.median(vals)
    cores = omp_cores()
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(v, 6), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": step_config(WL.SURVEY, world),
        "cpu_baseline": {"value": round(v, 6), "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": round(v, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_case(args):
    """One small case of one kernel family, for profiler captures: prints one JSON line with its
    median time and units (samples or voxels), not the benchmark's line."""
    import torch
    import paper_1707_00442_gb300 as shw
    from scene.camera import ortho_axis_camera
    nx, ny, nz = (int(v) for v in args.dims.split(","))
    cube = torch.from_numpy(scene.survey_cube(dims=(nx, ny, nz), n_sources=50)).cuda()
    lut = torch.from_numpy(scene.linear_lut()).cuda()
    if args.case == "smooth":
        out = torch.empty_like(cube)
        fn = lambda: shw.smooth(cube, WL.SURVEY["sigma"], WL.SURVEY["radius"], out=out)  # noqa: E731
    elif args.case == "smooth-zip":
        first = torch.from_numpy(scene.ratio_cube(cube.cpu().numpy())).cuda()
        out = torch.empty(tuple(cube.shape) + (2,), dtype=torch.float32, device="cuda")
        fn = lambda: shw.smooth_zip(cube, first, WL.SURVEY["sigma"], WL.SURVEY["radius"], out=out)  # noqa: E731
    elif args.case == "in-ray-smoothing":
        print(json.dumps(run_in_ray_smoothing(shw, torch, "cuda")), flush=True)
        shw.sync_status()
        return
    else:
        cam = ortho_axis_camera((nx, ny, nz), nx, ny) if args.case == "moment-map" else \
            scene.orbit_camera((nx, ny, nz), 30.0, 20.0, 960, 540)
        o = {"rgba": torch.empty((cam.height, cam.width, 4), device="cuda")}
        kw = dict(WL.MODE_PARAMS[args.mode])
        if args.smooth.startswith("box"):
            kw.update(smooth="box", smooth_arm=(int(args.smooth[3:]) - 1) // 2)
        elif args.smooth.startswith("gauss"):
            n = int(args.smooth[5:])
            kw.update(smooth="taps", smooth_taps=shw.binomial_taps(9, drop=2) if n == 9 else shw.binomial_taps(n))
        vol = cube
        if args.mode in ("ratio", "ratio_mip"):  # the survey step's form: the pair storage
            vol = torch.stack([cube, torch.from_numpy(scene.ratio_cube(cube.cpu().numpy())).cuda()], dim=-1)
            lut = torch.from_numpy(scene.ratio_lut()).cuda()
        fn = lambda: shw.render(vol, cam, args.mode, lut=lut, scalar=False, index=False,  # noqa: E731
                                nsamples=False, out=o, **kw)
        units = int(shw.render(vol, cam, args.mode, lut=lut, scalar=False, index=False, **kw)["nsamples"].sum(
            dtype=torch.int64).item())
    t = _timeit(torch, fn, reps=args.steps, warm=args.warmup)
    shw.sync_status()
    if args.case in ("smooth", "smooth-zip"):
        units = cube.numel()
    print(json.dumps({"case": args.case, "mode": args.mode, "dims": args.dims, "smooth": args.smooth,
                      "ms": round(t, 4), "units": units,
                      "unit": "voxels" if args.case.startswith("smooth") else "samples"}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the variant legs (moment-map view, 16-bit storages, batch, adjoint, paper shapes, "
                         "in-ray smoothing)")
    ap.add_argument("--workload", default="survey", choices=sorted(WORKLOADS),
                    help="survey: the headline workload; survey-small: the same step on a smaller cube "
                         "(profiler captures)")
    ap.add_argument("--case", choices=["moment-map", "render", "smooth", "smooth-zip", "in-ray-smoothing"],
                    help="run one small case of one kernel family for a profiler capture, then exit")
    ap.add_argument("--dims", default="384,384,768", help="--case: cube dims nx,ny,nz")
    ap.add_argument("--mode", default="mip", help="--case: transfer function")
    ap.add_argument("--smooth", default="raw", help="--case render: in-ray smoothing raw, boxN or gaussN")
    args = ap.parse_args()
    if args.case:
        run_case(args)
        return
    if args.warmup < 3 and args.impl == "ours":
        log("warning: fewer than 3 warm-up steps")
    if args.impl == "reference":
        run_reference(args)
        return
    res, samples_per = run_ours(args)
    if res is None:
        return
    if res["n_gpus"] == 1 and not args.no_cpu_baseline and args.workload == "survey":
        v, desc, _ = oracle_sample(budget_s=15.0, samples_per_frame=samples_per)
        res["cpu_baseline"] = {"value": round(v, 6), "unit": UNIT, "cores": omp_cores(), "kind": "oracle",
                               "sample": desc}
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
