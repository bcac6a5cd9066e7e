"""Named workloads: the input recipes (cube, camera, per-mode parameters) shared by the
parity tests, the smoke check and the benchmark.  Inputs only; no method arithmetic."""
from __future__ import annotations

# per-mode render parameters (colour-map domain [lo, hi] in noise-sigma units)
MODE_PARAMS = {
    "mip": dict(lo=-3.0, hi=8.0),
    "avg": dict(lo=-3.0, hi=8.0),
    "composite": dict(lo=-3.0, hi=8.0, opacity_scale=0.01, term_alpha=0.99),
    "spectral": dict(lo=-3.0, hi=8.0),
    "ratio": dict(lo=0.0, hi=1.0, ratio_floor=1.0),
}
MODES = ["mip", "avg", "composite", "spectral", "ratio"]

TINY = dict(name="tiny-64^3-ortho-z-128^2", dims=(64, 64, 64), view="ortho-z", width=128, height=128, step=0.5,
            sigma=1.0, radius=3, opacity_scale=0.05)

SURVEY = dict(name="survey-512x512x1024-persp-1920x1080", dims=(512, 512, 1024), yaw=30.0, pitch=20.0, fov=45.0,
              width=1920, height=1080, step=0.5, sigma=2.0, radius=6, interp="trilinear")

# the same step on a smaller cube (still larger than the 129 MB L2), for profiler captures
SURVEY_SMALL = dict(SURVEY, name="survey-small-384x384x512-persp-960x540", dims=(384, 384, 512), width=960,
                    height=540, n_sources=100)
SURVEY.setdefault("n_sources", 200)

# the moment-map view of the survey cube: parallel rays down the spectral axis
SURVEY_ORTHO_Z = dict(name="survey-512x512x1024-ortho-z-512^2", width=512, height=512, step=0.5)

# the paper's smoothing benchmark (Section 6, Appendix B) in shape: a U[0,1] cube, a
# 1000x1000 canvas, MIP and compositing, per-step fetch counts from raw to the 13-tap kernel
PAPER_SMOOTH = dict(name="paper-smoothing-512^3-U01-persp-1000^2", n=512, width=1000, height=1000, step=0.5,
                    yaws=(0.0, 120.0, 240.0), pitch=20.0, lo=0.0, hi=1.0, opacity_scale=0.22,
                    clip=(0.9, 1.0), box_arms=(1, 2, 3, 4), gauss_taps=(5, 9, 13))

# the paper's benchmark shapes (Section 6, Appendix B): U[0,1] cubes, a full rotation of views,
# MIP over a sweep of canvas sizes and compositing with k = 0.22 and a 0.9 minimum threshold
PAPER_SHAPE = dict(name="paper-shape-U01-128..1024^3-rotation36", cubes=(128, 256, 512, 1024),
                   canvases=(500, 1000, 1500, 2000), views=36, pitch=20.0, step=0.5, opacity_scale=0.22,
                   clip=(0.9, 1.0))

DIFF = dict(name="diff-256^3-persp-512^2", dims=(256, 256, 256), yaw=30.0, pitch=20.0, width=512, height=512,
            step=0.5, opacity_scale=0.02, target_scale=1.2, lut_sigma=0.05, ckpt_interval=64)

BATCH = dict(name="batch-2000-subcubes-256^2", n=2000, lo=32, hi=256, width=256, height=256, step=0.5,
             modes=("mip", "composite"), opacity_scale=0.02)


def survey_camera(width=None, height=None, w=None):
    from .camera import orbit_camera
    w = SURVEY if w is None else w
    return orbit_camera(w["dims"], w["yaw"], w["pitch"], width or w["width"], height or w["height"], fov_deg=w["fov"])


def survey_ortho_camera():
    from .camera import ortho_axis_camera
    return ortho_axis_camera(SURVEY["dims"], SURVEY_ORTHO_Z["width"], SURVEY_ORTHO_Z["height"])
