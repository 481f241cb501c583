"""Seeded synthetic inputs shaped like laparoscopy video (no method arithmetic here).

This package draws the workloads that both the CUDA path and the FP64 oracle are run
on: a procedural texture, a ground-truth deformation (a similarity plus Gaussian
displacement bumps), rendered frames, feature matches with noise and outliers, and the
canvas window a frame covers. It contains none of the EMDQ arithmetic (no dual
quaternions, no Gaussian blending, no EM, no bilinear sampling, no blending): frames are
rendered by evaluating an analytic texture at the exact inverse ground-truth position.
"""
from .scene import (  # noqa: F401
    Scene,
    make_scene,
    gt_forward,
    gt_inverse,
    pan_frames,
    texture,
    render_reference,
    render_frame,
    make_matches,
    make_pair_matches,
    footprint_window,
    canvas_origin,
    workload,
    WORKLOADS,
    mixed_pairs,
    MIXED_SIZES,
)
