"""Seeded synthetic inputs for the LiveCap non-rigid and pose solvers.

This package is the one piece of code that both the CUDA path (through its
tests and ``bench.py``) and the FP64 oracle consume.  It builds scenes — the
template mesh, albedo, material weights, skeleton, a ground-truth deformation,
the rendered target frame with its silhouette distance transform and noisy
joint detections — and nothing else.  It holds none of the solver's
arithmetic: no embedded graph, no node binding, no visibility keys, no
residuals, Jacobians or linear solves.  Its renderer and ground-truth
deformation are deliberately built differently from anything the solver does
(FP64 floating-point coverage, Gaussian-RBF control points), so that a target
frame is an independent input and never a copy of a solver intermediate.
"""
from .scenes import (  # noqa: F401
    Camera,
    Scene,
    capsule_mesh,
    body_template,
    value_noise_albedo,
    half_split_material,
    smooth_deformation,
    rbf_field,
    rbf_field_linear,
    ar1_draws,
    ar1_sequence,
    ar1_frame,
    stream_frame,
    render_frame,
    render,
    contour_distance_transform,
    make_scene,
    make_batch,
    make_batch_member,
    batch_specs,
    SKELETON_PARENTS,
    SKELETON_NAMES,
    N_POSE_DOF,
)
from .upload import setup_scene  # noqa: F401
