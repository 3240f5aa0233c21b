"""Upload of a seeded ``Scene`` into a library context (test and benchmark
helper).  It only marshals the scene's arrays through the library's calls:
template, camera, embedded graph on the device, weights, iteration counts,
frame and, for body scenes, the skeleton and the frame's start pose."""
from __future__ import annotations

import numpy as np

from .scenes import SKELETON_SITES


def setup_scene(ctx, scene, with_frame: bool = True):
    """Upload ``scene`` into the context ``ctx`` (a ``Context`` of the library
    binding)."""
    wp, ws, wa = scene.weights
    _, _, wsm, wed, wv, wac = scene.surface_weights
    ctx.set_params(w_photo=wp, w_sil=ws, w_arap=wa, n_gn=scene.n_gn, n_pcg=scene.n_pcg,
                   n_gn_pose=scene.n_gn_pose, w_smooth=wsm, w_edge=wed, w_velocity=wv, w_acceleration=wac,
                   n_gn_surface=scene.n_gn_surface, n_pcg_surface=scene.n_pcg_surface)
    ctx.set_camera(scene.cam.f, scene.cam.cx, scene.cam.cy, scene.cam.W, scene.cam.H)
    ctx.upload_template(scene.V, scene.F, scene.albedo, scene.material)
    ctx.build_graph(scene.n_nodes, scene.K)
    if scene.skeleton is not None:
        sk = scene.skeleton
        dof = np.ones(len(sk["parents"]), np.uint8)
        dof[SKELETON_SITES] = 0
        ctx.upload_skeleton(sk["parents"], sk["joints_rest"], dof, sk["skin_idx"], sk["skin_w"])
        ctx.set_pose(scene.pose_init)
    if with_frame:
        ctx.upload_frame(scene.rgb, scene.dt, scene.mask.astype(np.uint8), scene.joints2d, scene.joints3d)
