"""Helpers shared by the GPU tests: run the CUDA path and the oracle on one seeded scene and
compare them with the ambiguity-aware bound."""
import numpy as np
import torch

import oracle
import paper_2602_07860_gb300 as mbr
import scenes

ORACLE_MODE = {"plain": "exact", "fast": "fast"}
TOL = 1e-4  # absolute, intensities in [0, 1]


def degenerate_scene():
    """A rotating sphere plus three degenerate faces: a repeated vertex and three collinear
    vertices (both zero area), and a duplicate of face 5 (exact depth ties)."""
    sc = scenes.small_scene("rotate", subdiv=3, T=8, H=40, W=52)
    v, f, a = sc["verts"], sc["faces"], sc["albedo"]
    mid = 0.5 * (v[f[0, 0]] + v[f[0, 1]])  # a vertex on the first face's first edge
    m = len(v)
    extra = np.array([[f[0, 0], f[0, 0], f[0, 1]],
                      [f[0, 0], m, f[0, 1]],
                      f[5]], dtype=np.int32)
    return dict(sc, verts=np.vstack([v, mid[None, :]]), albedo=np.vstack([a, a[:1]]),
                faces=np.vstack([f, extra]).astype(np.int32))


def gpu_inputs(sc):
    v, f, a = mbr.mesh_tensors(sc)
    return v, f, a, mbr.motion_from_dict(sc["motion"]), mbr.camera_from_dict(sc["camera"])


def gpu_render(ctx, sc, solver):
    v, f, a, mo, ca = gpu_inputs(sc)
    img = ctx.render_blur(v, f, a, mo, ca, sc["T"], sc["H"], sc["W"], solver)
    torch.cuda.synchronize()
    return img.cpu().double().numpy()


def compare_images(gpu, orc, ambig, T):
    """Per-pixel bound: |gpu - oracle| <= TOL + (ambiguous samples at the pixel) / T per channel
    (a sample whose FP32 decision may legitimately differ changes the pixel by at most 1/T).
    Returns (max error on unambiguous pixels, fraction of ambiguous pixels, max excess over the
    bound)."""
    n_amb = ((ambig & oracle.AMB_IMAGE) != 0).sum(0)  # [h, w]
    err = np.abs(gpu - orc).max(-1)
    bound = TOL + n_amb / T
    clean = n_amb == 0
    max_clean = float(err[clean].max()) if clean.any() else 0.0
    excess = float((err - bound).max())
    return max_clean, float((~clean).mean()), excess
