"""Helpers shared by the GPU tests: run the CUDA path and the oracle on one seeded scene and
compare them with the ambiguity-aware bound."""
import numpy as np
import torch

import oracle
import paper_2602_07860_gb300 as mbr

ORACLE_MODE = {"plain": "exact", "fast": "fast"}
TOL = 1e-4  # absolute, intensities in [0, 1]


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
