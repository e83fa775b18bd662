"""Rotational recovery through an SDF (Sec. 5, rotation task) on the GPU: the field starts as the
paper's inclined ellipsoid, every iteration extracts a mesh (mbr_sdf_extract), renders five
rotation-blurred views with the fast solver and back-propagates Eq. loss-img plus the SDF
regularisers through the renderer and the extraction to the grid.  A short run must cut the
image loss and bring the extracted surface closer to the target's."""
import numpy as np
import pytest
import torch

import scenes

pytestmark = pytest.mark.gpu


def test_sdf_recovery_moves_towards_the_target():
    import paper_2602_07860_gb300 as mbr
    from paper_2602_07860_gb300.sdf import ellipsoid_sdf, extract_mesh, recover_rotational
    views_sc = scenes.config_sdf_rotation(T=12, H=64, W=64)
    ctx = mbr.Context()
    v, f, a = mbr.mesh_tensors(views_sc[0])
    views, targets = [], []
    for s in views_sc:
        mo, ca = mbr.motion_from_dict(s["motion"]), mbr.camera_from_dict(s["camera"])
        views.append((mo, ca))
        targets.append(ctx.render_blur(v, f, a, mo, ca, s["T"], s["H"], s["W"], "fast").clone())
    n, lo = 24, (-1.1, -1.1, -1.1)
    h = 2.2 / n
    s0 = ellipsoid_sdf(n, lo, h)

    def surface_gap(sdf):
        verts, _ = extract_mesh(sdf, lo, h, ctx)
        return float(torch.cdist(verts.detach(), v).min(dim=1).values.mean())

    gap0 = surface_gap(s0)
    sdf, hist = recover_rotational(s0, lo, h, views, torch.stack(targets), 12, 64, 64, iters=60, lr=4e-3)
    gap1 = surface_gap(sdf)
    assert all(np.isfinite(x[1]) for x in hist)
    assert hist[-1][0] < 0.6 * hist[0][0], (hist[0], hist[-1])
    assert gap1 < 0.8 * gap0, (gap0, gap1)
