"""Rotational shape recovery through a signed distance field (Sec. 5, rotation task).

Optimising mesh vertices directly rarely recovers a fast-rotating object, so the paper optimises
an SDF field instead: every iteration extracts a mesh from the field differentiably, renders its
motion-blurred views with the fast solver, and back-propagates the image loss through the
renderer and the extraction to the field's samples, with the SDF regularisers of its loss-term
appendix.  The extraction runs in the library (mbr_sdf_extract: marching tetrahedra on the
regular grid, in place of the paper's FlexiCubes); the regularisers are plain PyTorch on the grid
(they are not part of the renderer):

  Eikonal     mean over interior samples of | |grad s| - 1 |, central differences;
  singular H  mean over samples near the surface (|s| < 2h) of |det Hessian(s)|, differences;
  sign        over grid edges whose samples differ in sign, the cross-entropy of sigmoid(s_a)
              against the side of s_b, both ways (discourages spurious surfaces);
  deviation   (FlexiCubes' spread of a deformable grid vertex's neighbour distances) is constant
              on this fixed grid and left out.
"""
from __future__ import annotations

import math

import torch
import torch.nn.functional as Fnn

from .render import Context, render_blur


class _SdfMesh(torch.autograd.Function):
    """verts = extract(sdf); faces and the vertices' grid edges ride along (no gradient)."""

    @staticmethod
    def forward(ctx, sdf, lo, h, rctx):
        v, f, e = rctx.sdf_extract(sdf.detach().contiguous(), lo, h)
        ctx.save_for_backward(sdf, e)
        ctx.h, ctx.rctx = h, rctx
        ctx.mark_non_differentiable(f)
        return v, f

    @staticmethod
    def backward(ctx, g_verts, g_faces):
        sdf, e = ctx.saved_tensors
        if g_verts is None or e.shape[0] == 0:
            return torch.zeros_like(sdf), None, None, None
        return ctx.rctx.sdf_extract_backward(sdf.detach().contiguous(), ctx.h, e, g_verts.contiguous()), None, None, None


def extract_mesh(sdf, lo, h, rctx=None):
    """(verts [V,3] differentiable w.r.t. sdf, faces [F,3] int32) of the zero level set of the
    grid ``sdf`` [(n+1)]^3 (indexed [z, y, x]) sampled at lo + h (i, j, k)."""
    return _SdfMesh.apply(sdf, lo, h, rctx if rctx is not None else Context())


def grid_points(n, lo, h, device="cuda", dtype=torch.float32):
    """[(n+1), (n+1), (n+1), 3] sample positions (x, y, z), indexed [k, j, i] like the grid."""
    ax = [lo[q] + h * torch.arange(n + 1, device=device, dtype=dtype) for q in range(3)]
    Z, Y, X = torch.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return torch.stack([X, Y, Z], -1)


def ellipsoid_sdf(n, lo, h, device="cuda"):
    """The paper's initial shape, the inclined ellipsoid 4x^2 + 2.5y^2 + 2.5z^2 - 3yz = 1, as a
    first-order signed distance (q - 1) / |grad q| (App. hyperparameters: the field is pretrained on
    it; a grid can take the distance directly)."""
    P = grid_points(n, lo, h, device)
    x, y, z = P[..., 0], P[..., 1], P[..., 2]
    q = 4 * x * x + 2.5 * y * y + 2.5 * z * z - 3 * y * z
    g = torch.stack([8 * x, 5 * y - 3 * z, 5 * z - 3 * y], -1)
    return ((q - 1.0) / g.norm(dim=-1).clamp_min(1e-3)).contiguous()


def eikonal_loss(s, h):
    gx = (s[1:-1, 1:-1, 2:] - s[1:-1, 1:-1, :-2]) / (2 * h)
    gy = (s[1:-1, 2:, 1:-1] - s[1:-1, :-2, 1:-1]) / (2 * h)
    gz = (s[2:, 1:-1, 1:-1] - s[:-2, 1:-1, 1:-1]) / (2 * h)
    return (torch.sqrt(gx * gx + gy * gy + gz * gz + 1e-12) - 1.0).abs().mean()


def singular_hessian_loss(s, h, band=2.0):
    c = s[1:-1, 1:-1, 1:-1]

    def d2(a, b):
        return (a - 2 * c + b) / (h * h)

    hxx = d2(s[1:-1, 1:-1, 2:], s[1:-1, 1:-1, :-2])
    hyy = d2(s[1:-1, 2:, 1:-1], s[1:-1, :-2, 1:-1])
    hzz = d2(s[2:, 1:-1, 1:-1], s[:-2, 1:-1, 1:-1])

    def mixed(t):
        return t / (4 * h * h)

    hxy = mixed(s[1:-1, 2:, 2:] - s[1:-1, 2:, :-2] - s[1:-1, :-2, 2:] + s[1:-1, :-2, :-2])
    hxz = mixed(s[2:, 1:-1, 2:] - s[2:, 1:-1, :-2] - s[:-2, 1:-1, 2:] + s[:-2, 1:-1, :-2])
    hyz = mixed(s[2:, 2:, 1:-1] - s[2:, :-2, 1:-1] - s[:-2, 2:, 1:-1] + s[:-2, :-2, 1:-1])
    det = hxx * (hyy * hzz - hyz * hyz) - hxy * (hxy * hzz - hyz * hxz) + hxz * (hxy * hyz - hyy * hxz)
    near = (c.abs() < band * h).detach()
    return det.abs()[near].mean() if near.any() else s.sum() * 0.0


def sign_loss(s):
    total = s.sum() * 0.0
    for a, b in ((s[:, :, :-1], s[:, :, 1:]), (s[:, :-1, :], s[:, 1:, :]), (s[:-1], s[1:])):
        m = (a > 0) != (b > 0)
        if m.any():
            total = total + Fnn.binary_cross_entropy_with_logits(a[m], (b[m] > 0).to(s.dtype), reduction="sum") + \
                Fnn.binary_cross_entropy_with_logits(b[m], (a[m] > 0).to(s.dtype), reduction="sum")
    return total


def recover_rotational(sdf0, lo, h, views, targets, T, H, W, iters=1000, lr=5e-4, betas=(0.9, 0.999),
                       lam_crit=3e-3, lam_reg=1.0, lam_eik=50.0 / 53.0, lam_sh=3.0 / 53.0, lam_sign=1e-2,
                       grey=0.7, solver="fast", log_every=0, on_iter=None):
    """Adam on the SDF grid ``sdf0`` so that the blurred renders of its extracted mesh under
    ``views`` (list of (Motion, Camera)) match ``targets`` [n, H, W, 4] (grey objects).  Loss per
    iteration: Eq. loss-img (L1 of colour and alpha, summed over pixels, averaged over the views)
    + lam_crit (lam_eik Eikonal + lam_sh singular Hessian) + lam_reg lam_sign sign loss.  Returns
    (sdf, history of (image loss, total loss, faces))."""
    s = sdf0.detach().clone().contiguous().requires_grad_(True)
    opt = torch.optim.Adam([s], lr=lr, betas=betas)
    rctx = Context()
    hist = []
    for it in range(iters):
        opt.zero_grad(set_to_none=False)
        verts, faces = extract_mesh(s, lo, h, rctx)
        if faces.shape[0] == 0:
            raise RuntimeError("the SDF has no zero crossing")
        alb = torch.full_like(verts, grey)
        img_loss = 0.0
        for (mo, ca), tgt in zip(views, targets):
            img = render_blur(verts, alb, faces, mo, ca, T, H, W, solver, rctx)
            img_loss = img_loss + (img - tgt).abs().sum()
        img_loss = img_loss / len(views)
        loss = img_loss + lam_crit * (lam_eik * eikonal_loss(s, h) + lam_sh * singular_hessian_loss(s, h)) + \
            lam_reg * lam_sign * sign_loss(s)
        if on_iter is not None:
            on_iter(it, verts.detach(), faces, float(img_loss))
        loss.backward()
        opt.step()
        hist.append((float(img_loss), float(loss), int(faces.shape[0])))
        if log_every and it % log_every == 0:
            print(f"iter {it}: image loss {hist[-1][0]:.2f}, total {hist[-1][1]:.2f}, faces {hist[-1][2]}", flush=True)
    return s.detach(), hist
