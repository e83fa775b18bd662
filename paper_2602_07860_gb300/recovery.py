"""Shape recovery from motion-blurred views (Sec. 5): optimise mesh vertices (and colours) so that
their blurred renders match target images, with Adam.  ``recover_shape`` uses an L2 image loss and
uniform-Laplacian smoothing; ``recover_translational`` the paper's loss of Eq. loss-img (L1 on
colour and transparency, the smoothness and Laplacian terms of the loss-term appendix) with its
translational settings (views sampled in batches, Adam (0.01, 0.5, 0.99)).

The renders of all views of one iteration go through ``ViewBatch``: one batched, graph-captured
library call for the forward and one for the adjoint (include/mbr.h, mbr_render_blur_batch).  The
output and gradient buffers persist across iterations and Adam updates the vertex tensor in place,
so every iteration after the first replays the captured graphs.  The loss terms are plain PyTorch
(they are not part of the renderer).
"""
from __future__ import annotations

import torch

from .render import Context


class ViewBatch:
    """Blurred renders of one mesh under several (motion, camera) views, [n, H, W, 4], with the
    adjoint summed over views.  ``verts`` must keep its storage (optimisers update in place)."""

    def __init__(self, verts, faces, albedo, views, T, H, W, solver="fast"):
        self.verts, self.faces, self.albedo = verts, faces, albedo
        self.views, self.T, self.H, self.W, self.solver = list(views), T, H, W, solver
        n, dev = len(self.views), verts.device
        self.images = torch.zeros((n, H, W, 4), dtype=torch.float32, device=dev)
        self.dl_dimage = torch.zeros_like(self.images)
        self.images_bwd = torch.zeros_like(self.images)
        self.dl_dverts = torch.zeros((n,) + tuple(verts.shape), dtype=torch.float32, device=dev)
        self.dl_dalbedo = torch.zeros((n,) + tuple(albedo.shape), dtype=torch.float32, device=dev)
        # one context per direction: each keeps its own captured batch plan
        self.ctx_fwd, self.ctx_bwd = Context(), Context()

    def _items(self, backward):
        items = []
        for i, (motion, camera) in enumerate(self.views):
            it = dict(verts=self.verts, faces=self.faces, albedo=self.albedo, motion=motion, camera=camera,
                      T=self.T, H=self.H, W=self.W, solver=self.solver,
                      image=(self.images_bwd if backward else self.images)[i])
            if backward:
                it.update(dl_dimage=self.dl_dimage[i], dl_dverts=self.dl_dverts[i], dl_dalbedo=self.dl_dalbedo[i])
            items.append(it)
        return items

    def forward(self):
        self.ctx_fwd.render_batch(self._items(False), False)
        return self.images

    def backward(self, grad_images):
        self.dl_dimage.copy_(grad_images)
        self.ctx_bwd.render_batch(self._items(True), True)
        return self.dl_dverts.sum(0), self.dl_dalbedo.sum(0)

    def render(self):
        """Differentiable [n, H, W, 4] renders of the current ``verts`` (and ``albedo``)."""
        return _ViewBatchFn.apply(self.verts, self.albedo, self)


class _ViewBatchFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, verts, albedo, vb):
        ctx.vb = vb
        return vb.forward().clone()

    @staticmethod
    def backward(ctx, g):
        gv, ga = ctx.vb.backward(g.contiguous())
        return gv, ga, None


def edge_index(faces, V):
    """Undirected edges of a triangle mesh as a [2, E] index (both directions)."""
    f = faces.long()
    e = torch.cat([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]], 0)
    e = torch.cat([e, e.flip(1)], 0)
    key = torch.unique(e[:, 0] * V + e[:, 1])
    return torch.stack([key // V, key % V])


def laplacian_loss(verts, edges):
    """Uniform Laplacian smoothing: mean over vertices of |v_i - mean of its neighbours|^2."""
    V = verts.shape[0]
    deg = torch.zeros(V, device=verts.device, dtype=verts.dtype).index_add_(0, edges[0], torch.ones_like(edges[0], dtype=verts.dtype))
    nb = torch.zeros_like(verts).index_add_(0, edges[0], verts[edges[1]])
    lap = verts - nb / deg.clamp_min(1.0)[:, None]
    return (lap * lap).sum(1).mean()


def recover_shape(template, faces, albedo, views, targets, T, H, W, iters=500, lr=1e-3, lap_weight=0.1,
                  solver="fast", log_every=0, on_iter=None):
    """Adam on the vertices of ``template`` [V,3] so that their blurred renders under ``views``
    (list of (Motion, Camera)) match ``targets`` [n, H, W, 4].  Loss = mean squared RGBA error
    summed over views + lap_weight x Laplacian term.  ``on_iter(it, verts, image_loss)``, if
    given, sees the vertices each iteration renders (before its Adam step).  Returns (vertices,
    loss history)."""
    v = template.detach().clone().contiguous().requires_grad_(True)
    vb = ViewBatch(v, faces, albedo, views, T, H, W, solver)
    edges = edge_index(faces, v.shape[0])
    opt = torch.optim.Adam([v], lr=lr)
    hist = []
    for it in range(iters):
        opt.zero_grad(set_to_none=False)
        imgs = vb.render()
        img_loss = ((imgs - targets) ** 2).mean(dim=(1, 2, 3)).sum()
        loss = img_loss + lap_weight * laplacian_loss(v, edges)
        if on_iter is not None:
            on_iter(it, v.detach(), img_loss.detach())
        loss.backward()
        opt.step()
        hist.append((float(img_loss.detach()), float(loss.detach())))
        if log_every and it % log_every == 0:
            print(f"iter {it}: image loss {hist[-1][0]:.6f}, total {hist[-1][1]:.6f}", flush=True)
    return v.detach(), hist


def edge_opposites(faces):
    """For every edge shared by two faces: (a, b) the edge, c and d the opposite vertices of the two
    faces, as a [4, E] long tensor on faces' device."""
    import numpy as np
    f = faces.detach().cpu().numpy()
    seen = {}
    quads = []
    for t in f:
        for k in range(3):
            a, b, c = int(t[k]), int(t[(k + 1) % 3]), int(t[(k + 2) % 3])
            key = (min(a, b), max(a, b))
            if key in seen:
                quads.append((a, b, seen.pop(key), c))
            else:
                seen[key] = c
    q = torch.as_tensor(np.asarray(quads, dtype=np.int64).reshape(-1, 4).T.copy(), device=faces.device)
    return q


def smoothness_loss(verts, quads, eps=1e-12):
    """Sum over edges of (cos theta + 1)^2, theta the dihedral angle between the two faces of the edge
    measured through the surface (flat: theta = pi, no loss).  cos theta is the cosine between the
    parts of (c - a) and (d - a) perpendicular to the edge (a, b)."""
    a, b, c, d = (verts[quads[i]] for i in range(4))
    e = b - a
    e = e / (e.norm(dim=1, keepdim=True) + eps)
    u = (c - a) - ((c - a) * e).sum(1, keepdim=True) * e
    w = (d - a) - ((d - a) * e).sum(1, keepdim=True) * e
    cos = (u * w).sum(1) / (u.norm(dim=1) * w.norm(dim=1) + eps)
    return ((cos + 1.0) ** 2).sum()


def laplacian_delta_loss(verts, template, edges):
    """Sum over vertices of |delta_v - mean of delta over v's neighbours|^2, delta = verts - template
    (the displacement Laplacian of the loss-term appendix)."""
    delta = verts - template
    V = verts.shape[0]
    deg = torch.zeros(V, device=verts.device, dtype=verts.dtype).index_add_(0, edges[0], torch.ones_like(edges[0], dtype=verts.dtype))
    nb = torch.zeros_like(delta).index_add_(0, edges[0], delta[edges[1]])
    lap = delta - nb / deg.clamp_min(1.0)[:, None]
    return (lap * lap).sum()


def recover_translational(template, faces, albedo, views, targets, T, H, W, iters=1000, batch=16, lr=0.01,
                          betas=(0.5, 0.99), lam_s=3e-2, lam_l=3e-4, solver="fast", seed=0, optimize_albedo=True,
                          log_every=0):
    """Translational recovery with the paper's loss (Eq. loss-img) and settings: every iteration
    renders ``batch`` views sampled from ``views`` (list of (Motion, Camera)) and minimises
    L1(colour) + L1(alpha) (summed over pixels, averaged over the batch's views)
    + lam_s smoothness + lam_l displacement Laplacian, with Adam(lr, betas) on the vertices and,
    if optimize_albedo, the per-vertex colours.  Returns (vertices, colours, loss history)."""
    g = torch.Generator().manual_seed(seed)
    v = template.detach().clone().contiguous().requires_grad_(True)
    c = albedo.detach().clone().contiguous().requires_grad_(optimize_albedo)
    tmpl = template.detach().clone()
    n = len(views)
    k = min(batch, n)
    vb = ViewBatch(v, faces, c, views[:k], T, H, W, solver)
    edges = edge_index(faces, v.shape[0])
    quads = edge_opposites(faces)
    opt = torch.optim.Adam([v, c] if optimize_albedo else [v], lr=lr, betas=betas)
    hist = []
    for it in range(iters):
        pick = torch.randperm(n, generator=g)[:k].tolist()
        vb.views = [views[i] for i in pick]
        tgt = targets[pick]
        opt.zero_grad(set_to_none=False)
        imgs = vb.render()
        img_loss = (imgs - tgt).abs().sum(dim=(1, 2, 3)).mean()
        loss = img_loss + lam_s * smoothness_loss(v, quads) + lam_l * laplacian_delta_loss(v, tmpl, edges)
        loss.backward()
        opt.step()
        with torch.no_grad():
            c.clamp_(0.0, 1.0)
        hist.append((float(img_loss.detach()), float(loss.detach())))
        if log_every and it % log_every == 0:
            print(f"iter {it}: image loss {hist[-1][0]:.3f}, total {hist[-1][1]:.3f}", flush=True)
    return v.detach(), c.detach(), hist
