"""Shape recovery from motion-blurred views (Sec. 5): optimise mesh vertices so that their blurred
renders match target images, with Adam, an L2 image loss and uniform-Laplacian smoothing.

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
    deg = torch.zeros(V, device=verts.device).index_add_(0, edges[0], torch.ones_like(edges[0], dtype=verts.dtype))
    nb = torch.zeros_like(verts).index_add_(0, edges[0], verts[edges[1]])
    lap = verts - nb / deg.clamp_min(1.0)[:, None]
    return (lap * lap).sum(1).mean()


def recover_shape(template, faces, albedo, views, targets, T, H, W, iters=500, lr=1e-3, lap_weight=0.1,
                  solver="fast", log_every=0):
    """Adam on the vertices of ``template`` [V,3] so that their blurred renders under ``views``
    (list of (Motion, Camera)) match ``targets`` [n, H, W, 4].  Loss = mean squared RGBA error
    summed over views + lap_weight x Laplacian term.  Returns (vertices, loss history)."""
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
        loss.backward()
        opt.step()
        hist.append((float(img_loss.detach()), float(loss.detach())))
        if log_every and it % log_every == 0:
            print(f"iter {it}: image loss {hist[-1][0]:.6f}, total {hist[-1][1]:.6f}", flush=True)
    return v.detach(), hist
