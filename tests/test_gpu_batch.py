"""Batched renders (mbr_render_blur_batch): one persistent raster launch over items of different
sizes, solvers and sub-frame counts, captured in a CUDA graph and replayed.  Every item must equal
its own single render (mbr_render_blur / _backward); the parity of single renders with the FP64
oracle is covered by test_gpu_parity and test_gpu_backward."""
import math

import numpy as np
import pytest
import torch

import scenes
from gpu_util import gpu_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2602_07860_gb300 as mbr
    return mbr.Context()


def _items(specs, with_backward):
    items = []
    for sc, solver in specs:
        v, f, a, mo, ca = gpu_inputs(sc)
        it = dict(verts=v, faces=f, albedo=a, motion=mo, camera=ca, T=sc["T"], H=sc["H"], W=sc["W"],
                  solver=solver, image=torch.zeros((sc["H"], sc["W"], 4), device="cuda"))
        if with_backward:
            it["dl_dimage"] = torch.randn((sc["H"], sc["W"], 4), device="cuda",
                                          generator=torch.Generator("cuda").manual_seed(len(items)))
            it["dl_dverts"] = torch.zeros_like(v)
            it["dl_dalbedo"] = torch.zeros_like(a)
        items.append(it)
    return items


def _specs():
    return [
        (scenes.config1(), "fast"),
        (scenes.small_scene("rotate", subdiv=2, T=8, H=40, W=72), "plain"),
        (scenes.small_scene("rotate", subdiv=3, T=20, H=96, W=80, seed=7), "fast"),
        (scenes.small_scene("translate", subdiv=2, T=12, H=48, W=56, d=(0.9, -0.3, 1.1)), "plain"),
        (scenes.config2(T=16, H=80, W=96), "fast"),
    ]


def _check(ctx, items, with_backward, tol_img=1e-5, tol_grad=2e-4):
    for it in items:
        ref = ctx.render_blur(it["verts"], it["faces"], it["albedo"], it["motion"], it["camera"], it["T"], it["H"],
                              it["W"], it["solver"])
        assert float((it["image"] - ref).abs().max()) <= tol_img
        if with_backward:
            gv, ga = ctx.render_blur_backward(it["verts"], it["faces"], it["albedo"], it["motion"], it["camera"],
                                              it["T"], it["H"], it["W"], it["dl_dimage"], it["solver"])
            scale = float(gv.abs().max()) + 1e-30
            assert float((it["dl_dverts"] - gv).abs().max()) <= tol_grad * scale
            assert float((it["dl_dalbedo"] - ga).abs().max()) <= tol_grad * (float(ga.abs().max()) + 1e-30)


@pytest.mark.parametrize("with_backward", [False, True])
def test_batch_matches_single_renders(ctx, with_backward):
    items = _items(_specs(), with_backward)
    ctx.render_batch(items, with_backward)
    torch.cuda.synchronize()
    _check(ctx, items, with_backward)


def test_batch_graph_replay_follows_new_vertices_and_motion(ctx):
    items = _items(_specs(), True)
    ctx.render_batch(items, True)  # plans and captures
    for step in range(3):
        # move the vertices in place and change one motion: the replayed graph must see both
        for it in items:
            it["verts"].mul_(1.0 + 0.01 * (step + 1))
        items[2]["motion"].omega *= 1.05
        ctx.render_batch(items, True)
        torch.cuda.synchronize()
        _check(ctx, items, True)


def test_batch_replans_when_bins_overflow(ctx):
    items = _items(_specs()[:3], False)
    ctx.render_batch(items, False)
    for it in items:
        it["verts"].mul_(1.6)  # larger on screen: far more (tile, face) entries than the headroom
    ctx.render_batch(items, False)
    torch.cuda.synchronize()
    _check(ctx, items, False)


def test_autotune_picks_a_candidate_and_keeps_results(ctx):
    items = _items(_specs()[:3], True)
    tile, spt, ms = ctx.autotune(items, True)
    assert tile in (8, 16) and spt in (1, 2, 4) and math.isfinite(ms) and ms > 0
    ctx.render_batch(items, True)
    torch.cuda.synchronize()
    _check(ctx, items, True)
    ctx.set_tuning(16, 2, 0)


def test_single_renders_after_a_batch_keep_their_buffers():
    # a context that has rendered singly, then a batch, then singly again: the batch must not
    # disturb the context's own scratch buffers
    import paper_2602_07860_gb300 as mbr
    c = mbr.Context()
    sc = scenes.config2(T=16, H=80, W=96)
    v, f, a, mo, ca = gpu_inputs(sc)
    before = c.render_blur(v, f, a, mo, ca, sc["T"], sc["H"], sc["W"], "fast")
    c.render_batch(_items(_specs()[:2], True), True)
    after = c.render_blur(v, f, a, mo, ca, sc["T"], sc["H"], sc["W"], "fast")
    torch.cuda.synchronize()
    # the fills order each tile's face list by atomics, so the soft products may round differently
    assert float((before - after).abs().max()) <= 1e-5
