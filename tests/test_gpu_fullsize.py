"""Parity at the large configurations, in the launch configuration the benchmark uses (a fresh
context: default tiling, automatic splits), on sampled 16x16 windows the oracle computes:

* the 1024x1024 render of a 100k-face surface of revolution spinning 8 turns with T = 256 and 96
  segments (both solvers);
* items of the 32-object batch (mixed sizes, solvers, sub-frame counts) rendered by one
  graph-captured batch call.

Windows are placed from the scene geometry (the mesh's projected extent at mid-exposure,
computed by the oracle), never from GPU output."""
import numpy as np
import pytest
import torch

import oracle
import scenes
from gpu_util import ORACLE_MODE, TOL, compare_images

pytestmark = pytest.mark.gpu


def _silhouette_windows(sc, n=16):
    """Two windows centred on the leftmost and rightmost projected vertices at t = 0.5 (each at
    its own row), and one at the median vertex position."""
    st = oracle.vertex_state(sc, 0.5)
    H, W = sc["H"], sc["W"]
    px = (st[:, 0] + 1) * 0.5 * W - 0.5
    py = (1 - st[:, 1]) * 0.5 * H - 0.5

    def at(x, y):
        return (int(np.clip(round(x) - n // 2, 0, W - n)), int(np.clip(round(y) - n // 2, 0, H - n)), n, n)

    il, ir = int(np.argmin(px)), int(np.argmax(px))
    return [at(px[il], py[il]), at(px[ir], py[ir]), at(np.median(px), np.median(py))]


@pytest.mark.parametrize("solver", ["fast", "plain"])
def test_large_render_windows(solver):
    import paper_2602_07860_gb300 as mbr
    sc = scenes.config5()
    ctx = mbr.Context()
    v, f, a = mbr.mesh_tensors(sc)
    img = ctx.render_blur(v, f, a, mbr.motion_from_dict(sc["motion"]), mbr.camera_from_dict(sc["camera"]),
                          sc["T"], sc["H"], sc["W"], solver)
    g = img.cpu().double().numpy()
    assert np.isfinite(g).all()
    for win in _silhouette_windows(sc):
        x0, y0, w, h = win
        r = oracle.render(sc, ORACLE_MODE[solver], window=win, ambig=True)
        max_clean, frac, excess = compare_images(g[y0:y0 + h, x0:x0 + w], r["rgba"], r["ambig"], sc["T"])
        assert max_clean <= TOL and excess <= 0.0, (solver, win, max_clean, excess, frac)
        assert r["rgba"][..., 3].max() > 0.05  # the window sees the object or its blur


def test_batch_items_windows():
    import paper_2602_07860_gb300 as mbr
    items_sc = scenes.config4()
    ctx = mbr.Context()
    items = []
    for i, s in enumerate(items_sc):
        v, f, a = mbr.mesh_tensors(s)
        items.append(dict(verts=v, faces=f, albedo=a, motion=mbr.motion_from_dict(s["motion"]),
                          camera=mbr.camera_from_dict(s["camera"]), T=s["T"], H=s["H"], W=s["W"],
                          solver="fast" if i % 3 else "plain",
                          image=torch.zeros((s["H"], s["W"], 4), device="cuda")))
    ctx.render_batch(items, False)
    torch.cuda.synchronize()
    # a few items of different sizes: the smallest, the largest and two in between (by samples)
    by_size = sorted(range(len(items_sc)), key=lambda i: items_sc[i]["H"] * items_sc[i]["W"] * items_sc[i]["T"])
    picks = [by_size[0], by_size[len(by_size) // 3], by_size[2 * len(by_size) // 3], by_size[-1]]
    for i in picks:
        s = items_sc[i]
        g = items[i]["image"].cpu().double().numpy()
        x0, y0, w, h = _silhouette_windows(s)[1]
        r = oracle.render(s, ORACLE_MODE[items[i]["solver"]], window=(x0, y0, w, h), ambig=True)
        max_clean, frac, excess = compare_images(g[y0:y0 + h, x0:x0 + w], r["rgba"], r["ambig"], s["T"])
        assert max_clean <= TOL and excess <= 0.0, (i, items[i]["solver"], max_clean, excess, frac)


def test_more_than_2_31_samples_per_render():
    """T x H x W = 520 x 2048 x 2048 > 2^31 samples (the per-sample raster state alone is 10.9 GB):
    sample and pixel indices are 64-bit.  Silhouette windows of the image match the oracle, and the
    adjoint (reusing the forward's state, whose late sub-frames sit beyond index 2^31) matches the
    oracle's for a loss restricted to one window."""
    import paper_2602_07860_gb300 as mbr
    sc = scenes.small_scene("translate", subdiv=2, T=520, H=2048, W=2048, d=(0.6, 0.2, 0.0))
    assert sc["T"] * sc["H"] * sc["W"] > 2 ** 31
    ctx = mbr.Context()
    v, f, a = mbr.mesh_tensors(sc)
    mo, ca = mbr.motion_from_dict(sc["motion"]), mbr.camera_from_dict(sc["camera"])
    T, H, W = sc["T"], sc["H"], sc["W"]
    img = ctx.render_blur(v, f, a, mo, ca, T, H, W, "fast")
    wins = _silhouette_windows(sc)
    g = {}
    for (x0, y0, w, h) in wins:
        g[(x0, y0)] = img[y0:y0 + h, x0:x0 + w].cpu().double().numpy()
    for win in wins:
        x0, y0, w, h = win
        r = oracle.render(sc, "fast", window=win, ambig=True)
        max_clean, frac, excess = compare_images(g[(x0, y0)], r["rgba"], r["ambig"], T)
        assert max_clean <= TOL and excess <= 0.0, (win, max_clean, excess, frac)
        assert r["rgba"][..., 3].max() > 0.05
    # adjoint for a loss on the first window only
    x0, y0, w, h = wins[0]
    r = oracle.render(sc, "fast", window=wins[0], ambig=True, soft32=True)  # the kernels' truncation
    Gw = np.random.default_rng(2).normal(size=(h, w, 4))
    Gw[(r["ambig"] != 0).any(0)] = 0.0
    gv_o, _, _ = oracle.render_backward(sc, Gw, "fast", window=wins[0], soft32=True)
    G = torch.zeros((H, W, 4), device="cuda")
    G[y0:y0 + h, x0:x0 + w] = torch.as_tensor(Gw, dtype=torch.float32, device="cuda")
    gv, _ = ctx.render_blur_backward(v, f, a, mo, ca, T, H, W, G, "fast", reuse_forward=True)
    assert ctx.stats()["reused"] >= 1
    gv = gv.cpu().double().numpy()
    nv = np.linalg.norm(gv_o, axis=1)
    err = np.linalg.norm(gv - gv_o, axis=1)
    assert nv.max() > 0 and np.all(err <= 1e-3 * nv + 1e-4 * nv.max()), float((err / (nv + 1e-30)).max())
