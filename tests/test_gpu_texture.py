"""Textured renders (Eq. fore with texture-coordinate vertex attributes): the CUDA path against
the oracle for the image, the vertex gradient and the texel gradient, and the batched path
against single renders.  Same bounds as the untextured parity tests; dL/dimage is zeroed on
pixels the oracle flags (including the gradient-only texel-cell flag)."""
import numpy as np
import pytest
import torch

import oracle
import scenes
from gpu_util import ORACLE_MODE, TOL, compare_images, gpu_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2602_07860_gb300 as mbr
    return mbr.Context()


def _tex(sc):
    t = lambda x: torch.as_tensor(np.asarray(x), dtype=torch.float32, device="cuda").contiguous()
    return t(sc["uv"]), t(sc["texture"])


SCENES = {
    "rotate": lambda: scenes.textured(scenes.small_scene("rotate", subdiv=2, T=8, H=40, W=56)),
    "translate": lambda: scenes.textured(scenes.small_scene("translate", subdiv=2, T=10, H=44, W=52,
                                                             d=(0.9, -0.3, 0.6)), th=9, tw=31),
}


@pytest.mark.parametrize("solver", ["plain", "fast"])
@pytest.mark.parametrize("name", sorted(SCENES))
def test_textured_forward_matches_oracle(ctx, name, solver):
    sc = SCENES[name]()
    r = oracle.render(sc, ORACLE_MODE[solver], ambig=True)
    v, f, a, mo, ca = gpu_inputs(sc)
    uv, tex = _tex(sc)
    g = ctx.render_blur(v, f, a, mo, ca, sc["T"], sc["H"], sc["W"], solver, uv=uv, texture=tex)
    g = g.cpu().double().numpy()
    max_clean, frac, excess = compare_images(g, r["rgba"], r["ambig"], sc["T"])
    assert max_clean <= TOL and excess <= 0.0 and frac <= 0.05, (max_clean, excess, frac)
    # the texture matters: the untextured render differs
    plain = ctx.render_blur(v, f, a, mo, ca, sc["T"], sc["H"], sc["W"], solver).cpu().double().numpy()
    assert np.abs(plain - g).max() > 0.05


@pytest.mark.parametrize("solver", ["plain", "fast"])
@pytest.mark.parametrize("name", sorted(SCENES))
def test_textured_adjoint_matches_oracle(ctx, name, solver, rel=1e-3):
    sc = SCENES[name]()
    mode = ORACLE_MODE[solver]
    r = oracle.render(sc, mode, ambig=True, soft32=True)  # the kernels' soft truncation
    rng = np.random.default_rng(3)
    G = rng.normal(size=(sc["H"], sc["W"], 4))
    G[(r["ambig"] != 0).any(0)] = 0.0
    gt_o = np.zeros_like(np.asarray(sc["texture"], dtype=np.float64))
    gv_o, _, _ = oracle.render_backward(sc, G, mode, texture_grad=gt_o, soft32=True)
    v, f, a, mo, ca = gpu_inputs(sc)
    uv, tex = _tex(sc)
    gv, _, gt = ctx.render_blur_backward(v, f, a, mo, ca, sc["T"], sc["H"], sc["W"],
                                         torch.as_tensor(G, dtype=torch.float32, device="cuda"), solver,
                                         uv=uv, texture=tex)
    gv, gt = gv.cpu().double().numpy(), gt.cpu().double().numpy()
    nv = np.linalg.norm(gv_o, axis=1)
    err = np.linalg.norm(gv - gv_o, axis=1)
    assert nv.max() > 0 and np.all(err <= rel * nv + 1e-6 * nv.max()), float((err / (nv + 1e-30)).max())
    assert np.abs(gt_o).max() > 0
    assert np.abs(gt - gt_o).max() <= 1e-4 * np.abs(gt_o).max() + 1e-6, float(np.abs(gt - gt_o).max())


def test_textured_batch_equals_single_renders(ctx):
    import paper_2602_07860_gb300 as mbr
    sc = SCENES["rotate"]()
    v, f, a, mo, ca = gpu_inputs(sc)
    uv, tex = _tex(sc)
    T, H, W = sc["T"], sc["H"], sc["W"]
    G = torch.randn((H, W, 4), device="cuda", generator=torch.Generator("cuda").manual_seed(7))
    ref = ctx.render_blur(v, f, a, mo, ca, T, H, W, "fast", uv=uv, texture=tex)
    gv_r, _, gt_r = ctx.render_blur_backward(v, f, a, mo, ca, T, H, W, G, "fast", uv=uv, texture=tex)
    bctx = mbr.Context()
    img, gv, ga, gt = torch.empty_like(ref), torch.empty_like(v), torch.empty_like(a), torch.empty_like(tex)
    item = dict(verts=v, faces=f, albedo=a, uv=uv, texture=tex, motion=mo, camera=ca, T=T, H=H, W=W,
                solver="fast", image=img, dl_dimage=G, dl_dverts=gv, dl_dalbedo=ga, dl_dtexture=gt)
    for _ in range(2):  # plan, then graph replay
        bctx.render_batch([item], True)
        torch.cuda.synchronize()
        assert float((img - ref).abs().max()) <= 1e-5
        assert float((gv - gv_r).abs().max()) <= 2e-4 * float(gv_r.abs().max())
        assert float((gt - gt_r).abs().max()) <= 2e-4 * float(gt_r.abs().max())
