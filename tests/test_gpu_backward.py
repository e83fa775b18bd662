"""CUDA adjoint (mbr_render_blur_backward) vs the oracle's FP64 adjoint, which is itself pinned
to central finite differences.  The oracle runs with the kernels' single-precision soft truncation
(soft32: factors with exp(-d/delta) <= 2^-25 dropped, the ones an FP32 product cannot see), so
both sides differentiate the same function.  dL/dimage is zeroed on pixels whose samples the oracle flags as
ambiguous for FP32 (any flag, including the gradient-only ones), so both sides differentiate the
same discrete choices.  Bound: per-vertex |g_gpu - g_oracle|_2 <= 1e-3 |g_oracle|_2 + 1e-6 max."""
import numpy as np
import pytest
import torch

import oracle
import scenes
from gpu_util import ORACLE_MODE, degenerate_scene, gpu_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2602_07860_gb300 as mbr
    return mbr.Context()


@pytest.fixture(scope="module")
def ctx_free():
    """A context whose forward keeps no per-sample state: its adjoint recomputes coverage and the
    soft products (the state-free adjoint)."""
    import paper_2602_07860_gb300 as mbr
    c = mbr.Context()
    c.set_state_budget(0)
    return c


def _grad_check(ctx, sc, solver, seed=0, rel=1e-3):
    mode = ORACLE_MODE[solver]
    r = oracle.render(sc, mode, ambig=True, soft32=True)
    rng = np.random.default_rng(seed)
    G = rng.normal(size=(sc["H"], sc["W"], 4))
    G[(r["ambig"] != 0).any(0)] = 0.0
    gv_o, ga_o, _ = oracle.render_backward(sc, G, mode, soft32=True)
    v, f, a, mo, ca = gpu_inputs(sc)
    gv, ga = ctx.render_blur_backward(v, f, a, mo, ca, sc["T"], sc["H"], sc["W"],
                                      torch.as_tensor(G, dtype=torch.float32, device="cuda"), solver)
    torch.cuda.synchronize()
    gv = gv.cpu().double().numpy()
    ga = ga.cpu().double().numpy()
    nv_o = np.linalg.norm(gv_o, axis=1)
    scale = nv_o.max()
    assert scale > 0
    err = np.linalg.norm(gv - gv_o, axis=1)
    bad = err > rel * nv_o + 1e-6 * scale
    assert not bad.any(), (solver, int(bad.sum()), [(int(i), float(err[i] / nv_o[i]), float(nv_o[i] / scale))
                                                   for i in np.nonzero(bad)[0][:5]])
    na_o = np.linalg.norm(ga_o, axis=1)
    erra = np.linalg.norm(ga - ga_o, axis=1)
    assert np.all(erra <= rel * na_o + 1e-6 * na_o.max())
    return float(np.linalg.norm(gv - gv_o) / np.linalg.norm(gv_o))


GRAD_SCENES = {
    "rotate": lambda: scenes.small_scene("rotate", subdiv=2, T=8, H=40, W=52),
    "translate_depth": lambda: scenes.small_scene("translate", subdiv=2, T=10, H=44, W=48, d=(0.9, -0.3, 1.1)),
    "rotate_wide_soft": lambda: dict(scenes.small_scene("rotate", subdiv=1, T=6, H=32, W=40),
                                     camera=dict(scenes.small_scene("rotate", subdiv=1)["camera"], delta=2e-3)),
    "c1": lambda: scenes.config1(),
    "parabolic": lambda: dict(scenes.small_scene("parabolic", subdiv=2, T=10, H=40, W=48),
                              camera=scenes.camera(scenes.look_at(scenes.orbit_eye(5.0, 0, 10.0)))),
    "rotate_sigmoid_prob": lambda: dict(scenes.small_scene("rotate", subdiv=1, T=6, H=32, W=40),
                                        camera=scenes.camera(scenes.look_at((0, 0, -4)), delta=2e-3, prob="sigmoid")),
    "static_zero_motion": lambda: scenes.small_scene("translate", subdiv=2, T=6, H=36, W=44, d=(0.0, 0.0, 0.0)),
    # zero-area faces and a duplicated face (the oracle flags the exact depth ties as ambiguous)
    "degenerate_faces": degenerate_scene,
    # one-pixel-wide images: every tile is ragged
    "strip_1x37": lambda: scenes.small_scene("rotate", subdiv=2, T=8, H=1, W=37),
    "strip_41x1": lambda: scenes.small_scene("rotate", subdiv=2, T=8, H=41, W=1),
    "rotate_perspective_attrs": lambda: dict(
        scenes.small_scene("rotate", subdiv=2, T=8, H=40, W=48),
        camera=scenes.camera(scenes.look_at((0.4, 0.3, -2.6)), fov_deg=60.0, interp="perspective")),
}


@pytest.mark.parametrize("solver", ["plain", "fast"])
@pytest.mark.parametrize("name", sorted(GRAD_SCENES))
def test_adjoint_matches_oracle(ctx, name, solver):
    _grad_check(ctx, GRAD_SCENES[name](), solver)


@pytest.mark.parametrize("solver", ["plain", "fast"])
@pytest.mark.parametrize("name", ["rotate", "translate_depth", "c1", "degenerate_faces", "strip_1x37", "parabolic",
                                  "rotate_perspective_attrs"])
def test_state_free_adjoint_matches_oracle(ctx_free, name, solver):
    _grad_check(ctx_free, GRAD_SCENES[name](), solver)


@pytest.mark.parametrize("tile,spt", [(16, 4), (8, 4), (8, 1), (16, 1), (8, 2)])
@pytest.mark.parametrize("state_free", [False, True])
def test_adjoint_tuning_variants(tile, spt, state_free):
    """The fast solver's adjoint at every tile size and samples-per-group choice the autotuner can
    make: one sample per group, two (per-sample coefficients staged per candidate) and four (the
    staged record, coefficients formed per pair), with stored and with recomputed state."""
    import paper_2602_07860_gb300 as mbr
    c = mbr.Context()
    c.set_tuning(tile, spt, 0)
    if state_free:
        c.set_state_budget(0)
    try:
        _grad_check(c, scenes.small_scene("rotate", subdiv=2, T=20, H=45, W=61), "fast")
        _grad_check(c, scenes.small_scene("translate", subdiv=2, T=16, H=40, W=48, d=(0.9, -0.3, 1.1)), "fast")
    finally:
        c.close()


@pytest.mark.parametrize("solver", ["plain", "fast"])
def test_state_free_adjoint_at_T256(ctx_free, solver):
    """T = 256 sub-frames (the large workload's count) with no stored sample state."""
    _grad_check(ctx_free, scenes.small_scene("rotate", subdiv=2, T=256, H=32, W=40, omega=4 * np.pi), solver)


@pytest.mark.parametrize("solver", ["plain", "fast"])
def test_state_free_equals_stored_state(ctx, ctx_free, solver):
    """The two adjoint modes compute the same gradients (up to the order of floating-point sums),
    through the autograd path and through the recomputing call; a budget below one render's
    state selects the state-free mode by itself."""
    import paper_2602_07860_gb300 as mbr
    sc = scenes.small_scene("rotate", subdiv=3, T=16, H=56, W=64, seed=4)
    v, f, a, mo, ca = gpu_inputs(sc)
    G = torch.randn((sc["H"], sc["W"], 4), device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    T, H, W = sc["T"], sc["H"], sc["W"]
    ref_v, ref_a = ctx.render_blur_backward(v, f, a, mo, ca, T, H, W, G, solver)
    small = mbr.Context()
    small.set_state_budget(T * H * W * 5 - 1)
    for c in (ctx_free, small):
        c.render_blur(v, f, a, mo, ca, T, H, W, solver)
        gv, ga = c.render_blur_backward(v, f, a, mo, ca, T, H, W, G, solver, reuse_forward=True)
        torch.cuda.synchronize()
        assert float((gv - ref_v).abs().max()) <= 1e-4 * float(ref_v.abs().max())
        assert float((ga - ref_a).abs().max()) <= 1e-4 * float(ref_a.abs().max())
    with pytest.raises(Exception):
        small.set_state_budget(-1)


@pytest.mark.parametrize("solver", ["plain", "fast"])
@pytest.mark.parametrize("state_free", [False, True])
def test_adjoint_is_finite_where_pixels_lie_on_edges(ctx, ctx_free, solver, state_free):
    """The undisplaced icosphere of the shape-recovery workload seen by two of its full-size views
    (256^2, T = 64): its symmetric tessellation puts pixel centres exactly on triangle edges, where
    an uncovered sample's soft factor 1 - exp(-d / delta) rounds to zero.  Forward and adjoint must
    take the same single-precision decision there (a factor the forward counted as vanishing is not
    divided out by the adjoint), so every vertex gradient is finite."""
    import paper_2602_07860_gb300 as mbr
    views, template = scenes.config3()
    c = ctx_free if state_free else ctx
    for k in (0, 7):
        sc = dict(views[k], verts=template)
        v, f, a, mo, ca = gpu_inputs(sc)
        G = torch.as_tensor(np.random.default_rng(3).normal(size=(sc["H"], sc["W"], 4)).astype(np.float32),
                            device="cuda")
        gv, ga = c.render_blur_backward(v, f, a, mo, ca, sc["T"], sc["H"], sc["W"], G, solver)
        torch.cuda.synchronize()
        assert torch.isfinite(gv).all() and torch.isfinite(ga).all(), (k, solver, state_free)
        assert float(gv.abs().max()) > 0


@pytest.mark.parametrize("solver", ["plain", "fast"])
def test_adjoint_is_zero_without_visible_geometry_or_loss(ctx, solver):
    """No faces, a mesh far outside the view, or a zero dL/dimage: both gradients are exactly zero
    (and the buffers the call overwrites hold no stale values)."""
    sc = scenes.small_scene("translate", subdiv=1, T=4, H=20, W=24)
    G = torch.randn((sc["H"], sc["W"], 4), device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    cases = [(dict(sc, faces=np.zeros((0, 3), dtype=np.int32)), G),
             (dict(sc, verts=sc["verts"] + np.array([50.0, 0.0, 0.0])), G),
             (sc, torch.zeros_like(G))]
    for case, g in cases:
        v, f, a, mo, ca = gpu_inputs(case)
        gv, ga = ctx.render_blur_backward(v, f, a, mo, ca, case["T"], case["H"], case["W"], g, solver)
        torch.cuda.synchronize()
        assert gv.shape == v.shape and ga.shape == a.shape
        assert float(gv.abs().max()) == 0.0 and float(ga.abs().max()) == 0.0


@pytest.mark.parametrize("solver", ["plain", "fast"])
def test_autograd_function_uses_the_adjoint(ctx, solver):
    import paper_2602_07860_gb300 as mbr
    sc = scenes.small_scene("rotate", subdiv=2, T=6, H=32, W=36)
    v, f, a, mo, ca = gpu_inputs(sc)
    vv = v.clone().requires_grad_(True)
    aa = a.clone().requires_grad_(True)
    img = mbr.render_blur(vv, aa, f, mo, ca, sc["T"], sc["H"], sc["W"], solver, ctx)
    G = torch.randn_like(img)
    (img * G).sum().backward()
    gv, ga = ctx.render_blur_backward(v, f, a, mo, ca, sc["T"], sc["H"], sc["W"], G, solver)
    assert torch.allclose(vv.grad, gv, rtol=1e-4, atol=1e-5 * gv.abs().max().item())
    assert torch.allclose(aa.grad, ga, rtol=1e-4, atol=1e-6)


@pytest.mark.parametrize("state_free", [False, True])
@pytest.mark.parametrize("x0,y0", [(116, 100), (56, 88), (56, 152)])
def test_full_size_rotation_gradient_window(ctx, ctx_free, x0, y0, state_free):
    """Full-size rotation workload (the benchmark's) with an L2 image loss against a target (the
    same object scaled by 1.02) on a 24x24 window: GPU adjoint vs the oracle adjoint.

    Bound: globally |g - g_o| <= 1e-3 |g_o|; per vertex |g_v - g_o,v| <= 1e-3 |g_o,v| + 1e-4 max|g_o|.
    The floor is the FP32 limit of the soft term: exp(-d / delta) with delta = 1e-4 turns the
    ~6e-8 absolute error of single-precision screen positions into ~(2 r / delta) 6e-8 ~ 6e-5
    relative error per term, which shows where a vertex's contributions nearly cancel."""
    ctx = ctx_free if state_free else ctx
    sc = scenes.config2()
    w, h = 24, 24
    target = dict(sc, verts=sc["verts"] * 1.02)
    for solver in ("fast", "plain"):
        mode = ORACLE_MODE[solver]
        r = oracle.render(sc, mode, window=(x0, y0, w, h), ambig=True, soft32=True)
        tgt = oracle.render(target, mode, window=(x0, y0, w, h), soft32=True)["rgba"]
        Gw = 2.0 * (r["rgba"] - tgt)
        Gw[(r["ambig"] != 0).any(0)] = 0.0
        gv_o, _, _ = oracle.render_backward(sc, Gw, mode, window=(x0, y0, w, h), soft32=True)
        G = np.zeros((sc["H"], sc["W"], 4))
        G[y0:y0 + h, x0:x0 + w] = Gw
        v, f, a, mo, ca = gpu_inputs(sc)
        gv, _ = ctx.render_blur_backward(v, f, a, mo, ca, sc["T"], sc["H"], sc["W"],
                                         torch.as_tensor(G, dtype=torch.float32, device="cuda"), solver)
        gv = gv.cpu().double().numpy()
        nv_o = np.linalg.norm(gv_o, axis=1)
        assert nv_o.max() > 0 and (Gw != 0).any(-1).mean() > 0.1
        assert np.linalg.norm(gv - gv_o) <= 1e-3 * np.linalg.norm(gv_o)
        err = np.linalg.norm(gv - gv_o, axis=1)
        assert np.all(err <= 1e-3 * nv_o + 1e-4 * nv_o.max()), (solver, float(err.max()), float(nv_o.max()))


@pytest.mark.parametrize("solver", ["fast", "plain"])
def test_adjoint_reusing_the_forward_front_half(ctx, solver):
    """mbr_render_blur_backward_reuse right after the forward reuses its front half (counted in
    the stats) and equals the recomputing adjoint; with another call in between it recomputes and
    is still right."""
    sc = scenes.small_scene("rotate", subdiv=2, T=12, H=48, W=56, seed=9)
    other = scenes.small_scene("translate", subdiv=2, T=8, H=40, W=40, seed=10)
    v, f, a, mo, ca = gpu_inputs(sc)
    v2, f2, a2, mo2, ca2 = gpu_inputs(other)
    g = torch.randn((sc["H"], sc["W"], 4), device="cuda", generator=torch.Generator("cuda").manual_seed(2))
    T, H, W = sc["T"], sc["H"], sc["W"]
    ref_v, ref_a = ctx.render_blur_backward(v, f, a, mo, ca, T, H, W, g, solver)
    s0 = ctx.stats()["reused"]
    ctx.render_blur(v, f, a, mo, ca, T, H, W, solver)
    gv, ga = ctx.render_blur_backward(v, f, a, mo, ca, T, H, W, g, solver, reuse_forward=True)
    torch.cuda.synchronize()
    assert ctx.stats()["reused"] == s0 + 1
    scale = float(ref_v.abs().max())
    assert float((gv - ref_v).abs().max()) <= 1e-5 * scale
    assert float((ga - ref_a).abs().max()) <= 1e-5 * float(ref_a.abs().max())
    # another render in between: the adjoint must recompute (no reuse) and still be right
    ctx.render_blur(v, f, a, mo, ca, T, H, W, solver)
    ctx.render_blur(v2, f2, a2, mo2, ca2, other["T"], other["H"], other["W"], solver)
    gv2, _ = ctx.render_blur_backward(v, f, a, mo, ca, T, H, W, g, solver, reuse_forward=True)
    torch.cuda.synchronize()
    assert ctx.stats()["reused"] == s0 + 1
    assert float((gv2 - ref_v).abs().max()) <= 1e-5 * scale
    # a changed camera is a different render: no reuse
    ctx.render_blur(v, f, a, mo, ca, T, H, W, solver)
    ca_moved = mbr_camera_with_delta(ca, 2e-4)
    ctx.render_blur_backward(v, f, a, mo, ca_moved, T, H, W, g, solver, reuse_forward=True)
    torch.cuda.synchronize()
    assert ctx.stats()["reused"] == s0 + 1


def mbr_camera_with_delta(ca, delta):
    import dataclasses
    return dataclasses.replace(ca, delta=delta)
