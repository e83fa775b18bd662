"""CUDA path vs the FP64 oracle, element by element, on seeded scenes (GPU required).

Bound: |gpu - oracle| <= 1e-4 absolute per channel on every pixel none of whose samples the
oracle flags as ambiguous for FP32 (within 2e-6 NDC of a triangle boundary, inverse-depth gap
below 2e-5 relative, near-degenerate triangle, or a fast-mode closest-edge tie); flagged pixels
may differ by at most (flagged samples)/T.  z-test winner ids are bit-exact on unflagged samples.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import scenes
from gpu_util import ORACLE_MODE, TOL, compare_images, degenerate_scene, gpu_inputs, gpu_render

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2602_07860_gb300 as mbr
    return mbr.Context()


# Fraction of pixels with an FP32-ambiguous sample (a property of the oracle's scene alone), as
# measured per scene and solver: at most 1% everywhere except where the scene makes ties on
# purpose or crowds edges.  The degenerate scene's duplicated face ties on every pixel it covers;
# the 96 x 80 subdiv-4 render has about 5000 faces over 7680 pixels (plain 1.21%, fast 0.90%),
# and the depth-moving translation gives keyframe closest-feature ties to the fast solver
# (1.45%).  Bounds sit just above the measurement, so more flagged pixels than the scene's
# own fail the test.
FLAG_FRAC = {"degenerate_faces": 0.033, "subdiv4_sh_96x80": 0.0125, "translate_depth_motion": 0.015}


def _check(ctx, sc, solver, max_flag_frac=0.01):
    r = oracle.render(sc, ORACLE_MODE[solver], ambig=True)
    g = gpu_render(ctx, sc, solver)
    assert np.isfinite(g).all()
    max_clean, frac, excess = compare_images(g, r["rgba"], r["ambig"], sc["T"])
    assert max_clean <= TOL, (max_clean, frac)
    assert excess <= 0.0, (excess, frac)
    assert frac <= max_flag_frac, frac
    return r, g


def _off_axis(sc):
    return dict(sc, camera=scenes.camera(scenes.look_at((0.13, 0.07, -4))))


SCENES = {
    "c1_translate_64": lambda: scenes.config1(),
    "rotate_ragged_72x40": lambda: scenes.small_scene("rotate", subdiv=2, T=8, H=40, W=72),
    "translate_depth_motion": lambda: scenes.small_scene("translate", subdiv=2, T=12, H=48, W=56, d=(0.9, -0.3, 1.1)),
    "rotate_midpoint": lambda: scenes.small_scene("rotate", subdiv=3, T=10, H=50, W=66, time_rule="midpoint"),
    "rotate_fast_spin_S_gt_T": lambda: scenes.small_scene("rotate", subdiv=2, T=5, H=36, W=36, omega=6 * math.pi),
    "subdiv4_sh_96x80": lambda: scenes.config2(T=16, H=80, W=96),
    "single_subframe": lambda: scenes.small_scene("rotate", subdiv=2, T=1, H=33, W=47),
    # the appendix's combined rotation and parabolic translation (6 segments for the half turn)
    "parabolic_appendix": lambda: dict(scenes.small_scene("parabolic", subdiv=2, T=16, H=48, W=64),
                                       camera=scenes.camera(scenes.look_at(scenes.orbit_eye(5.0, 0, 10.0)))),
    # the SoftRas probability map the paper replaces (sigmoid instead of exp), with a wide delta
    "rotate_sigmoid_prob": lambda: dict(scenes.small_scene("rotate", subdiv=2, T=8, H=40, W=56),
                                        camera=scenes.camera(scenes.look_at((0, 0, -4)), delta=2e-3, prob="sigmoid")),
    # no motion at all: every sub-frame is the same static render
    "static_zero_motion": lambda: scenes.small_scene("translate", subdiv=2, T=6, H=36, W=44, d=(0.0, 0.0, 0.0)),
    # degenerate input: zero-area faces (a repeated vertex, three collinear vertices) and a
    # duplicated face (exact depth ties, resolved to the smaller id)
    "degenerate_faces": degenerate_scene,
    # soft band far below a pixel (delta 1e-6) and far above it (delta 1e-2)
    "rotate_tiny_delta": lambda: dict(scenes.small_scene("rotate", subdiv=2, T=6, H=40, W=48),
                                      camera=scenes.camera(scenes.look_at((0, 0, -4)), delta=1e-6)),
    "rotate_wide_delta": lambda: dict(scenes.small_scene("rotate", subdiv=1, T=4, H=32, W=40),
                                      camera=scenes.camera(scenes.look_at((0, 0, -4)), delta=1e-2)),
    # one-pixel images and strips: every tile is ragged.  The camera looks slightly off the
    # optical axis, so the pixel row / column does not run along the mesh's vertices and edges
    # (on the axis most of its samples are flagged as FP32-ambiguous)
    "pixel_1x1_off_axis": lambda: _off_axis(scenes.small_scene("rotate", subdiv=2, T=8, H=1, W=1)),
    "strip_1x37_off_axis": lambda: _off_axis(scenes.small_scene("rotate", subdiv=2, T=8, H=1, W=37)),
    "strip_41x1_off_axis": lambda: _off_axis(scenes.small_scene("rotate", subdiv=2, T=8, H=41, W=1)),
    # perspective-correct attribute weights, camera close to the mesh (strong depth variation)
    "translate_perspective_attrs": lambda: dict(
        scenes.small_scene("translate", subdiv=2, T=10, H=44, W=60, d=(0.8, -0.2, 1.0)),
        camera=scenes.camera(scenes.look_at((0.4, 0.3, -2.6)), fov_deg=60.0, interp="perspective")),
}


@pytest.mark.parametrize("solver", ["plain", "fast"])
@pytest.mark.parametrize("name", sorted(SCENES))
def test_forward_matches_oracle(ctx, name, solver):
    _check(ctx, SCENES[name](), solver, FLAG_FRAC.get(name, 0.01))


@pytest.mark.parametrize("solver", ["plain", "fast"])
def test_winner_ids_bit_exact(ctx, solver):
    sc = scenes.small_scene("rotate", subdiv=3, T=6, H=44, W=52)
    r = oracle.render(sc, ORACLE_MODE[solver], winners=True, ambig=True)
    v, f, a, mo, ca = gpu_inputs(sc)
    for k in range(sc["T"]):
        ids = ctx.debug_winners(v, f, a, mo, ca, sc["T"], sc["H"], sc["W"], k, solver).cpu().numpy()
        clean = r["ambig"][k] == 0
        assert np.array_equal(ids[clean], r["winners"][k][clean]), k
        assert (ids >= 0).sum() > 50


@pytest.mark.parametrize("tile,spt", [(16, 4), (8, 4), (16, 1), (8, 2)])
def test_tuning_variants_agree(ctx, tile, spt):
    sc = scenes.small_scene("rotate", subdiv=2, T=20, H=45, W=61)
    ref = gpu_render(ctx, sc, "fast")
    ctx.set_tuning(tile, spt, 0)
    try:
        for solver in ("fast", "plain"):
            _check(ctx, sc, solver, 0.0125)  # measured: plain 1.17%, fast 1.24% of the pixels flagged
        g = gpu_render(ctx, sc, "fast")
        assert np.max(np.abs(g - ref)) < 2e-6
    finally:
        ctx.set_tuning(16, 2, 0)


def test_splits_agree(ctx):
    sc = scenes.small_scene("rotate", subdiv=2, T=24, H=40, W=40)
    imgs = []
    for splits in (1, 3, 24):
        ctx.set_tuning(16, 2, splits)
        imgs.append(gpu_render(ctx, sc, "plain"))
    ctx.set_tuning(16, 2, 0)
    assert np.max(np.abs(imgs[0] - imgs[1])) < 2e-6 and np.max(np.abs(imgs[0] - imgs[2])) < 2e-6


def test_empty_mesh_and_offscreen(ctx):
    sc = scenes.small_scene("translate", subdiv=1, T=4, H=20, W=24)
    empty = dict(sc, faces=np.zeros((0, 3), dtype=np.int32))
    for solver in ("plain", "fast"):
        assert np.all(gpu_render(ctx, empty, solver) == 0.0)
    far = dict(sc, verts=sc["verts"] + np.array([50.0, 0.0, 0.0]))
    for solver in ("plain", "fast"):
        assert np.all(gpu_render(ctx, far, solver) == 0.0)


def test_behind_camera_is_skipped(ctx):
    """Triangles with a vertex at camera z <= znear are skipped, identically in both paths."""
    sc = scenes.small_scene("translate", subdiv=2, T=6, H=30, W=30, d=(0.0, 0.0, -3.5))
    for solver in ("plain", "fast"):
        _check(ctx, sc, solver)


def test_full_size_rotation_windows(ctx):
    """Full-size rotation workload (subdiv-4 SH sphere, T = 64, 256x256, 12 segments), the launch
    configuration the benchmark times, against the oracle on sampled 16x16 windows."""
    sc = scenes.config2()
    for solver in ("fast", "plain"):
        g = gpu_render(ctx, sc, solver)
        for (x0, y0) in [(120, 120), (60, 128), (176, 72), (8, 8)]:
            win = (x0, y0, 16, 16)
            r = oracle.render(sc, ORACLE_MODE[solver], window=win, ambig=True)
            gw = g[y0:y0 + 16, x0:x0 + 16]
            max_clean, frac, excess = compare_images(gw, r["rgba"], r["ambig"], sc["T"])
            assert max_clean <= TOL and excess <= 0.0, (solver, win, max_clean, excess, frac)


def test_candidate_count_matches_oracle(ctx):
    sc = scenes.small_scene("rotate", subdiv=2, T=8, H=40, W=72)
    v, f, a, mo, ca = gpu_inputs(sc)
    for solver in ("plain", "fast"):
        n = ctx.count_candidates(v, f, a, mo, ca, sc["T"], sc["H"], sc["W"], solver)
        ref = oracle.render(sc, ORACLE_MODE[solver])["counters"][oracle.CNT_CAND]
        assert abs(n - ref) <= 1e-3 * ref, (solver, n, ref)


@pytest.mark.parametrize("solver", ["plain", "fast"])
@pytest.mark.parametrize("kind", ["translate", "rotate"])
def test_work_counts_match_oracle(ctx, kind, solver):
    """The roofline's work units counted by the GPU path (mbr_count_work) against the oracle's
    counters: N_cand, soft terms of uncovered samples above the single-precision cutoff, covered
    samples.  FP32 decisions near a boundary may differ: 1e-3 relative."""
    sc = scenes.small_scene(kind, subdiv=2, T=8, H=40, W=72)
    v, f, a, mo, ca = gpu_inputs(sc)
    img = torch.zeros((sc["H"], sc["W"], 4), device="cuda")
    d = ctx.count_work(v, f, a, mo, ca, sc["T"], sc["H"], sc["W"], solver, out=img, detail=True)
    n_cand, n_soft, n_cov = d["n_cand"], d["n_soft"], d["n_cov"]
    assert 0 < d["n_box"] < n_cand and d["cov_tests"] >= d["n_box"] * 0.5
    c = oracle.render(sc, ORACLE_MODE[solver])["counters"]
    assert abs(n_cand - c[oracle.CNT_CAND]) <= 1e-3 * c[oracle.CNT_CAND], (n_cand, c[oracle.CNT_CAND])
    assert abs(n_soft - c[oracle.CNT_SOFT32]) <= 1e-3 * c[oracle.CNT_SOFT32] + 2, (n_soft, c[oracle.CNT_SOFT32])
    assert abs(n_cov - c[oracle.CNT_COVERED]) <= 1e-3 * c[oracle.CNT_COVERED] + 2, (n_cov, c[oracle.CNT_COVERED])
    assert n_soft > 0 and n_cov > 0
    # the counting build renders the same image
    ref = gpu_render(ctx, sc, solver)
    assert float((img - torch.as_tensor(ref, device="cuda")).abs().max()) <= 1e-5


def test_bad_arguments_return_errors(ctx):
    import paper_2602_07860_gb300 as mbr
    from paper_2602_07860_gb300._lib import MbrError
    sc = scenes.small_scene("rotate", subdiv=1, T=4, H=16, W=16)
    v, f, a, mo, ca = gpu_inputs(sc)
    with pytest.raises(MbrError):
        ctx.render_blur(v, f, a, mo, ca, 0, 16, 16, "fast")
    bad = mbr.Motion(kind="rotate", axis=(0.0, 0.0, 0.0), omega=1.0)
    with pytest.raises(MbrError):
        ctx.render_blur(v, f, a, bad, ca, 4, 16, 16, "fast")
    with pytest.raises(MbrError):
        ctx.set_tuning(12, 8, 0)
    # the context stays usable after errors
    assert np.isfinite(gpu_render(ctx, sc, "fast")).all()


def test_segment_count_convergence(ctx):
    """Segmentation analysis: the fast solver linearises the rotation per segment, so its image
    approaches the exact per-sub-frame render as segments go 6 -> 12 -> 24 -> 48 (one turn)."""
    import dataclasses
    sc = scenes.config2(T=48, H=96, W=96)
    v, f, a, mo, ca = gpu_inputs(sc)
    exact = ctx.render_blur(v, f, a, mo, ca, sc["T"], sc["H"], sc["W"], "plain")
    errs = []
    for S in (6, 12, 24, 48):
        img = ctx.render_blur(v, f, a, dataclasses.replace(mo, segments=S), ca, sc["T"], sc["H"], sc["W"], "fast")
        errs.append(float((img - exact).abs().mean()))
    torch.cuda.synchronize()
    assert all(errs[i + 1] < errs[i] for i in range(3)), errs
    assert errs[-1] < 0.25 * errs[0], errs
