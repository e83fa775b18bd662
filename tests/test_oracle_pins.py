"""Pins of the FP64 oracle against things other than itself: the paper's printed appendix
coefficients (symbolic identity), closed forms, invariants, special cases and brute force.

Every test here runs on the CPU (no GPU marker)."""
import math
import os

import numpy as np
import pytest

import oracle
import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "appendix_A_coefficients.txt")


def _golden_exprs():
    import sympy as sp
    out = {}
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, expr = line.split("=", 1)
            out[name.strip()] = sp.sympify(expr)
    return out


# ----------------------------------------------------------------------------- Appendix A

def test_appendix_coefficients_equal_adjugate_expansion():
    """Appendix A: adj(F(t)) p and det F(t) with linearly moving vertices expand to exactly the
    printed A_1..A_3 and a_1..a_3 (symbolic identity, all components)."""
    sp = pytest.importorskip("sympy")
    g = _golden_exprs()
    t, u, v = sp.symbols("t u v")
    xs = {(i, T): sp.Symbol(f"x{i}{T}") for i in range(3) for T in range(2)}
    ys = {(i, T): sp.Symbol(f"y{i}{T}") for i in range(3) for T in range(2)}
    x = [(1 - t) * xs[(i, 0)] + t * xs[(i, 1)] for i in range(3)]
    y = [(1 - t) * ys[(i, 0)] + t * ys[(i, 1)] for i in range(3)]
    F = sp.Matrix([[x[0], x[1], x[2]], [y[0], y[1], y[2]], [1, 1, 1]])
    num = F.adjugate() * sp.Matrix([u, v, 1])
    det = sp.expand(F.det())
    for i in range(3):
        poly = sp.Poly(sp.expand(num[i]), t)
        assert sp.expand(poly.coeff_monomial(t ** 2) - g[f"A1_{i}"]) == 0
        assert sp.expand(poly.coeff_monomial(t) - g[f"A2_{i}"]) == 0
        assert sp.expand(poly.coeff_monomial(1) - g[f"A3_{i}"]) == 0
    dp = sp.Poly(det, t)
    assert sp.expand(dp.coeff_monomial(t ** 2) - g["a1"]) == 0
    assert sp.expand(dp.coeff_monomial(t) - g["a2"]) == 0
    assert sp.expand(dp.coeff_monomial(1) - g["a3"]) == 0
    # the numerators sum to the denominator: barycentrics sum to one at every t
    for p, q in (("A1", "a1"), ("A2", "a2"), ("A3", "a3")):
        assert sp.expand(g[f"{p}_0"] + g[f"{p}_1"] + g[f"{p}_2"] - g[q]) == 0


def test_oracle_barycentric_matches_printed_quadratic_rational():
    """The oracle's Gaussian-elimination solve of F(t) w = p equals Eq. time-dependent2 evaluated
    with the printed coefficients, on random moving triangles and times."""
    sp = pytest.importorskip("sympy")
    g = _golden_exprs()
    names = sorted({s.name for e in g.values() for s in e.free_symbols})
    fns = {k: sp.lambdify([sp.Symbol(n) for n in names], e, "numpy") for k, e in g.items()}
    rng = np.random.default_rng(7)
    worst = 0.0
    for _ in range(2000):
        k0 = rng.uniform(-1, 1, 6)
        k1 = k0 + rng.uniform(-0.5, 0.5, 6)
        u, v = rng.uniform(-1, 1, 2)
        t = rng.uniform(0, 1)
        env = {f"x{i}0": k0[2 * i] for i in range(3)}
        env.update({f"y{i}0": k0[2 * i + 1] for i in range(3)})
        env.update({f"x{i}1": k1[2 * i] for i in range(3)})
        env.update({f"y{i}1": k1[2 * i + 1] for i in range(3)})
        env.update(u=u, v=v)
        args = [env[n] for n in names]
        den = fns["a1"](*args) * t * t + fns["a2"](*args) * t + fns["a3"](*args)
        w_q = np.array([(fns[f"A1_{i}"](*args) * t * t + fns[f"A2_{i}"](*args) * t + fns[f"A3_{i}"](*args)) / den
                        for i in range(3)])
        tri = (1 - t) * k0 + t * k1
        w_o, det = oracle.barycentric(tri, u, v)
        if abs(det) < 1e-3:
            continue
        worst = max(worst, np.max(np.abs(w_o - w_q)) / max(1.0, np.max(np.abs(w_q))))
    assert worst < 1e-9


def test_barycentric_invariants():
    """Sec. 3.1: sum_i w_i = 1 and sum_i w_i v_i = p (reproduces the pixel)."""
    rng = np.random.default_rng(3)
    for _ in range(2000):
        tri = rng.uniform(-1, 1, 6)
        u, v = rng.uniform(-1.5, 1.5, 2)
        w, det = oracle.barycentric(tri, u, v)
        if abs(det) < 1e-3:
            continue
        assert abs(w.sum() - 1.0) < 1e-12
        assert abs(w @ tri[0::2] - u) < 1e-12 and abs(w @ tri[1::2] - v) < 1e-12
        assert abs(det - np.linalg.det(np.array([tri[0::2], tri[1::2], [1, 1, 1]]))) < 1e-12


# ----------------------------------------------------------------------------- closest point

def _segment_min_dense(a, b, p, n=200001):
    t = np.linspace(0.0, 1.0, n)
    q = a[None, :] + t[:, None] * (b - a)[None, :]
    d = np.sum((q - p[None, :]) ** 2, axis=1)
    return d.min()


def test_closest_point_matches_dense_boundary_sampling():
    """Appendix (Euclidean distance approximation): for points outside the triangle the three
    clamped edge projections give the exact squared distance; checked against dense sampling of
    the boundary (2e5 points per edge; sampling error <= (edge/2e5)^2 / 4)."""
    rng = np.random.default_rng(11)
    checked = 0
    while checked < 60:
        tri = rng.uniform(-1, 1, 6)
        p = rng.uniform(-1.5, 1.5, 2)
        w, det = oracle.barycentric(tri, *p)
        if abs(det) < 1e-2 or np.all(w >= 0):
            continue
        d2, wstar, region = oracle.closest_point(tri, *p)
        V = tri.reshape(3, 2)
        dense = min(_segment_min_dense(V[i], V[(i + 1) % 3], p) for i in range(3))
        assert abs(d2 - dense) < 1e-9
        assert abs(wstar.sum() - 1.0) < 1e-15 and np.all(wstar >= 0)
        q = wstar @ V
        assert abs(np.sum((q - p) ** 2) - d2) < 1e-12
        checked += 1


# ----------------------------------------------------------------------------- normals / motion / camera

def test_vertex_normals_octahedron_closed_form():
    """Area-weighted vertex normals: on a regular octahedron every vertex normal is the vertex
    direction exactly (by symmetry of the four incident faces)."""
    v = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)
    f = np.array([[0, 2, 4], [2, 1, 4], [1, 3, 4], [3, 0, 4], [2, 0, 5], [1, 2, 5], [3, 1, 5], [0, 3, 5]],
                 dtype=np.int32)
    sc = scenes.scene(v, f, np.full_like(v, 0.5), scenes.translate((0, 0, 0)),
                      scenes.camera(scenes.look_at((0, 0, -4))), 1, 8, 8)
    n = oracle.vertex_normals(sc)
    assert np.allclose(n, v, atol=1e-15)


def test_vertex_normals_weight_faces_by_area():
    """Vertex normals are the normalised sum of the incident faces' UN-normalised cross products
    (area weighting).  Vertex 0 touches a face of area 2 with normal +z and a face of area 1/2
    with normal -x, so its normal is (-1, 0, 4) / sqrt(17), computed by hand.  The other common
    rules give different vectors here and would fail: the unweighted mean of unit face normals is
    (-1, 0, 1) / sqrt(2), and the angle-weighted mean (incident angles 90 and 26.57 degrees) is
    about (-0.283, 0, 0.959)."""
    v = np.array([[0, 0, 0], [2, 0, 0], [0, 2, 0], [0, 1, -0.5]], float)
    f = np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32)
    sc = scenes.scene(v, f, np.full_like(v, 0.5), scenes.translate((0, 0, 0)),
                      scenes.camera(scenes.look_at((0, 0, -4))), 1, 8, 8)
    n = oracle.vertex_normals(sc)
    area = np.array([-1.0, 0.0, 4.0]) / math.sqrt(17.0)
    assert np.allclose(n[0], area, atol=1e-15) and np.allclose(n[2], area, atol=1e-15)
    assert np.allclose(n[1], [0, 0, 1], atol=1e-15) and np.allclose(n[3], [-1, 0, 0], atol=1e-15)
    # the rejected rules really are far from the pinned value at vertex 0
    assert np.linalg.norm(area - np.array([-1.0, 0.0, 1.0]) / math.sqrt(2.0)) > 0.5
    ang = np.array([-math.atan2(1.0, 2.0), 0.0, math.pi / 2])
    assert np.linalg.norm(area - ang / np.linalg.norm(ang)) > 0.04


def _screen_quad(x0, x1, y0, y1, zc, th):
    """World vertices (camera at (0, 0, -4) looking along +z) of a quad facing the camera whose
    screen extent is [x0, x1] x [y0, y1] at camera depth zc; faces wound so the normal is -z."""
    wz = zc - 4.0
    v = np.array([[x0 * zc * th, y0 * zc * th, wz], [x1 * zc * th, y0 * zc * th, wz],
                  [x1 * zc * th, y1 * zc * th, wz], [x0 * zc * th, y1 * zc * th, wz]], float)
    return v, np.array([[0, 2, 1], [0, 3, 2]], dtype=np.int32)


def _two_quads(va, fa, ca, vb, fb, cb, a_first, W=64, H=48):
    """One static scene of two quads with their own vertices and constant albedos; faces of
    quad A listed first (a_first) or second."""
    parts = [(va, fa, ca), (vb, fb, cb)] if a_first else [(vb, fb, cb), (va, fa, ca)]
    verts, faces, alb, off = [], [], [], 0
    for v, f, c in parts:
        verts.append(v)
        faces.append(f + off)
        alb.append(np.tile(np.asarray(c, float), (len(v), 1)))
        off += len(v)
    return scenes.scene(np.vstack(verts), np.vstack(faces), np.vstack(alb), scenes.translate((0, 0, 0)),
                        scenes.camera(scenes.look_at((0, 0, -4))), 1, H, W)


def _lambert(cam, n):
    L = np.asarray(cam["light_dir"], float) / np.linalg.norm(cam["light_dir"])
    n = np.asarray(n, float) / np.linalg.norm(n)
    return cam["k_ambient"] + cam["k_diffuse"] * max(0.0, float(n @ L))


def _pixel_centres(H, W):
    u = (2 * (np.arange(W) + 0.5) / W - 1)[None, :].repeat(H, 0)
    v = (1 - 2 * (np.arange(H) + 0.5) / H)[:, None].repeat(W, 1)
    return u, v


@pytest.mark.parametrize("a_first", [True, False])
def test_ztest_nearer_quad_wins_the_overlap(a_first):
    """Sec. 3.1 z-test: two overlapping screen-aligned quads, A at camera depth 3 (near, red) and
    B at depth 5 (far, blue).  Pixels inside both show A's closed-form Lambert colour, whichever
    quad's faces are listed first; pixels inside one quad show that quad.  A reversed test
    (farthest wins) would show B in the overlap, and a first-listed-wins rule would flip with the
    listing order."""
    th = math.tan(math.radians(20))
    ax0, ax1, ay0, ay1 = -0.61, 0.23, -0.43, 0.37
    bx0, bx1, by0, by1 = -0.17, 0.69, -0.29, 0.53
    va, fa = _screen_quad(ax0, ax1, ay0, ay1, 3.0, th)
    vb, fb = _screen_quad(bx0, bx1, by0, by1, 5.0, th)
    ca, cb = (0.8, 0.25, 0.2), (0.2, 0.3, 0.85)
    sc = _two_quads(va, fa, ca, vb, fb, cb, a_first)
    img = oracle.render(sc, "exact")["rgba"]
    shade = _lambert(sc["camera"], (0, 0, -1))
    u, v = _pixel_centres(sc["H"], sc["W"])
    in_a = (u >= ax0) & (u <= ax1) & (v >= ay0) & (v <= ay1)
    in_b = (u >= bx0) & (u <= bx1) & (v >= by0) & (v <= by1)
    assert (in_a & in_b).sum() > 100 and (in_b & ~in_a).sum() > 50
    assert np.abs(img[in_a][:, :3] - shade * np.array(ca)).max() < 1e-12
    assert np.abs(img[in_b & ~in_a][:, :3] - shade * np.array(cb)).max() < 1e-12
    assert np.abs(img[in_a | in_b][:, 3] - 1.0).max() < 1e-12


@pytest.mark.parametrize("a_first", [True, False])
def test_ztest_exact_depth_tie_goes_to_the_smaller_face_id(a_first):
    """Sec. 3.1 z-test tie rule: quad B duplicates quad A's geometry exactly (its own vertices,
    bit-identical positions, same winding) with another colour.  Every covered pixel is an exact
    depth tie, resolved to the smaller face id, i.e. to the quad listed first: the image shows A
    when A's faces come first and B otherwise."""
    th = math.tan(math.radians(20))
    va, fa = _screen_quad(-0.51, 0.33, -0.41, 0.47, 4.0, th)
    ca, cb = (0.8, 0.25, 0.2), (0.2, 0.3, 0.85)
    sc = _two_quads(va, fa, ca, va.copy(), fa, cb, a_first)
    img = oracle.render(sc, "exact")["rgba"]
    u, v = _pixel_centres(sc["H"], sc["W"])
    inside = (u >= -0.51) & (u <= 0.33) & (v >= -0.41) & (v <= 0.47)
    want = np.array(ca if a_first else cb) * _lambert(sc["camera"], (0, 0, -1))
    assert inside.sum() > 300
    assert np.abs(img[inside][:, :3] - want).max() < 1e-12


def _affine_z_winner(sc, u, v):
    """The REJECTED rule, for contrast: per pixel, the face whose screen-space (affine)
    interpolation of vertex camera depths sum_i w_i z_i is smallest.  Returns face ids (-1: none)."""
    st = oracle.vertex_state(sc, 0.5)
    best = np.full(u.shape, np.inf)
    win = np.full(u.shape, -1)
    for fi, (a, b, c) in enumerate(sc["faces"]):
        P = st[[a, b, c]]
        M = np.array([P[:, 0], P[:, 1], np.ones(3)])
        w = np.linalg.solve(M, np.stack([u.ravel(), v.ravel(), np.ones(u.size)])).T.reshape(u.shape + (3,))
        inside = (w >= 0).all(-1)
        z = w @ P[:, 2]
        take = inside & (z < best)
        best[take] = z[take]
        win[take] = fi
    return win


@pytest.mark.parametrize("a_first", [True, False])
def test_ztest_uses_perspective_correct_depth(a_first):
    """Sec. 3.1 z-test with a tilted quad: B lies in the camera-space plane z_c = 4 + x_c / 2 and
    crosses the screen-aligned quad A (z_c = 4) at x_c = 0.  On screen, B's true depth is
    z_c(u) = 4 / (1 - u tan(20 deg) / 2), nearer than A exactly where u < 0, so the overlap shows
    B's colour left of u = 0 and A's colour right of it.  The perspective-correct key
    sum_i w_i / z_i is exactly 1 / z_c for planar faces and reproduces this.  An affine depth
    key sum_i w_i z_i moves the crossing by several pixels: the test checks that it would fail."""
    th = math.tan(math.radians(20))
    va, fa = _screen_quad(-0.6, 0.6, -0.5, 0.5, 4.0, th)
    xc = np.array([-1.2, 1.2, 1.2, -1.2])
    zc = 4.0 + 0.5 * xc
    yc = np.array([-0.35, -0.35, 0.35, 0.35]) * 4.0 * th
    vb = np.stack([xc, yc, zc - 4.0], 1)
    fb = np.array([[0, 2, 1], [0, 3, 2]], dtype=np.int32)
    ca, cb = (0.8, 0.25, 0.2), (0.2, 0.3, 0.85)
    sc = _two_quads(va, fa, ca, vb, fb, cb, a_first)
    img = oracle.render(sc, "exact")["rgba"]
    cam = sc["camera"]
    col_a = np.array(ca) * _lambert(cam, (0, 0, -1))
    col_b = np.array(cb) * _lambert(cam, (0.5, 0, -1))
    u, v = _pixel_centres(sc["H"], sc["W"])
    # B's screen footprint: x from its projected left to right edge, |y| below its edges' projection
    zb = 4.0 / (1.0 - 0.5 * th * u)
    in_b = (zb * th * u >= -1.2) & (zb * th * u <= 1.2) & (np.abs(v) * zb * th <= 0.35 * 4.0 * th)
    in_a = (np.abs(u) <= 0.6) & (np.abs(v) <= 0.5)
    both = in_a & in_b
    left, right = both & (u < 0), both & (u > 0)
    assert left.sum() > 100 and right.sum() > 100
    assert np.abs(img[left][:, :3] - col_b).max() < 1e-12
    assert np.abs(img[right][:, :3] - col_a).max() < 1e-12
    # the affine key picks the wrong quad on a band of overlap pixels
    ids = _affine_z_winner(sc, u, v)
    b_ids = {2, 3} if a_first else {0, 1}
    affine_b = np.isin(ids, list(b_ids))
    assert ((affine_b != (u < 0)) & both).sum() >= 40


def test_camera_optical_axis_and_fov_edge():
    """Camera (scene settings): a point on the optical axis projects to (0, 0); a point at the
    half-FOV angle projects to ndc 1; camera z is the distance along the view direction."""
    th = math.tan(math.radians(20))
    pts = np.array([[0, 0, 0], [4 * th, 0, 0], [0, -4 * th, 0], [2 * th * 3, 0, 2.0]], float)
    f = np.array([[0, 1, 2]], dtype=np.int32)
    sc = scenes.scene(pts, np.array([[0, 1, 2], [1, 2, 3]], dtype=np.int32), np.full_like(pts, 0.5),
                      scenes.translate((0, 0, 0)), scenes.camera(scenes.look_at((0, 0, -4))), 1, 8, 8)
    st = oracle.vertex_state(sc, 0.0)
    assert np.allclose(st[0, :3], [0, 0, 4])
    assert np.allclose(st[1, :3], [1, 0, 4])
    assert np.allclose(st[2, :3], [0, -1, 4])
    assert np.allclose(st[3, :3], [1, 0, 6])
    del f


def test_motion_translation_and_rotation():
    """Motion parameters: translation moves v to v + o + t d; rotation about +y by a quarter turn
    maps +x to -z (right-handed, matching the parabolic-motion formula), a full turn is the
    identity, and the axis itself is fixed."""
    v = np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]])
    f = np.array([[0, 1, 2]], dtype=np.int32)
    cam = scenes.camera(scenes.look_at((0, 0, -4)))
    th = cam["tan_half_fov"]
    sc = scenes.scene(v, f, np.full_like(v, 0.5), scenes.rotate((0, 1, 0), 2 * math.pi), cam, 1, 8, 8)
    s0, s1, sq = oracle.vertex_state(sc, 0.0), oracle.vertex_state(sc, 1.0), oracle.vertex_state(sc, 0.25)
    assert np.allclose(s0, s1, atol=1e-12)
    # +x rotated a quarter turn about +y lands at -z: ndc (0, 0), camera z = 4 - 1
    assert np.allclose(sq[0, :3], [0, 0, 3.0], atol=1e-12)
    assert np.allclose(sq[1, :3], s0[1, :3], atol=1e-12)  # on the axis
    # +z lands at +x: x_c = 1, z_c = 4
    assert np.allclose(sq[2, :3], [1 / (4 * th), 0, 4.0], atol=1e-12)
    sct = scenes.scene(v, f, np.full_like(v, 0.5), scenes.translate((0.8, 0.0, 0.0)), cam, 1, 8, 8)
    a, b = oracle.vertex_state(sct, 0.0), oracle.vertex_state(sct, 1.0)
    # v + o (o = -d/2) and v + o + d: screen x differs by d / (z tan)
    assert np.allclose(b[:, 0] - a[:, 0], 0.8 / (a[:, 2] * th))
    assert np.allclose(a[0, 0], (1 - 0.4) / (4 * th))


def test_sample_times_and_segments():
    """Sec. 3.2: t_k = k/(K-1) with both endpoints; Sec. 3.3: 12 segments per turn, t = (s+tau)/S."""
    sc = scenes.small_scene("rotate", T=64)
    assert oracle.num_segments(sc) == 12
    ts = [oracle.sample_time(sc, k) for k in range(64)]
    for k, (s, t, tau) in enumerate(ts):
        assert abs(t - k / 63) < 1e-15
        assert 0 <= s < 12 and 0.0 <= tau <= 1.0
        assert abs((s + tau) / 12 - t) < 1e-14
    assert ts[-1][0] == 11 and ts[-1][2] == 1.0
    one = dict(sc, T=1)
    assert oracle.sample_time(one, 0)[1] == 0.5
    mid = dict(sc, camera=dict(sc["camera"], time_rule="midpoint"))
    assert abs(oracle.sample_time(mid, 0)[1] - 0.5 / 64) < 1e-15
    tr = scenes.small_scene("translate")
    assert oracle.num_segments(tr) == 1
    # omega = 2 pi rounded to single precision (how the CUDA path receives it) is still 12 segments
    f32 = dict(sc, motion=dict(sc["motion"], omega=float(np.float32(2 * math.pi))))
    assert oracle.num_segments(f32) == 12
    assert oracle.num_segments(dict(sc, motion=dict(sc["motion"], omega=16 * math.pi))) == 96


# ----------------------------------------------------------------------------- special cases

def _static_copy(sc, t):
    """The scene with the motion at time t baked into the base vertices and no motion left."""
    m = sc["motion"]
    v = sc["verts"]
    if m["kind"] == "translate":
        v = v + m["offset"] + t * m["dir"]
    else:
        k = np.asarray(m["axis"], float) / np.linalg.norm(m["axis"])
        th = m["omega"] * t
        K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
        R = np.eye(3) + math.sin(th) * K + (1 - math.cos(th)) * K @ K
        v = v @ R.T
    return dict(sc, verts=v, motion=scenes.translate((0, 0, 0)), T=1)


@pytest.mark.parametrize("kind", ["rotate", "translate"])
@pytest.mark.parametrize("mode", ["exact", "linear", "fast"])
def test_single_subframe_equals_static_render(kind, mode):
    """T = 1 renders the pose at t = 0.5, equal to a static render of that pose.  In fast mode the
    background distance is measured through keyframe F(X) (Eq. euc-dist-approx-2), which a moving
    scene does not share with its static copy, so there only the foreground must agree."""
    sc = dict(scenes.small_scene(kind, T=1, H=33, W=47), T=1)
    a = oracle.render(sc, mode)["rgba"]
    b = oracle.render(_static_copy(sc, 0.5), mode)["rgba"]
    ch = slice(0, 3) if mode == "fast" else slice(0, 4)
    assert np.max(np.abs(a[..., ch] - b[..., ch])) < 1e-12
    assert a[..., 3].max() > 0.99  # the object is in view


def _quad_scene(T, D, L0=-0.37, R0=0.113, B=-0.29, Tp=0.41, H=24, W=40, rule="paper"):
    cam = scenes.camera(scenes.look_at((0, 0, -4)), time_rule=rule)
    th = cam["tan_half_fov"]
    z = 4.0
    # world quad in the plane z = 0 whose screen extent at t = 0 is [L0, R0] x [B, Tp]
    xs = np.array([L0, R0]) * z * th
    ys = np.array([B, Tp]) * z * th
    v = np.array([[xs[0], ys[0], 0], [xs[1], ys[0], 0], [xs[1], ys[1], 0], [xs[0], ys[1], 0]], float)
    f = np.array([[0, 2, 1], [0, 3, 2]], dtype=np.int32)
    d = D * z * th  # world translation giving a screen shift of D
    return scenes.scene(v, f, np.full((4, 3), 0.6), scenes.translate((d, 0, 0), offset=(0, 0, 0)), cam, T, H, W)


def _quad_counts(sc, L0, R0, B, Tp, D):
    """#{k : L0 + t_k D <= u <= R0 + t_k D} for every pixel centre inside [B, Tp] vertically,
    computed by enumerating the sample times."""
    H, W, T = sc["H"], sc["W"], sc["T"]
    u = 2 * (np.arange(W) + 0.5) / W - 1
    v = 1 - 2 * (np.arange(H) + 0.5) / H
    t = np.arange(T) / (T - 1) if sc["camera"]["time_rule"] == "paper" else (np.arange(T) + 0.5) / T
    inside = (u[None, :] >= L0 + t[:, None] * D) & (u[None, :] <= R0 + t[:, None] * D)
    cnt = inside.sum(0)
    rows = (v >= B) & (v <= Tp)
    return rows[:, None] * cnt[None, :]


@pytest.mark.parametrize("mode", ["exact", "linear", "fast"])
def test_translating_quad_box_count_closed_form(mode):
    """A constant-colour, screen-aligned quad translating along x: pixel RGB = c_full * n/T with
    n the number of sample times whose shifted quad covers the pixel centre."""
    L0, R0, B, Tp, D = -0.37, 0.113, -0.29, 0.41, 0.6131
    sc = _quad_scene(17, D, L0, R0, B, Tp)
    img = oracle.render(sc, mode)["rgba"]
    cam = sc["camera"]
    # one covered sample: albedo 0.6 under Lambert with the quad normal (0, 0, -1) facing the camera
    full = 0.6 * (cam["k_ambient"] + cam["k_diffuse"] * -cam["light_dir"][2] / np.linalg.norm(cam["light_dir"]))
    cnt = _quad_counts(sc, L0, R0, B, Tp, D)
    assert np.max(np.abs(img[..., 0] - full * cnt / sc["T"])) < 1e-12
    assert np.max(np.abs(img[..., :3] - img[..., :1])) < 1e-12  # grey albedo -> equal channels
    covered = cnt > 0
    assert np.all(img[..., 3][cnt == sc["T"]] > 1 - 1e-12)
    assert covered.any()


def test_translating_quad_converges_to_box_filter():
    """As T grows the box count tends to the box-filtered edge profile
    |[(u - R0)/D, (u - L0)/D] intersect [0, 1]|, with O(1/T) error."""
    L0, R0, B, Tp, D = -0.37, 0.113, -0.29, 0.41, 0.6131
    T = 4096
    sc = _quad_scene(T, D, L0, R0, B, Tp, H=8, W=40)
    img = oracle.render(sc, "fast")["rgba"]
    full = 0.6 * (sc["camera"]["k_ambient"] + sc["camera"]["k_diffuse"] *
                  0.7 / np.linalg.norm(sc["camera"]["light_dir"]))
    u = 2 * (np.arange(40) + 0.5) / 40 - 1
    prof = np.clip(np.minimum(1.0, (u - L0) / D) - np.maximum(0.0, (u - R0) / D), 0.0, None)
    row = 4  # a row inside [B, Tp]
    assert np.max(np.abs(img[row, :, 0] / full - prof)) < 2.0 / T


def _seg_dist2(px, py, ax, ay, bx, by):
    ex, ey = bx - ax, by - ay
    t = np.clip(((px - ax) * ex + (py - ay) * ey) / (ex * ex + ey * ey), 0.0, 1.0)
    return (px - ax - t * ex) ** 2 + (py - ay - t * ey) ** 2


def test_soft32_counter_is_the_uncovered_terms_above_the_single_precision_cutoff():
    """CNT_SOFT32 (the work measure of the soft term) on a static screen-aligned quad: for every
    pixel outside the quad, each of its two triangles whose squared distance is below
    delta 25 ln 2 (exp(-d/delta) > 2^-25) counts once per sample; pixels inside count nothing."""
    L0, R0, B, Tp = -0.37, 0.113, -0.29, 0.41
    T, delta = 3, 4e-3
    sc = _quad_scene(T, 0.0, L0, R0, B, Tp)
    sc["camera"]["delta"] = delta
    c = oracle.render(sc, "exact")["counters"]
    H, W = sc["H"], sc["W"]
    u = (2 * (np.arange(W) + 0.5) / W - 1)[None, :].repeat(H, 0)
    v = (1 - 2 * (np.arange(H) + 0.5) / H)[:, None].repeat(W, 1)
    BL, BR, TR, TL = (L0, B), (R0, B), (R0, Tp), (L0, Tp)
    inside = (u >= L0) & (u <= R0) & (v >= B) & (v <= Tp)
    n = np.zeros((H, W), dtype=np.int64)
    for tri in ((BL, TR, BR), (BL, TL, TR)):
        d2 = np.min([_seg_dist2(u, v, *tri[q], *tri[(q + 1) % 3]) for q in range(3)], axis=0)
        n += (d2 < delta * 25 * np.log(2)) & ~inside
    assert c[oracle.CNT_SOFT32] == T * n.sum() > 0
    assert c[oracle.CNT_SOFT] > c[oracle.CNT_SOFT32]  # the oracle's own truncation reaches farther
    assert c[oracle.CNT_COVERED] == T * inside.sum()


@pytest.mark.parametrize("prob", ["exp", "sigmoid"])
def test_static_quad_soft_alpha_closed_form(prob):
    """Static screen-aligned quad (two triangles): a pixel inside has alpha 1; a pixel outside has
    alpha = 1 - prod over the two triangles of (1 - A(d)), d the squared distance to the triangle
    (the minimum over its edges), A(d) = exp(-d/delta) or sigmoid(-d/delta), terms beyond
    delta ln 1e12 dropped (Eqs. probability-function and back)."""
    L0, R0, B, Tp = -0.37, 0.113, -0.29, 0.41
    T, delta = 2, 4e-3
    sc = _quad_scene(T, 0.0, L0, R0, B, Tp)
    sc["camera"] = dict(sc["camera"], delta=delta, prob=prob)
    a = oracle.render(sc, "exact")["rgba"][..., 3]
    H, W = sc["H"], sc["W"]
    u = (2 * (np.arange(W) + 0.5) / W - 1)[None, :].repeat(H, 0)
    v = (1 - 2 * (np.arange(H) + 0.5) / H)[:, None].repeat(W, 1)
    BL, BR, TR, TL = (L0, B), (R0, B), (R0, Tp), (L0, Tp)
    inside = (u >= L0) & (u <= R0) & (v >= B) & (v <= Tp)
    keep = np.ones((H, W))
    for tri in ((BL, TR, BR), (BL, TL, TR)):
        d2 = np.min([_seg_dist2(u, v, *tri[q], *tri[(q + 1) % 3]) for q in range(3)], axis=0)
        x = d2 / delta
        A = np.exp(-x) if prob == "exp" else 1.0 / (1.0 + np.exp(x))
        keep *= np.where(d2 <= delta * np.log(1e12), 1.0 - A, 1.0)
    expect = np.where(inside, 1.0, 1.0 - keep)
    assert np.max(np.abs(a - expect)) < 1e-12
    if prob == "sigmoid":  # at the quad's edge the SoftRas map gives 1/2 per triangle
        assert np.all(expect[~inside] < 0.75 + 1e-12)


def test_perspective_correct_attributes_are_affine_in_world_space():
    """A static triangle tilted in depth, albedo an affine function of world position: with
    perspective-correct weights every covered pixel shows shade x (alpha . P + beta) at the 3D
    point P where the pixel's ray meets the triangle's plane, the defining property of
    perspective-correct interpolation; screen-space weights (Eq. fore) miss it."""
    tri = np.array([[-1.3, -1.0, -0.9], [1.4, -0.8, 1.1], [0.1, 1.3, 0.3]])
    alpha = np.array([[0.20, -0.10, 0.15], [0.05, 0.12, -0.08], [-0.11, 0.04, 0.10]])
    beta = np.array([0.5, 0.45, 0.55])
    alb = tri @ alpha.T + beta
    view = scenes.look_at((0.0, 0.0, -4.0))
    sc = scenes.scene(tri, np.array([[0, 1, 2]], dtype=np.int32), alb,
                      scenes.translate((0.0, 0.0, 0.0), offset=(0.0, 0.0, 0.0)),
                      scenes.camera(view, interp="perspective"), 1, 36, 44)
    out = oracle.render(sc, "exact", ambig=True)
    rgba, amb = out["rgba"], out["ambig"][0]
    R, tvec = view[:, :3], view[:, 3]
    th = sc["camera"]["tan_half_fov"]
    cam = tri @ R.T + tvec                      # camera-space vertices
    nrm = np.cross(cam[1] - cam[0], cam[2] - cam[0])
    n_world = np.cross(tri[1] - tri[0], tri[2] - tri[0])
    n_world /= np.linalg.norm(n_world)
    L = np.asarray(scenes.LIGHT_DIR) / np.linalg.norm(scenes.LIGHT_DIR)
    shade = scenes.K_AMBIENT + scenes.K_DIFFUSE * max(0.0, float(n_world @ L))
    H, W = sc["H"], sc["W"]
    checked, worst_screen = 0, 0.0
    screen = oracle.render(dict(sc, camera=dict(sc["camera"], interp="screen")), "exact")["rgba"]
    for j in range(H):
        for i in range(W):
            if rgba[j, i, 3] < 1.0 or amb[j, i]:
                continue  # not covered, or within rounding of an edge
            u, v = 2 * (i + 0.5) / W - 1, 1 - 2 * (j + 0.5) / H
            ray = np.array([u * th, v * th, 1.0])
            s_hit = (nrm @ cam[0]) / (nrm @ ray)
            P = R.T @ (s_hit * ray - tvec)        # back to world space
            expect = shade * (alpha @ P + beta)
            assert np.max(np.abs(rgba[j, i, :3] - expect)) < 1e-12, (i, j)
            worst_screen = max(worst_screen, float(np.max(np.abs(screen[j, i, :3] - expect))))
            checked += 1
    assert checked > 200
    assert worst_screen > 1e-3  # the screen-space weights are not perspective-correct here


def test_rotation_relabel_invariance_midpoint_rule():
    """With t_k = (k + 0.5)/T, omega = 2 pi and T a multiple of n, pre-rotating the mesh by 2 pi/n
    about the motion axis permutes the sub-frames and leaves the blurred image unchanged."""
    sc = scenes.small_scene("rotate", T=12, H=30, W=38, time_rule="midpoint")
    n = 4
    m = sc["motion"]
    k = np.asarray(m["axis"])
    th = 2 * math.pi / n
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    R = np.eye(3) + math.sin(th) * K + (1 - math.cos(th)) * K @ K
    sc2 = dict(sc, verts=sc["verts"] @ R.T)
    a = oracle.render(sc, "exact")["rgba"]
    b = oracle.render(sc2, "exact")["rgba"]
    assert np.max(np.abs(a - b)) < 1e-9


def test_full_turn_endpoints_identical_paper_rule():
    """With the paper's t_k = k/(K-1) over one full turn, the first and last sub-frames show the
    same pose: identical z-test winners."""
    sc = scenes.small_scene("rotate", T=7, H=30, W=38)
    r = oracle.render(sc, "exact", winners=True)
    assert np.array_equal(r["winners"][0], r["winners"][-1])


def test_fast_foreground_equals_plain_linear():
    """Sec. 4.1: under linear motion the fast solver's foreground equals per-frame rendering;
    only background alpha differs (distance approximation)."""
    sc = scenes.small_scene("rotate", T=9, H=36, W=44)
    a = oracle.render(sc, "linear", winners=True)
    b = oracle.render(sc, "fast", winners=True)
    assert np.array_equal(a["winners"], b["winners"])
    assert np.max(np.abs(a["rgba"][..., :3] - b["rgba"][..., :3])) == 0.0


def test_linear_screen_motion_exact_equals_linear():
    """Translation perpendicular to the optical axis keeps camera z fixed, so projected motion is
    exactly linear: PLAIN_EXACT and PLAIN_LINEAR agree on the whole image."""
    sc = scenes.config1()
    a = oracle.render(sc, "exact")["rgba"]
    b = oracle.render(sc, "linear")["rgba"]
    assert np.max(np.abs(a - b)) < 1e-12


def test_soft_truncation_bound():
    """Dropping terms with d > delta ln 1e12 changes alpha by at most F * 1e-12."""
    sc = scenes.small_scene("rotate", subdiv=1, T=4, H=20, W=26)
    for mode in ("exact", "fast"):
        a = oracle.render(sc, mode)["rgba"]
        b = oracle.render(sc, mode, soft_all=True)["rgba"]
        assert np.max(np.abs(a - b)) <= len(sc["faces"]) * 1e-12 + 1e-15


def test_single_precision_truncation():
    """soft32 keeps exactly the soft factors above 2^-25: covered samples and colour are untouched
    (RGB identical), alpha moves by at most F 2^-25, every term the single-precision counter sees
    is kept, and no term beyond it is."""
    sc = scenes.small_scene("rotate", subdiv=1, T=4, H=20, W=26)
    for mode in ("exact", "fast"):
        a = oracle.render(sc, mode)
        b = oracle.render(sc, mode, soft32=True)
        assert np.array_equal(a["rgba"][..., :3], b["rgba"][..., :3])
        gap = np.max(np.abs(a["rgba"][..., 3] - b["rgba"][..., 3]))
        assert 0.0 < gap <= len(sc["faces"]) * 2.0 ** -25
        ca, cb = a["counters"], b["counters"]
        assert cb[oracle.CNT_SOFT32] == ca[oracle.CNT_SOFT32]
        assert cb[oracle.CNT_SOFT32] <= cb[oracle.CNT_SOFT] < ca[oracle.CNT_SOFT]
        assert cb[oracle.CNT_COVERED] == ca[oracle.CNT_COVERED]


# ----------------------------------------------------------------------------- brute force

def _seg_min_ternary(a, b, p, iters=100):
    """min_t |a + t (b - a) - p|^2 on [0, 1] by ternary search (vectorised over leading axes)."""
    lo = np.zeros(p.shape[:-1])
    hi = np.ones(p.shape[:-1])
    f = lambda t: np.sum((a + t[..., None] * (b - a) - p) ** 2, axis=-1)
    for _ in range(iters):
        m1 = lo + (hi - lo) / 3
        m2 = hi - (hi - lo) / 3
        left = f(m1) < f(m2)
        hi = np.where(left, m2, hi)
        lo = np.where(left, lo, m1)
    t = 0.5 * (lo + hi)
    return f(t), t


def _brute_force(sc, mode):
    """All pixel x triangle x sample triples, no bounding boxes, no truncation, np.linalg.solve
    barycentrics, closest points by ternary search along the edges."""
    V, F = sc["verts"], sc["faces"]
    T, H, W = sc["T"], sc["H"], sc["W"]
    cam = sc["camera"]
    L = np.asarray(cam["light_dir"]) / np.linalg.norm(cam["light_dir"])
    S = oracle.num_segments(sc)
    u = 2 * (np.arange(W) + 0.5) / W - 1
    v = 1 - 2 * (np.arange(H) + 0.5) / H
    P = np.stack(np.meshgrid(u, v), -1).reshape(-1, 2)
    img = np.zeros((H * W, 4))
    for k in range(T):
        s, t, tau = oracle.sample_time(sc, k)
        if mode == "exact":
            st = oracle.vertex_state(sc, t)
        else:
            k0, k1 = oracle.vertex_state(sc, s / S), oracle.vertex_state(sc, (s + 1) / S)
            st = (1 - tau) * k0 + tau * k1
            X = 0 if tau <= 0.5 else 1
            kx = k0 if X == 0 else k1
        best = np.full(len(P), -np.inf)
        bw = np.zeros((len(P), 3))
        bf = np.full(len(P), -1)
        prod = np.ones(len(P))
        for f in range(len(F)):
            tri = st[F[f]]
            M = np.array([tri[:, 0], tri[:, 1], [1, 1, 1]])
            if abs(np.linalg.det(M)) <= 1e-10:
                continue
            w = np.linalg.solve(M[None], np.concatenate([P, np.ones((len(P), 1))], 1)[..., None])[..., 0]
            cov = np.all(w >= 0, axis=1)
            key = w @ (1 / tri[:, 2])
            upd = cov & ((key > best) | ((key == best) & (f < bf)))
            best[upd], bf[upd], bw[upd] = key[upd], f, w[upd]
            if mode == "fast":
                trx = kx[F[f]][:, :2]
                pp = w @ trx
                base = trx
            else:
                pp = P
                base = tri[:, :2]
            ds, ts = [], []
            for e in range(3):
                d, tt = _seg_min_ternary(base[e][None], base[(e + 1) % 3][None], pp)
                ds.append(d)
                ts.append(tt)
            ds = np.stack(ds, 1)
            ei = np.argmin(ds, 1)
            tt = np.stack(ts, 1)[np.arange(len(P)), ei]
            a_i = tri[ei, :2]
            b_i = tri[(ei + 1) % 3, :2]
            q = a_i + tt[:, None] * (b_i - a_i)
            d = np.sum((P - q) ** 2, 1)
            prod[~cov] *= 1 - np.exp(-d[~cov] / cam["delta"])
        for p in range(len(P)):
            if bf[p] >= 0:
                ids = F[bf[p]]
                col = bw[p] @ sc["albedo"][ids]
                n = bw[p] @ st[ids, 3:6]
                sh = cam["k_ambient"] + cam["k_diffuse"] * max(0.0, n @ L / np.linalg.norm(n))
                img[p, :3] += col * sh
                img[p, 3] += 1
            else:
                img[p, 3] += 1 - prod[p]
    return (img / T).reshape(H, W, 4)


@pytest.mark.parametrize("mode", ["exact", "linear", "fast"])
def test_brute_force_tiny_mesh(mode):
    """Brute-force enumeration on an 8-triangle mesh (octahedron, albedo per vertex) at 12x14 px."""
    rng = np.random.default_rng(5)
    v = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float) * 0.6
    v += rng.normal(0, 0.05, v.shape)
    f = np.array([[0, 2, 4], [2, 1, 4], [1, 3, 4], [3, 0, 4], [2, 0, 5], [1, 2, 5], [3, 1, 5], [0, 3, 5]],
                 dtype=np.int32)
    f = scenes._orient_outward(v, f)
    cam = scenes.camera(scenes.look_at(scenes.orbit_eye(4.0, 20, 10)))
    cam["delta"] = 3e-3  # a wide soft band so the background term is exercised on a 12x14 grid
    sc = scenes.scene(v, f, rng.uniform(0.2, 0.9, (6, 3)), scenes.rotate((0.3, 1, 0.2), 1.3, segments=2),
                      cam, 5, 12, 14)
    a = oracle.render(sc, mode, soft_all=True)["rgba"]
    b = _brute_force(sc, mode)
    assert np.max(np.abs(a - b)) < 1e-9
    assert a[..., 3].max() > 0.5 and (a[..., 3] > 0).mean() < 1.0


def _with_motion(sc, motion):
    return dict(sc, motion=motion)


@pytest.mark.parametrize("mode", ["exact", "linear", "fast"])
def test_parabolic_motion_reduces_to_translation_and_rotation(mode):
    """The parabolic kind with no rotation and no quadratic term is the translation kind, and with
    no translation it is the rotation kind: identical images, bit for bit."""
    sc = scenes.small_scene("translate", subdiv=2, T=6, H=24, W=32, d=(0.7, 0.2, 0.3))
    m = sc["motion"]
    par = scenes.parabolic(axis=(0.0, 1.0, 0.0), omega=0.0, offset=m["offset"], dir=m["dir"], acc=(0.0, 0.0, 0.0))
    a = oracle.render(sc, mode)["rgba"]
    b = oracle.render(_with_motion(sc, par), mode)["rgba"]
    assert np.array_equal(a, b)
    scr = scenes.small_scene("rotate", subdiv=2, T=6, H=24, W=32)
    mr = scr["motion"]
    par = scenes.parabolic(axis=mr["axis"], omega=mr["omega"], offset=(0, 0, 0), dir=(0, 0, 0), acc=(0, 0, 0))
    a = oracle.render(scr, mode)["rgba"]
    b = oracle.render(_with_motion(scr, par), mode)["rgba"]
    assert np.array_equal(a, b)


def test_parabolic_trajectory_is_quadratic():
    """With omega = 0 a vertex moves on a quadratic: its camera-space position has a constant second
    difference 2 acc h^2 (the camera is an affine map), and a zero one for acc = 0."""
    sc = scenes.small_scene("translate", subdiv=1, T=4, H=16, W=16)
    cam = sc["camera"]
    R = np.asarray(cam["view"]).reshape(3, 4)[:, :3]
    acc = np.array([0.3, -4.0, 0.2])
    par = scenes.parabolic(omega=0.0, offset=(0.1, 0.2, 0.0), dir=(-1.0, 4.0, -1.0), acc=acc)
    s = _with_motion(sc, par)
    th = cam["tan_half_fov"]

    def camera_pos(t):
        st = oracle.vertex_state(s, t)  # ndc x, ndc y, camera z
        z = st[:, 2]
        return np.stack([st[:, 0] * z * th, st[:, 1] * z * th, z], 1)

    h = 0.125
    for t in (0.25, 0.5, 0.75):
        d2 = camera_pos(t + h) - 2 * camera_pos(t) + camera_pos(t - h)
        assert np.allclose(d2, (R @ (2 * acc * h * h))[None, :], atol=1e-9)
    # the appendix's trajectory: T(t) = (s, -4 s^2 + 0.5, s), s = 0.5 - t, peaks at t = 0.5
    pap = scenes.parabolic(omega=0.0)
    s2 = _with_motion(sc, pap)
    p = {t: oracle.vertex_state(s2, t) for t in (0.0, 0.5, 1.0)}
    disp = lambda t: (lambda st: np.stack([st[:, 0] * st[:, 2] * th, st[:, 1] * st[:, 2] * th, st[:, 2]], 1))(p[t])
    up = disp(0.5) - 0.5 * (disp(0.0) + disp(1.0))
    assert np.allclose(up, (R @ np.array([0.0, 1.0, 0.0]))[None, :], atol=1e-9)  # +1 in world y at mid-exposure


# ----------------------------------------------------------------------------- textures

def _textured_quad(tex, T=1, D=0.0, L0=-0.55, R0=0.45, B=-0.4, Tp=0.52, H=30, W=40, uv_box=(0.0, 1.0, 0.0, 1.0)):
    """Static (or translating) screen-aligned quad whose corners carry uv = the corners of
    ``uv_box`` (u0, u1, v0, v1): u grows to the right, v grows downwards on screen."""
    sc = _quad_scene(T, D, L0, R0, B, Tp, H=H, W=W)
    u0, u1, v0, v1 = uv_box
    # quad corners: 0 = (L0, B), 1 = (R0, B), 2 = (R0, Tp), 3 = (L0, Tp)
    sc["uv"] = np.array([[u0, v1], [u1, v1], [u1, v0], [u0, v0]], float)
    sc["texture"] = np.asarray(tex, float)
    return sc


def test_texture_affine_in_texel_space_is_reproduced():
    """A texture whose texels are an affine function of their indices (value a + b x + c y at
    texel (x, y)) is reproduced exactly by the bilinear lookup between texel centres, and the
    uv of a screen-aligned quad is affine in screen space: every covered pixel shows
    shade x (a + b X + c Y), X = u tw - 1/2, Y = v th - 1/2 (clamped to the texel-centre range)."""
    th, tw = 6, 9
    ys, xs = np.meshgrid(np.arange(th), np.arange(tw), indexing="ij")
    coef = np.array([[0.30, 0.05, 0.02], [0.55, -0.03, 0.04], [0.20, 0.02, 0.06]])
    tex = np.stack([c[0] + c[1] * xs + c[2] * ys for c in coef], axis=-1)
    L0, R0, B, Tp = -0.55, 0.45, -0.4, 0.52
    sc = _textured_quad(tex, L0=L0, R0=R0, B=B, Tp=Tp)
    out = oracle.render(sc, "exact", winners=True, ambig=True)
    rgba = out["rgba"]
    covered = (out["winners"][0] >= 0) & (out["ambig"][0] == 0)
    H, W = sc["H"], sc["W"]
    n = np.array([0.0, 0.0, 1.0])
    L = np.asarray(scenes.LIGHT_DIR) / np.linalg.norm(scenes.LIGHT_DIR)
    shades = [scenes.K_AMBIENT + scenes.K_DIFFUSE * max(0.0, s * float(n @ L)) for s in (1.0, -1.0)]
    checked = 0
    for j in range(H):
        for i in range(W):
            if not covered[j, i]:
                continue
            x, y = 2 * (i + 0.5) / W - 1, 1 - 2 * (j + 0.5) / H
            u = (x - L0) / (R0 - L0)
            v = (Tp - y) / (Tp - B)
            X = np.clip(u * tw - 0.5, 0, tw - 1)
            Y = np.clip(v * th - 0.5, 0, th - 1)
            val = coef[:, 0] + coef[:, 1] * X + coef[:, 2] * Y
            err = min(np.max(np.abs(rgba[j, i, :3] - sh * val)) for sh in shades)
            assert err < 1e-12, (i, j, err)
            checked += 1
    assert checked > 200


def test_texture_gradient_is_exact_and_vertex_gradient_matches_differences():
    """L is linear in the texels: dL/dtexture equals the change of L for a unit texel step.  The
    vertex gradient through uv interpolation and the texture slope matches central differences
    (skipping steps that move a sample across a texel cell, part of the decision hash)."""
    rng = np.random.default_rng(5)
    th, tw = 5, 7
    tex = rng.uniform(0.1, 0.9, size=(th, tw, 3))
    sc = _textured_quad(tex, T=4, D=0.3, uv_box=(0.1, 0.85, 0.05, 0.9))
    G = rng.normal(size=(sc["H"], sc["W"], 4))
    gt = np.zeros_like(tex)
    gv, _, _ = oracle.render_backward(sc, G, "exact", texture_grad=gt)

    def loss(s):
        r = oracle.render(s, "exact")
        return float(np.sum(r["rgba"] * G)), int(r["counters"][oracle.CNT_HASH])

    l0, h0 = loss(sc)
    for (y, x, c) in [(0, 0, 0), (2, 3, 1), (4, 6, 2), (1, 5, 0)]:
        t2 = tex.copy()
        t2[y, x, c] += 1.0
        l1, _ = loss(dict(sc, texture=t2))
        assert abs((l1 - l0) - gt[y, x, c]) < 1e-9 * max(1.0, abs(gt[y, x, c]))
    h = 1e-6
    checked = 0
    for v in range(4):
        for c in range(2):
            p, m = dict(sc, verts=sc["verts"].copy()), dict(sc, verts=sc["verts"].copy())
            p["verts"][v, c] += h
            m["verts"][v, c] -= h
            (lp, hp), (lm, hm) = loss(p), loss(m)
            if hp != h0 or hm != h0:
                continue
            fd = (lp - lm) / (2 * h)
            assert abs(fd - gv[v, c]) <= 1e-5 * abs(fd) + 1e-7 * np.max(np.abs(gv)), (v, c, fd, gv[v, c])
            checked += 1
    assert checked >= 4
