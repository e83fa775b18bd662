"""Seeded synthetic scene generators shared by the CUDA path's tests/bench and the oracle.

This module holds input generation only: meshes, per-vertex albedo, motion parameters and
camera matrices.  It contains none of the renderer's arithmetic (no projection, no
barycentrics, no shading).  Everything is NumPy and float64; the GPU side casts to float32.

The paper's datasets (ShapeNet, the FMO benchmark, real captures) are not available, so the
scenes below stand in for them with the shapes the paper's experiments use: closed, star-shaped
objects of unit size (every object is scaled so max |v| = 1, Sec. "Object Initialization"),
viewed by a perspective camera, moving by translation or by rotation about an axis through the
object centre ("Motion Parameters").

Scene dictionaries
------------------
``verts``  float64 [V,3]   base (t-independent) vertex positions, world units
``faces``  int32   [F,3]   triangle vertex indices, counter-clockwise seen from outside
``albedo`` float64 [V,3]   per-vertex colour in [0.2, 0.9]
``motion`` dict: kind ('translate'|'rotate'), offset[3], dir[3], axis[3], omega, segments
``camera`` dict: view (3x4 world->camera, +z forward), tan_half_fov, znear, light_dir[3],
           k_ambient, k_diffuse, delta, time_rule ('paper'|'midpoint')
``T, H, W`` sub-frames and image size
"""
from __future__ import annotations

import math

import numpy as np

MASTER_SEED = 20260207

# Paper constants (Sec. "Hyperparameter Settings": delta = 1e-4; Sec. 3.3: 12 segments per turn).
DELTA = 1e-4
SEGMENTS_PER_TURN = 12
# Shading constants of the Lambertian reading (the paper's Eq. "fore" interpolates attributes only).
K_AMBIENT = 0.3
K_DIFFUSE = 0.7
LIGHT_DIR = (0.4, 0.6, -0.7)
ZNEAR = 0.1


# ----------------------------------------------------------------------------- meshes

def icosphere(subdiv: int):
    """Unit icosphere: icosahedron subdivided ``subdiv`` times, vertices projected to |v| = 1.

    subdiv 0/1/2/3/4/5 -> 12/42/162/642/2562/10242 vertices, 20/80/320/1280/5120/20480 faces.
    """
    p = (1.0 + math.sqrt(5.0)) / 2.0
    verts = [(-1, p, 0), (1, p, 0), (-1, -p, 0), (1, -p, 0),
             (0, -1, p), (0, 1, p), (0, -1, -p), (0, 1, -p),
             (p, 0, -1), (p, 0, 1), (-p, 0, -1), (-p, 0, 1)]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    verts = [np.array(v, dtype=np.float64) / np.linalg.norm(v) for v in verts]
    for _ in range(subdiv):
        cache = {}
        new_faces = []

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            new_faces += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = new_faces
    v = np.stack(verts)
    f = np.asarray(faces, dtype=np.int32)
    return v, _orient_outward(v, f)


def _orient_outward(v, f):
    """Flip faces whose geometric normal points towards the origin (star-shaped meshes)."""
    a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    n = np.cross(b - a, c - a)
    bad = np.einsum("ij,ij->i", n, a + b + c) < 0
    f = f.copy()
    f[bad] = f[bad][:, [0, 2, 1]]
    return f


def _assoc_legendre(lmax: int, x: np.ndarray):
    """P_l^m(x) for 0<=m<=l<=lmax by the standard upward recurrences (no Condon-Shortley phase)."""
    P = {}
    sx = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    P[(0, 0)] = np.ones_like(x)
    for m in range(1, lmax + 1):
        P[(m, m)] = P[(m - 1, m - 1)] * (2 * m - 1) * sx
    for m in range(0, lmax):
        P[(m + 1, m)] = x * (2 * m + 1) * P[(m, m)]
    for m in range(0, lmax + 1):
        for l in range(m + 2, lmax + 1):
            P[(l, m)] = ((2 * l - 1) * x * P[(l - 1, m)] - (l + m - 1) * P[(l - 2, m)]) / (l - m)
    return P


def real_sh(lmax: int, dirs: np.ndarray) -> np.ndarray:
    """Real orthonormal spherical harmonics Y_lm at unit directions; returns [(lmax+1)^2, N]."""
    x, y, z = dirs[:, 0], dirs[:, 1], dirs[:, 2]
    phi = np.arctan2(y, x)
    P = _assoc_legendre(lmax, np.clip(z, -1.0, 1.0))
    out = []
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            k = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
            if m == 0:
                out.append(k * P[(l, 0)])
            elif m > 0:
                out.append(math.sqrt(2) * k * P[(l, am)] * np.cos(am * phi))
            else:
                out.append(math.sqrt(2) * k * P[(l, am)] * np.sin(am * phi))
    return np.stack(out)


def sh_displace(verts: np.ndarray, lmax: int, sigma: float, rng: np.random.Generator) -> np.ndarray:
    """Radial displacement r = max(0.2, 1 + sum c_lm Y_lm), c_lm ~ N(0, sigma); rescaled to max|v| = 1."""
    dirs = verts / np.linalg.norm(verts, axis=1, keepdims=True)
    Y = real_sh(lmax, dirs)
    c = rng.normal(0.0, sigma, size=Y.shape[0])
    r = np.maximum(0.2, 1.0 + c @ Y)
    v = dirs * r[:, None]
    return v / np.max(np.linalg.norm(v, axis=1))


def _bspline_basis(knots, degree, x):
    """Cox-de Boor basis functions N_{i,degree}(x); returns [n_basis, len(x)]."""
    n = len(knots) - degree - 1
    x = np.asarray(x, dtype=np.float64)
    B = np.zeros((len(knots) - 1, x.size))
    for i in range(len(knots) - 1):
        B[i] = (knots[i] <= x) & (x < knots[i + 1])
    # include the right end point in the last non-empty span
    last = np.max(np.nonzero(knots[:-1] < knots[1:])[0])
    B[last, x >= knots[-1]] = 1.0
    for d in range(1, degree + 1):
        Bn = np.zeros((len(knots) - 1 - d, x.size))
        for i in range(len(knots) - 1 - d):
            a = knots[i + d] - knots[i]
            b = knots[i + d + 1] - knots[i + 1]
            t1 = (x - knots[i]) / a * B[i] if a > 0 else 0.0
            t2 = (knots[i + d + 1] - x) / b * B[i + 1] if b > 0 else 0.0
            Bn[i] = t1 + t2
        B = Bn
    return B[:n]


def surface_of_revolution(n_theta: int, n_rings: int, rng: np.random.Generator, n_ctrl: int = 12,
                          bump_sigma: float = 0.1, bump_amp: float = 0.15):
    """Closed surface of revolution about +y with a radius profile from a clamped cubic B-spline
    (``n_ctrl`` control radii ~ U[0.3, 1]) and one Gaussian bump (sigma in (theta, y) units) that
    breaks the rotational symmetry.  Grid of n_theta x (n_rings-1) quads (2 triangles each) plus
    two polar fans; the result is scaled so max |v| = 1.
    """
    ctrl = rng.uniform(0.3, 1.0, size=n_ctrl)
    deg = 3
    inner = np.linspace(0.0, 1.0, n_ctrl - deg + 1)
    knots = np.concatenate([[0.0] * deg, inner, [1.0] * deg])
    s = np.linspace(0.0, 1.0, n_rings)
    prof = ctrl @ _bspline_basis(knots, deg, s)
    ys = np.linspace(-1.0, 1.0, n_rings)
    # taper the profile to zero radius at the poles so the surface closes smoothly
    prof = prof * np.sqrt(np.maximum(0.0, 1.0 - ys ** 2)) ** 0.5
    th = np.arange(n_theta) * (2 * math.pi / n_theta)
    b_th = rng.uniform(0, 2 * math.pi)
    b_y = rng.uniform(-0.6, 0.6)
    dth = np.angle(np.exp(1j * (th[None, :] - b_th)))
    bump = bump_amp * np.exp(-(dth ** 2 + (ys[:, None] - b_y) ** 2) / (2 * bump_sigma ** 2))
    r = prof[:, None] * (1.0 + bump)
    ring = np.stack([r * np.cos(th)[None, :], np.broadcast_to(ys[:, None], r.shape),
                     -r * np.sin(th)[None, :]], axis=-1)
    # drop the degenerate first/last rings (radius 0) and close with pole vertices instead
    ring = ring[1:-1]
    nr = ring.shape[0]
    verts = ring.reshape(-1, 3)
    south = len(verts)
    north = south + 1
    verts = np.concatenate([verts, [[0.0, -1.0, 0.0], [0.0, 1.0, 0.0]]])
    faces = []
    idx = np.arange(nr * n_theta).reshape(nr, n_theta)
    for i in range(nr - 1):
        a = idx[i]
        b = idx[i + 1]
        a1 = np.roll(a, -1)
        b1 = np.roll(b, -1)
        faces.append(np.stack([a, b, a1], 1))
        faces.append(np.stack([a1, b, b1], 1))
    first, last = idx[0], idx[-1]
    faces.append(np.stack([np.full(n_theta, south), first, np.roll(first, -1)], 1))
    faces.append(np.stack([np.full(n_theta, north), np.roll(last, -1), last], 1))
    f = np.concatenate(faces).astype(np.int32)
    v = verts / np.max(np.linalg.norm(verts, axis=1))
    return v, _orient_outward_centroid(v, f)


def uv_sphere(n_theta: int = 50, n_inner: int = 27):
    """Unit UV sphere: n_inner rings of n_theta vertices between two poles, quads split in two and
    polar fans.  The defaults give 1352 vertices and 2700 faces, the size of the template mesh of
    the translational recovery experiment."""
    ys = np.cos(np.linspace(0.0, math.pi, n_inner + 2))[1:-1]
    rs = np.sqrt(np.maximum(0.0, 1.0 - ys ** 2))
    th = np.arange(n_theta) * (2 * math.pi / n_theta)
    ring = np.stack([rs[:, None] * np.cos(th)[None, :], np.broadcast_to(ys[:, None], (n_inner, n_theta)),
                     -rs[:, None] * np.sin(th)[None, :]], axis=-1)
    verts = np.concatenate([ring.reshape(-1, 3), [[0.0, 1.0, 0.0], [0.0, -1.0, 0.0]]], 0)
    north, south = n_inner * n_theta, n_inner * n_theta + 1
    faces = []
    for i in range(n_inner - 1):
        for j in range(n_theta):
            a, b = i * n_theta + j, i * n_theta + (j + 1) % n_theta
            c, d = a + n_theta, b + n_theta
            faces += [[a, c, b], [b, c, d]]
    for j in range(n_theta):
        faces.append([north, j, (j + 1) % n_theta])
        last = (n_inner - 1) * n_theta
        faces.append([south, last + (j + 1) % n_theta, last + j])
    f = np.asarray(faces, dtype=np.int32)
    return verts, _orient_outward_centroid(verts, f)


def _orient_outward_centroid(v, f):
    """Orient faces away from the y axis point at the face's height (surfaces of revolution)."""
    a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    n = np.cross(b - a, c - a)
    cen = (a + b + c) / 3.0
    out = cen.copy()
    out[:, 1] = 0.0
    flat = np.linalg.norm(out, axis=1) < 1e-9
    out[flat] = cen[flat]
    bad = np.einsum("ij,ij->i", n, out) < 0
    f = f.copy()
    f[bad] = f[bad][:, [0, 2, 1]]
    return f


def radial_jitter(verts, sigma, rng):
    r = 1.0 + rng.normal(0.0, sigma, size=len(verts))
    d = verts / np.linalg.norm(verts, axis=1, keepdims=True)
    return d * r[:, None]


def random_albedo(n, rng):
    return rng.uniform(0.2, 0.9, size=(n, 3))


def random_unit(rng):
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


# ----------------------------------------------------------------------------- camera / motion

def look_at(eye, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0)) -> np.ndarray:
    """3x4 world->camera matrix [R | -R eye]; camera +z looks from ``eye`` at ``target``,
    +x is screen right and +y is screen up."""
    eye = np.asarray(eye, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(np.asarray(up, dtype=np.float64), f)
    if np.linalg.norm(r) < 1e-9:
        r = np.cross(np.array([0.0, 0.0, 1.0]), f)
    r /= np.linalg.norm(r)
    u = np.cross(f, r)
    R = np.stack([r, u, f])
    return np.concatenate([R, (-R @ eye)[:, None]], axis=1)


def orbit_eye(dist, azimuth_deg, elevation_deg):
    """Eye on a sphere around the origin; azimuth 0 / elevation 0 is (0, 0, -dist)."""
    a = math.radians(azimuth_deg)
    e = math.radians(elevation_deg)
    return (dist * math.cos(e) * math.sin(a), dist * math.sin(e), -dist * math.cos(e) * math.cos(a))


def camera(view, fov_deg=40.0, time_rule="paper", delta=DELTA, prob="exp", interp="screen"):
    return dict(view=np.asarray(view, dtype=np.float64), tan_half_fov=math.tan(math.radians(fov_deg) / 2),
                znear=ZNEAR, light_dir=np.array(LIGHT_DIR, dtype=np.float64), k_ambient=K_AMBIENT,
                k_diffuse=K_DIFFUSE, delta=delta, time_rule=time_rule, prob=prob, interp=interp)


def translate(d, offset=None, segments=0):
    d = np.asarray(d, dtype=np.float64)
    o = -0.5 * d if offset is None else np.asarray(offset, dtype=np.float64)
    return dict(kind="translate", offset=o, dir=d, axis=np.array([0.0, 1.0, 0.0]), omega=0.0,
                segments=segments)


def rotate(axis, omega, segments=0):
    a = np.asarray(axis, dtype=np.float64)
    return dict(kind="rotate", offset=np.zeros(3), dir=np.zeros(3), axis=a / np.linalg.norm(a),
                omega=float(omega), segments=segments)


def parabolic(axis=(0.0, 1.0, 0.0), omega=math.pi, offset=(0.5, -0.5, 0.5), dir=(-1.0, 4.0, -1.0),
              acc=(0.0, -4.0, 0.0), segments=0):
    """Rotation R(omega t) about unit(axis) plus the translation offset + t dir + t^2 acc.  The
    defaults are the appendix's parabolic trajectory: a half turn about +y and
    T(t) = (s, -4 s^2 + 0.5, s) with s = 0.5 - t."""
    a = np.asarray(axis, dtype=np.float64)
    return dict(kind="parabolic", offset=np.asarray(offset, np.float64), dir=np.asarray(dir, np.float64),
                axis=a / np.linalg.norm(a), omega=float(omega), segments=int(segments),
                acc=np.asarray(acc, np.float64))


def spherical_uv(verts):
    """Per-vertex texture coordinates from the direction of each vertex: u = longitude / 2 pi,
    v = colatitude / pi (a seam where the longitude wraps)."""
    v = np.asarray(verts, dtype=np.float64)
    r = np.linalg.norm(v, axis=1)
    u = 0.5 + np.arctan2(v[:, 2], v[:, 0]) / (2 * math.pi)
    w = np.arccos(np.clip(v[:, 1] / np.maximum(r, 1e-12), -1.0, 1.0)) / math.pi
    return np.stack([u, w], axis=1)


def smooth_texture(th, tw, rng, terms=4):
    """RGB texture [th, tw, 3] in [0.1, 0.9]: a few random low-frequency sinusoids per channel."""
    ys, xs = np.meshgrid(np.arange(th) / th, np.arange(tw) / tw, indexing="ij")
    tex = np.full((th, tw, 3), 0.5)
    for c in range(3):
        for _ in range(terms):
            fx, fy = rng.integers(1, 4, size=2)
            ph = rng.uniform(0, 2 * math.pi)
            tex[..., c] += 0.1 * np.sin(2 * math.pi * (fx * xs + fy * ys) + ph)
    return np.clip(tex, 0.1, 0.9)


def textured(sc, th=16, tw=24, seed=MASTER_SEED + 300):
    """The scene with spherical per-vertex uv and a smooth random texture (colours come from the
    texture instead of the per-vertex albedo)."""
    rng = np.random.default_rng(seed)
    return dict(sc, uv=spherical_uv(sc["verts"]), texture=smooth_texture(th, tw, rng))


def scene(verts, faces, albedo, motion, cam, T, H, W):
    return dict(verts=np.ascontiguousarray(verts, dtype=np.float64),
                faces=np.ascontiguousarray(faces, dtype=np.int32),
                albedo=np.ascontiguousarray(albedo, dtype=np.float64),
                motion=motion, camera=cam, T=int(T), H=int(H), W=int(W))


# ----------------------------------------------------------------------------- workloads

def config1(seed=MASTER_SEED + 1):
    """Forward-only translation: icosphere subdiv 2 (162 v / 320 f) with radial jitter N(0, 0.02),
    d = (1.5, 0, 0) centred on the origin, T = 16, 64x64, camera at distance 4 with a 40 deg FOV."""
    rng = np.random.default_rng(seed)
    v, f = icosphere(2)
    v = radial_jitter(v, 0.02, rng)
    return scene(v, f, random_albedo(len(v), rng), translate((1.5, 0.0, 0.0)),
                 camera(look_at(orbit_eye(4.0, 0, 0))), 16, 64, 64)


def sh_sphere(subdiv, lmax, sigma, rng):
    v, f = icosphere(subdiv)
    return sh_displace(v, lmax, sigma, rng), f


def config2(seed=MASTER_SEED + 2, T=64, H=256, W=256):
    """Rotation, plain vs fast: icosphere subdiv 4 (2562 v / 5120 f) with SH displacement of degree
    <= 6 (coefficients N(0, 0.05)); one full turn about a seeded random unit axis; T = 64, 256x256;
    12 segments per turn."""
    rng = np.random.default_rng(seed)
    v, f = sh_sphere(4, 6, 0.05, rng)
    alb = random_albedo(len(v), rng)
    axis = random_unit(rng)
    return scene(v, f, alb, rotate(axis, 2 * math.pi), camera(look_at(orbit_eye(4.0, 0, 0))), T, H, W)


def config2_translate(seed=MASTER_SEED + 2, T=64, H=256, W=256):
    """Translation counterpart of config2 (the paper times its solvers on linear translation,
    Sec. 4.2): the same subdiv-4, SH-6 mesh and albedo, moved by d = (1.5, 0, 0) perpendicular
    to the view axis and centred on the origin (o = -d/2); T = 64, 256x256, one linear segment."""
    sc = config2(seed, T, H, W)
    return dict(sc, motion=translate((1.5, 0.0, 0.0)))


def config3(seed=MASTER_SEED + 3, T=64, H=256, W=256):
    """Shape recovery: target subdiv-4 sphere with SH displacement (degree <= 8, N(0, 0.08)); 8 blurred
    views (4 translations with |d| ~ U[0.5, 2], 4 rotations with omega ~ U[pi, 4pi]) seen from
    azimuths 0, 45, ..., 315 deg at elevation 0 and distance 4.  Returns (target scenes, template
    vertices) -- the template is the undisplaced subdiv-4 sphere with the target's faces/albedo."""
    rng = np.random.default_rng(seed)
    v, f = sh_sphere(4, 8, 0.08, rng)
    alb = random_albedo(len(v), rng)
    views = []
    for i in range(8):
        cam = camera(look_at(orbit_eye(4.0, 45.0 * i, 0.0)))
        if i % 2 == 0:
            d = random_unit(rng) * rng.uniform(0.5, 2.0)
            mot = translate(d)
        else:
            omega = rng.uniform(math.pi, 4 * math.pi)
            mot = rotate(random_unit(rng), omega)
        views.append(scene(v, f, alb, mot, cam, T, H, W))
    template, _ = icosphere(4)
    return views, template


def config4(seed=MASTER_SEED + 4, n_objects=32):
    """Batching: 32 objects, icosphere subdiv 2..5 with SH displacement, half translating and half
    rotating, T from {16, 32, 64, 128, 256}, square resolution from {128, 256, 512}."""
    rng = np.random.default_rng(seed)
    items = []
    for i in range(n_objects):
        sub = int(rng.integers(2, 6))
        v, f = sh_sphere(sub, 6, 0.05, rng)
        alb = random_albedo(len(v), rng)
        T = int(rng.choice([16, 32, 64, 128, 256]))
        R = int(rng.choice([128, 256, 512]))
        if i % 2 == 0:
            mot = translate(random_unit(rng) * rng.uniform(0.5, 2.0))
        else:
            mot = rotate(random_unit(rng), rng.uniform(math.pi, 4 * math.pi))
        cam = camera(look_at(orbit_eye(4.0, rng.uniform(0, 360), rng.uniform(-30, 30))))
        items.append(scene(v, f, alb, mot, cam, T, R, R))
    return items


def config5(seed=MASTER_SEED + 5, T=256, H=1024, W=1024):
    """Large: a ~100k-face surface of revolution (224 x 224 grid x 2 triangles plus polar fans;
    radius profile from 12 B-spline control points; Gaussian bump sigma = 0.1) spinning about its
    axis (+y) at 8 turns per exposure, T = 256, 1024x1024, 96 segments."""
    rng = np.random.default_rng(seed)
    v, f = surface_of_revolution(224, 226, rng)
    alb = random_albedo(len(v), rng)
    return scene(v, f, alb, rotate((0.0, 1.0, 0.0), 16 * math.pi),
                 camera(look_at(orbit_eye(4.0, 0, 20.0))), T, H, W)


def config_sdf_rotation(seed=MASTER_SEED + 6, T=24, H=128, W=128, n_views=5):
    """Rotational recovery through an SDF (the paper's rotation task): a target subdiv-4 sphere with
    SH displacement (degree <= 4, N(0, 0.08)) spinning one turn about +y per exposure (12
    segments), seen from ``n_views`` cameras at elevations from -40 to 40 degrees (azimuths 30
    degrees apart), distance 4; grey albedo 0.7.  Returns the scenes (one per view) -- they share
    the target mesh."""
    rng = np.random.default_rng(seed)
    v, f = sh_sphere(4, 4, 0.08, rng)
    alb = np.full((len(v), 3), 0.7)
    out = []
    for i in range(n_views):
        e = -40.0 + 80.0 * i / max(1, n_views - 1)
        cam = camera(look_at(orbit_eye(4.0, 30.0 * i, e)))
        out.append(scene(v, f, alb, rotate((0.0, 1.0, 0.0), 2 * math.pi), cam, T, H, W))
    return out


def small_scene(kind="rotate", subdiv=2, T=8, H=40, W=72, seed=MASTER_SEED + 100, lmax=4, sigma=0.05,
                time_rule="paper", omega=2 * math.pi, segments=0, d=(1.2, 0.3, 0.0), eye=(0.0, 0.0),
                fov=40.0):
    """Small seeded scene for parity and oracle tests (ragged image sizes on purpose)."""
    rng = np.random.default_rng(seed)
    v, f = sh_sphere(subdiv, lmax, sigma, rng)
    alb = random_albedo(len(v), rng)
    if kind == "rotate":
        mot = rotate(random_unit(rng), omega, segments)
    elif kind == "parabolic":
        mot = parabolic(segments=segments)
    else:
        mot = translate(d, segments=segments)
    cam = camera(look_at(orbit_eye(4.0, eye[0], eye[1])), fov_deg=fov, time_rule=time_rule)
    return scene(v, f, alb, mot, cam, T, H, W)
