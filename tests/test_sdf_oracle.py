"""Pins of the FP64 SDF -> mesh extraction oracle (rotational recovery, Sec. 5) against facts
other than itself: exact planes, the analytic sphere (second-order convergence of the vertices,
area and volume), the topology of closed surfaces (every edge in two faces with opposite
directions, Euler characteristic), and finite differences of its adjoint.  CPU only."""
import math
from collections import Counter

import numpy as np
import pytest

import oracle


def _grid(n, lo=-1.2, hi=1.2):
    h = (hi - lo) / n
    ax = lo + h * np.arange(n + 1)
    Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
    return X, Y, Z, np.array([lo, lo, lo]), h


def _directed_edges(f):
    E = Counter()
    for t in f:
        for q in range(3):
            E[(int(t[q]), int(t[(q + 1) % 3]))] += 1
    return E


def _closed_and_oriented(f):
    """Every directed edge once, and its reverse once: a closed, consistently oriented surface."""
    E = _directed_edges(f)
    return all(c == 1 and E.get((b, a), 0) == 1 for (a, b), c in E.items()), len(E) // 2


def _area_volume(v, f):
    a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    cr = np.cross(b - a, c - a)
    return 0.5 * np.linalg.norm(cr, axis=1).sum(), np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0


def test_plane_is_extracted_exactly():
    """A linear SDF s = x - c is interpolated exactly along every edge: all vertices lie on x = c,
    the surface covers the grid's cross-section (area (2.4)^2), and the faces point to +x (the
    outside)."""
    X, Y, Z, lo, h = _grid(8)
    c = 0.137
    v, e, f = oracle.sdf_extract(X - c, lo, h)
    assert np.abs(v[:, 0] - c).max() < 1e-14
    a, b, cc = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    nrm = np.cross(b - a, cc - a)
    assert (nrm[:, 0] > 0).all()
    assert abs(0.5 * np.linalg.norm(nrm, axis=1).sum() - 2.4 ** 2) < 1e-12


@pytest.mark.parametrize("n", [12, 24])
def test_sphere_is_closed_outward_and_genus_zero(n):
    """s = |x| - R (an exact SDF): a closed, consistently oriented surface of Euler characteristic
    V - E + F = 2, with positive enclosed volume (outward faces)."""
    X, Y, Z, lo, h = _grid(n)
    v, e, f = oracle.sdf_extract(np.sqrt(X ** 2 + Y ** 2 + Z ** 2) - 0.83, lo, h)
    ok, n_edges = _closed_and_oriented(f)
    assert ok
    assert len(v) - n_edges + len(f) == 2
    assert _area_volume(v, f)[1] > 0


def test_sphere_converges_at_second_order():
    """Vertices of the exact sphere SDF lie within h^2 / R of the sphere; the error, the area and
    the volume converge like h^2 (each halving of h cuts the error by more than 3x)."""
    R = 0.83
    errs, dA, dV = [], [], []
    for n in (12, 24, 48):
        X, Y, Z, lo, h = _grid(n)
        v, e, f = oracle.sdf_extract(np.sqrt(X ** 2 + Y ** 2 + Z ** 2) - R, lo, h)
        err = np.abs(np.linalg.norm(v, axis=1) - R).max()
        assert err <= h * h / R
        A, Vol = _area_volume(v, f)
        errs.append(err)
        dA.append(abs(A - 4 * math.pi * R ** 2))
        dV.append(abs(Vol - 4 / 3 * math.pi * R ** 3))
    for seq in (errs, dA, dV):
        assert seq[0] / seq[1] > 3.0 and seq[1] / seq[2] > 3.0, seq


def test_random_fields_give_closed_oriented_surfaces():
    """Any field that is positive on the grid boundary has a closed zero set inside: the extracted
    surface must have every edge in exactly two faces with opposite directions (this fails when
    neighbouring cubes split a shared face along different diagonals, or when a case emits a
    triangle with the wrong winding).  Random smooth and rough fields, including exact zeros."""
    rng = np.random.default_rng(3)
    for trial in range(12):
        n = int(rng.integers(3, 9))
        X, Y, Z, lo, h = _grid(n, -1.0, 1.0)
        s = rng.normal(size=X.shape) if trial % 2 else np.sin(3 * X + rng.normal()) * np.cos(2 * Y) + 0.3 * Z
        if trial % 3 == 0:
            s = np.round(s * 2) / 2  # exact zeros on the grid
        s[0], s[-1], s[:, 0], s[:, -1], s[:, :, 0], s[:, :, -1] = 1, 1, 1, 1, 1, 1
        v, e, f = oracle.sdf_extract(s, lo, h)
        if len(f) == 0:
            continue
        ok, n_edges = _closed_and_oriented(f)
        assert ok, trial
        # vertices sit on sign-changing grid edges at the zero of the linear interpolant
        sf = s.reshape(-1)
        assert ((sf[e[:, 0]] < 0) != (sf[e[:, 1]] < 0)).all()


def test_one_inside_corner_gives_the_corner_triangles():
    """One negative sample at the centre of a 2-cell grid: the surface is the link of that grid
    vertex in the tetrahedral split, crossing each incident edge once.  In this split (Kuhn's
    triangulation of the cube grid) an interior vertex has 14 neighbours and lies in 24
    tetrahedra, so the surface has 14 vertices and 24 triangles, closed with V - E + F = 2; the
    six axis-edge crossings sit at the edge midpoints (s = -1 and +1)."""
    X, Y, Z, lo, h = _grid(2, -1.0, 1.0)
    s = np.ones_like(X)
    s[1, 1, 1] = -1.0
    v, e, f = oracle.sdf_extract(s, lo, h)
    assert len(v) == 14
    assert (e == 13).any(axis=1).all()  # every vertex on an edge of the centre sample (index 13)
    assert np.allclose(np.linalg.norm(v, axis=1)[np.abs(v).sum(1) <= 0.5 + 1e-12], 0.5)  # axis edges: midpoints
    ok, n_edges = _closed_and_oriented(f)
    assert ok and len(v) - n_edges + len(f) == 2
    assert len(f) == 24


def test_adjoint_matches_central_differences():
    """dL/ds of L = sum g . v over the extracted vertices against central differences (topology
    fixed: the step never changes a sign)."""
    X, Y, Z, lo, h = _grid(10)
    rng = np.random.default_rng(5)
    s = np.sqrt(X ** 2 + (1.3 * Y) ** 2 + Z ** 2) - 0.8 + 0.05 * np.sin(4 * X)
    v, e, f = oracle.sdf_extract(s, lo, h)
    g = rng.normal(size=v.shape)
    grad = oracle.sdf_extract_backward(s, lo, h, e, g)
    used = np.unique(e.reshape(-1))
    assert np.abs(grad).sum() > 0 and set(np.nonzero(grad.reshape(-1))[0]) <= set(used.tolist())
    eps = 1e-7
    for idx in rng.choice(used, size=25, replace=False):
        sp, sm = s.copy().reshape(-1), s.copy().reshape(-1)
        if min(abs(sp[idx]) - eps, 1) <= 0:
            continue
        sp[idx] += eps
        sm[idx] -= eps
        vp, ep, fp = oracle.sdf_extract(sp.reshape(s.shape), lo, h)
        vm, em, fm = oracle.sdf_extract(sm.reshape(s.shape), lo, h)
        assert np.array_equal(ep, e) and np.array_equal(em, e)
        fd = ((vp - vm) * g).sum() / (2 * eps)
        assert abs(fd - grad.reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(fd)), (idx, fd, grad.reshape(-1)[idx])
