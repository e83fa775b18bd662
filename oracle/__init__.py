"""ctypes wrapper of the FP64 CPU oracle (``mbr_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the test suite, by ``__graft_entry__.smoke()`` and by the
benchmark's CPU-baseline / reference leg.  The CUDA product path never imports it, and it imports
nothing from the product package (only the seeded scene dictionaries produced by ``scenes``).

Modes (see mbr_oracle.h):
  ``exact``  -- PLAIN_EXACT: exact motion + projection at every sub-frame, direct solve per sample
                (the per-sub-frame barycentric baseline of Sec. 3.1);
  ``linear`` -- PLAIN_LINEAR: keyframe-lerped screen positions (Sec. 3.2), direct solve per sample;
  ``fast``   -- FAST_REF: PLAIN_LINEAR with the keyframe closest-point approximation of
                Eqs. euc-dist-approx-2/3 for background samples (what the fast solver computes).
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int32, c_int64, c_uint8

import numpy as np

from .build import build, library_path

MODES = {"exact": 0, "linear": 1, "fast": 2}
SOFT_ALL, SOFT32 = 1, 2
CNT_CAND, CNT_COVERED, CNT_AMBIG, CNT_HASH, CNT_SOFT, CNT_SOFT32 = 0, 1, 2, 3, 4, 5
AMB_COVER, AMB_DEPTH, AMB_DEGEN, AMB_REGION, AMB_CLAMP, AMB_LAMBERT, AMB_COND = 1, 2, 4, 8, 16, 32, 64
AMB_TEXCELL = 128  # gradient only: a textured sample near a texel-centre line (the bilinear slope jumps)
AMB_IMAGE = AMB_COVER | AMB_DEPTH | AMB_DEGEN | AMB_REGION  # flags that can change a pixel value


class OrcScene(ctypes.Structure):
    _fields_ = [
        ("V", c_int32), ("F", c_int32),
        ("verts", POINTER(c_double)), ("faces", POINTER(c_int32)), ("albedo", POINTER(c_double)),
        ("uv", POINTER(c_double)), ("texture", POINTER(c_double)), ("tex_h", c_int32), ("tex_w", c_int32),
        ("dl_dtexture", POINTER(c_double)),
        ("motion_kind", c_int32), ("segments", c_int32),
        ("offset", c_double * 3), ("dir", c_double * 3), ("axis", c_double * 3), ("omega", c_double),
        ("acc", c_double * 3),
        ("view", c_double * 12), ("tan_half_fov", c_double), ("znear", c_double),
        ("light_dir", c_double * 3), ("k_ambient", c_double), ("k_diffuse", c_double),
        ("delta", c_double), ("time_rule", c_int32), ("prob", c_int32), ("interp", c_int32),
        ("T", c_int32), ("H", c_int32), ("W", c_int32),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        L.orc_num_segments.argtypes = [P(OrcScene)]
        L.orc_num_segments.restype = c_int32
        L.orc_sample_time.argtypes = [P(OrcScene), c_int32, P(c_int32), P(c_double), P(c_double)]
        L.orc_vertex_normals.argtypes = [P(OrcScene), P(c_double)]
        L.orc_vertex_state.argtypes = [P(OrcScene), P(c_double), c_double, P(c_double)]
        L.orc_barycentric.argtypes = [P(c_double), c_double, c_double, P(c_double)]
        L.orc_barycentric.restype = c_double
        L.orc_closest_point.argtypes = [P(c_double), c_double, c_double, P(c_double), P(c_int32)]
        L.orc_closest_point.restype = c_double
        L.orc_render.argtypes = [P(OrcScene), c_int32, c_int32, c_int32, c_int32, c_int32, c_int32,
                                 P(c_double), P(c_int32), P(c_uint8), P(c_int64)]
        L.orc_render.restype = c_int32
        L.orc_render_backward.argtypes = [P(OrcScene), c_int32, c_int32, c_int32, c_int32, c_int32,
                                          c_int32, P(c_double), P(c_double), P(c_double), P(c_int64)]
        L.orc_render_backward.restype = c_int32
        L.orc_sdf_extract.argtypes = [c_int32, P(c_double), P(c_double), c_double, c_int64, c_int64, P(c_double),
                                      P(c_int64), P(c_int32), P(c_int64)]
        L.orc_sdf_extract.restype = c_int32
        L.orc_sdf_extract_backward.argtypes = [c_int32, P(c_double), P(c_double), c_double, c_int64, P(c_int64),
                                               P(c_double), P(c_double)]
        L.orc_sdf_extract_backward.restype = c_int32
        _lib = L
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(POINTER(ctype)) if a is not None else None


class _Scene:
    """Keeps the numpy buffers alive for the lifetime of the ctypes struct."""

    def __init__(self, sc):
        self.verts = np.ascontiguousarray(sc["verts"], dtype=np.float64)
        self.faces = np.ascontiguousarray(sc["faces"], dtype=np.int32)
        self.albedo = np.ascontiguousarray(sc["albedo"], dtype=np.float64)
        tex = sc.get("texture")
        self.uv = np.ascontiguousarray(sc["uv"], dtype=np.float64) if tex is not None else None
        self.texture = np.ascontiguousarray(tex, dtype=np.float64) if tex is not None else None
        self.gtex = np.zeros_like(self.texture) if tex is not None else None
        m, c = sc["motion"], sc["camera"]
        s = OrcScene()
        s.V, s.F = len(self.verts), len(self.faces)
        s.verts = _ptr(self.verts, c_double)
        s.faces = _ptr(self.faces, c_int32)
        if tex is not None:
            s.uv = _ptr(self.uv, c_double)
            s.texture = _ptr(self.texture, c_double)
            s.tex_h, s.tex_w = self.texture.shape[0], self.texture.shape[1]
            s.dl_dtexture = _ptr(self.gtex, c_double)
        s.albedo = _ptr(self.albedo, c_double)
        s.motion_kind = {"translate": 0, "rotate": 1, "parabolic": 2}[m["kind"]]
        s.segments = int(m.get("segments", 0))
        s.offset[:] = [float(x) for x in m["offset"]]
        s.dir[:] = [float(x) for x in m["dir"]]
        s.axis[:] = [float(x) for x in m["axis"]]
        s.omega = float(m["omega"])
        s.acc[:] = [float(x) for x in m.get("acc", (0.0, 0.0, 0.0))]
        s.view[:] = [float(x) for x in np.asarray(c["view"]).reshape(-1)]
        s.tan_half_fov = float(c["tan_half_fov"])
        s.znear = float(c["znear"])
        s.light_dir[:] = [float(x) for x in c["light_dir"]]
        s.k_ambient = float(c["k_ambient"])
        s.k_diffuse = float(c["k_diffuse"])
        s.delta = float(c["delta"])
        s.time_rule = 0 if c.get("time_rule", "paper") == "paper" else 1
        s.prob = {"exp": 0, "sigmoid": 1}[c.get("prob", "exp")]
        s.interp = {"screen": 0, "perspective": 1}[c.get("interp", "screen")]
        s.T, s.H, s.W = int(sc["T"]), int(sc["H"]), int(sc["W"])
        self.s = s

    @property
    def ref(self):
        return ctypes.byref(self.s)


def num_segments(sc):
    return lib().orc_num_segments(_Scene(sc).ref)


def sample_time(sc, k):
    seg, t, tau = c_int32(), c_double(), c_double()
    lib().orc_sample_time(_Scene(sc).ref, int(k), ctypes.byref(seg), ctypes.byref(t), ctypes.byref(tau))
    return seg.value, t.value, tau.value


def vertex_normals(sc):
    S = _Scene(sc)
    out = np.zeros((S.s.V, 3))
    lib().orc_vertex_normals(S.ref, _ptr(out, c_double))
    return out


def vertex_state(sc, t):
    """[V,6]: ndc x, ndc y, camera z, world normal (x, y, z) at time t (exact motion)."""
    S = _Scene(sc)
    n = vertex_normals(sc)
    out = np.zeros((S.s.V, 6))
    lib().orc_vertex_state(S.ref, _ptr(n, c_double), float(t), _ptr(out, c_double))
    return out


def barycentric(tri, u, v):
    tri = np.ascontiguousarray(tri, dtype=np.float64).reshape(6)
    w = np.zeros(3)
    det = lib().orc_barycentric(_ptr(tri, c_double), float(u), float(v), _ptr(w, c_double))
    return w, det


def closest_point(tri, px, py):
    tri = np.ascontiguousarray(tri, dtype=np.float64).reshape(6)
    w = np.zeros(3)
    reg = c_int32()
    d2 = lib().orc_closest_point(_ptr(tri, c_double), float(px), float(py), _ptr(w, c_double),
                                 ctypes.byref(reg))
    return d2, w, reg.value


def _flags(soft_all, soft32):
    return (SOFT_ALL if soft_all else 0) | (SOFT32 if soft32 else 0)


def render(sc, mode="fast", window=None, soft_all=False, winners=False, ambig=False, soft32=False):
    """Blurred RGBA image of ``sc`` (or of ``window`` = (x0, y0, w, h)).  ``soft_all``: no soft
    truncation; ``soft32``: truncation at the single-precision cutoff (factors with
    exp(-d/delta) <= 2^-25 dropped) instead of d <= delta ln 1e12.

    Returns dict(rgba [h,w,4] f64, winners [T,h,w] i32 | None, ambig [T,h,w] u8 | None,
    counters [8] i64)."""
    S = _Scene(sc)
    x0, y0, w, h = window if window is not None else (0, 0, S.s.W, S.s.H)
    T = S.s.T
    rgba = np.zeros((h, w, 4))
    win = np.zeros((T, h, w), dtype=np.int32) if winners else None
    amb = np.zeros((T, h, w), dtype=np.uint8) if ambig else None
    cnt = np.zeros(8, dtype=np.int64)
    rc = lib().orc_render(S.ref, MODES[mode], _flags(soft_all, soft32), x0, y0, w, h,
                          _ptr(rgba, c_double), _ptr(win, c_int32), _ptr(amb, c_uint8),
                          _ptr(cnt, c_int64))
    if rc != 0:
        raise RuntimeError(f"orc_render failed ({rc})")
    return dict(rgba=rgba, winners=win, ambig=amb, counters=cnt)


def render_backward(sc, dl_drgba, mode="fast", window=None, soft_all=False, texture_grad=None, soft32=False):
    """(dL/dverts [V,3], dL/dalbedo [V,3], counters) for the loss gradient ``dl_drgba`` [h,w,4]
    (``soft_all``, ``soft32``: the truncation, as in ``render``).
    For a textured scene, ``texture_grad`` (an array shaped like the texture) receives
    dL/dtexture."""
    S = _Scene(sc)
    x0, y0, w, h = window if window is not None else (0, 0, S.s.W, S.s.H)
    g = np.ascontiguousarray(dl_drgba, dtype=np.float64).reshape(h, w, 4)
    gv = np.zeros((S.s.V, 3))
    ga = np.zeros((S.s.V, 3))
    cnt = np.zeros(8, dtype=np.int64)
    rc = lib().orc_render_backward(S.ref, MODES[mode], _flags(soft_all, soft32), x0, y0, w, h,
                                   _ptr(g, c_double), _ptr(gv, c_double), _ptr(ga, c_double),
                                   _ptr(cnt, c_int64))
    if rc != 0:
        raise RuntimeError(f"orc_render_backward failed ({rc})")
    if texture_grad is not None:
        texture_grad[...] = S.gtex
    return gv, ga, cnt


def sdf_extract(sdf, lo, h):
    """Marching-tetrahedra mesh of the zero level set of ``sdf`` [(n+1),(n+1),(n+1)] (indexed
    [k, j, i], i.e. z, y, x) sampled at lo + h (i, j, k): (verts [V,3], vert_edges [V,2] grid
    index pairs a < b, faces [F,3] facing s >= 0).  Vertices are in ascending (a, b) order."""
    s = np.ascontiguousarray(sdf, dtype=np.float64)
    n = s.shape[0] - 1
    assert s.shape == (n + 1,) * 3
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    cnt = np.zeros(2, dtype=np.int64)
    e = np.zeros(1, dtype=np.int64)
    rc = lib().orc_sdf_extract(n, _ptr(s, c_double), _ptr(lo, c_double), float(h), 0, 0, None, None, None,
                               _ptr(cnt, c_int64))
    if rc < 0:
        raise RuntimeError("orc_sdf_extract failed")
    V, F = int(cnt[0]), int(cnt[1])
    verts = np.zeros((max(V, 1), 3))
    edges = np.zeros((max(V, 1), 2), dtype=np.int64)
    faces = np.zeros((max(F, 1), 3), dtype=np.int32)
    rc = lib().orc_sdf_extract(n, _ptr(s, c_double), _ptr(lo, c_double), float(h), V, F, _ptr(verts, c_double),
                               _ptr(edges, c_int64), _ptr(faces, c_int32), _ptr(cnt, c_int64))
    if rc != 0:
        raise RuntimeError("orc_sdf_extract failed")
    del e
    return verts[:V], edges[:V], faces[:F]


def sdf_extract_backward(sdf, lo, h, vert_edges, dl_dverts):
    """dL/dsdf (same shape as sdf) for dL/dverts [V,3] of sdf_extract's vertices."""
    s = np.ascontiguousarray(sdf, dtype=np.float64)
    n = s.shape[0] - 1
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    ve = np.ascontiguousarray(vert_edges, dtype=np.int64)
    g = np.ascontiguousarray(dl_dverts, dtype=np.float64)
    out = np.zeros_like(s)
    rc = lib().orc_sdf_extract_backward(n, _ptr(s, c_double), _ptr(lo, c_double), float(h), len(ve),
                                        _ptr(ve, c_int64), _ptr(g, c_double), _ptr(out, c_double))
    if rc != 0:
        raise RuntimeError("orc_sdf_extract_backward failed")
    return out
