"""PyTorch-facing API of the motion-blurred renderer: device tensors in, device tensors out, the
caller's current CUDA stream, and a ``torch.autograd.Function`` whose backward is the library's
hand-written adjoint.  PyTorch supplies device memory and streams only; all arithmetic of the
renderer runs in the CUDA kernels behind the C ABI."""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import MbrCamera, MbrError, MbrItem, MbrMesh, MbrMotion


_KINDS = {"translate": _lib.MBR_TRANSLATE, "rotate": _lib.MBR_ROTATE, "parabolic": _lib.MBR_PARABOLIC}


@dataclass
class Motion:
    kind: str = "translate"          # 'translate' | 'rotate' | 'parabolic' (see include/mbr.h)
    offset: tuple = (0.0, 0.0, 0.0)
    dir: tuple = (0.0, 0.0, 0.0)
    axis: tuple = (0.0, 1.0, 0.0)
    omega: float = 0.0
    segments: int = 0
    acc: tuple = (0.0, 0.0, 0.0)     # parabolic: quadratic term of the translation

    def c(self):
        m = MbrMotion()
        m.kind = _KINDS[self.kind]
        m.segments = int(self.segments)
        m.offset[:] = [float(x) for x in self.offset]
        m.dir[:] = [float(x) for x in self.dir]
        m.axis[:] = [float(x) for x in self.axis]
        m.omega = float(self.omega)
        m.acc[:] = [float(x) for x in self.acc]
        return m


@dataclass
class Camera:
    view: tuple                      # 12 floats, 3x4 row-major world->camera
    tan_half_fov: float
    znear: float = 0.1
    light_dir: tuple = (0.4, 0.6, -0.7)
    k_ambient: float = 0.3
    k_diffuse: float = 0.7
    delta: float = 1e-4
    time_rule: str = "paper"         # 'paper' | 'midpoint'
    prob: str = "exp"                # soft-coverage map: 'exp' (the paper's) | 'sigmoid' (SoftRas)
    interp: str = "screen"           # attribute weights: 'screen' (Eq. fore) | 'perspective'

    def c(self):
        c = MbrCamera()
        c.view[:] = [float(x) for x in np.asarray(self.view, dtype=np.float64).reshape(-1)]
        c.tan_half_fov = float(self.tan_half_fov)
        c.znear = float(self.znear)
        c.light_dir[:] = [float(x) for x in self.light_dir]
        c.k_ambient = float(self.k_ambient)
        c.k_diffuse = float(self.k_diffuse)
        c.delta = float(self.delta)
        c.time_rule = _lib.MBR_TIME_PAPER if self.time_rule == "paper" else _lib.MBR_TIME_MIDPOINT
        c.prob = {"exp": _lib.MBR_PROB_EXP, "sigmoid": _lib.MBR_PROB_SIGMOID}[self.prob]
        c.interp = {"screen": _lib.MBR_INTERP_SCREEN, "perspective": _lib.MBR_INTERP_PERSPECTIVE}[self.interp]
        return c


def motion_from_dict(m):
    return Motion(kind=m["kind"], offset=tuple(m["offset"]), dir=tuple(m["dir"]), axis=tuple(m["axis"]),
                  omega=float(m["omega"]), segments=int(m.get("segments", 0)),
                  acc=tuple(m.get("acc", (0.0, 0.0, 0.0))))


def camera_from_dict(c):
    return Camera(view=tuple(np.asarray(c["view"]).reshape(-1)), tan_half_fov=c["tan_half_fov"], znear=c["znear"],
                  light_dir=tuple(c["light_dir"]), k_ambient=c["k_ambient"], k_diffuse=c["k_diffuse"],
                  delta=c["delta"], time_rule=c.get("time_rule", "paper"), prob=c.get("prob", "exp"),
                  interp=c.get("interp", "screen"))


def mesh_tensors(scene, device="cuda"):
    """(verts f32 [V,3], faces i32 [F,3], albedo f32 [V,3]) on ``device`` from a scene dict."""
    v = torch.as_tensor(np.asarray(scene["verts"], dtype=np.float32), device=device).contiguous()
    f = torch.as_tensor(np.asarray(scene["faces"], dtype=np.int32), device=device).contiguous()
    a = torch.as_tensor(np.asarray(scene["albedo"], dtype=np.float32), device=device).contiguous()
    return v, f, a


def _check(t, dtype, shape, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous() or tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: expected contiguous {dtype} {tuple(shape)}, got {t.dtype} {tuple(t.shape)}")


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Context:
    """Owns one library context (scratch memory) on the current CUDA device."""

    def __init__(self):
        self.L = _lib.load()
        if not torch.cuda.is_available():
            raise RuntimeError("the motion-blur renderer needs a CUDA device (no CPU fallback)")
        torch.cuda.init()
        h = ctypes.c_void_p()
        rc = self.L.mbr_create(ctypes.byref(h))
        if rc != _lib.MBR_OK:
            raise MbrError(rc, "mbr_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.L.mbr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _raise(self, rc):
        if rc != _lib.MBR_OK:
            raise MbrError(rc, self.L.mbr_last_error(self.h).decode())

    @staticmethod
    def _mesh(verts, faces, albedo, uv=None, texture=None, dl_dtexture=None):
        V, F = verts.shape[0], faces.shape[0]
        _check(verts, torch.float32, (V, 3), "verts")
        _check(faces, torch.int32, (F, 3), "faces")
        _check(albedo, torch.float32, (V, 3), "albedo")
        m = MbrMesh()
        m.V, m.F = V, F
        m.verts, m.faces, m.albedo = verts.data_ptr(), faces.data_ptr(), albedo.data_ptr()
        if texture is not None:  # textured: the vertex attribute is uv, the colour a texture sample
            if uv is None or texture.dim() != 3:
                raise ValueError("a texture [th, tw, 3] needs uv [V, 2]")
            _check(uv, torch.float32, (V, 2), "uv")
            _check(texture, torch.float32, (texture.shape[0], texture.shape[1], 3), "texture")
            m.uv, m.texture = uv.data_ptr(), texture.data_ptr()
            m.tex_h, m.tex_w = texture.shape[0], texture.shape[1]
            if dl_dtexture is not None:
                _check(dl_dtexture, torch.float32, tuple(texture.shape), "dl_dtexture")
                m.dl_dtexture = dl_dtexture.data_ptr()
        return m

    def set_profiling(self, on=True):
        self._raise(self.L.mbr_set_profiling(self.h, int(bool(on))))

    def stats(self):
        st = _lib.MbrStats()
        self._raise(self.L.mbr_get_stats(self.h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in st._fields_}

    def sdf_extract(self, sdf, lo, h, want_edges=True):
        """Triangle mesh of the zero level set of ``sdf`` [(n+1)]^3 (float32, indexed [z, y, x])
        sampled at lo + h (i, j, k) (mbr_sdf_extract): (verts [V,3], faces [F,3] int32,
        vert_edges [V,2] int32 or None), sized to the mesh."""
        n = sdf.shape[0] - 1
        _check(sdf, torch.float32, (n + 1, n + 1, n + 1), "sdf")
        lo_c = (ctypes.c_float * 3)(*[float(x) for x in lo])
        counts = (ctypes.c_int32 * 2)()
        # capacities that always suffice (7 edges per grid point, 12 triangles per cube), one call
        max_v, max_f = 7 * (n + 1) ** 3, 12 * n ** 3
        verts = torch.empty((max_v, 3), dtype=torch.float32, device=sdf.device)
        faces = torch.empty((max_f, 3), dtype=torch.int32, device=sdf.device)
        edges = torch.empty((max_v, 2), dtype=torch.int32, device=sdf.device) if want_edges else None
        self._raise(self.L.mbr_sdf_extract(
            self.h, n, ctypes.c_void_p(sdf.data_ptr()), lo_c, float(h), max_v, max_f, ctypes.c_void_p(verts.data_ptr()),
            ctypes.c_void_p(faces.data_ptr()), ctypes.c_void_p(edges.data_ptr() if edges is not None else 0), counts,
            _stream()))
        V, F = counts[0], counts[1]
        verts, faces = verts[:V], faces[:F]
        edges = edges[:V] if edges is not None else None
        return verts, faces, edges

    def sdf_extract_backward(self, sdf, h, vert_edges, dl_dverts):
        """dL/dsdf for dL/dverts of sdf_extract's vertices (mbr_sdf_extract_backward)."""
        n = sdf.shape[0] - 1
        V = vert_edges.shape[0]
        _check(vert_edges, torch.int32, (V, 2), "vert_edges")
        _check(dl_dverts, torch.float32, (V, 3), "dl_dverts")
        out = torch.empty_like(sdf)
        self._raise(self.L.mbr_sdf_extract_backward(
            self.h, n, ctypes.c_void_p(sdf.data_ptr()), float(h), V, ctypes.c_void_p(vert_edges.data_ptr()),
            ctypes.c_void_p(dl_dverts.data_ptr()), ctypes.c_void_p(out.data_ptr()), _stream()))
        return out

    def measure_fp32_peak(self, iters=20000, launches=10):
        """Measured FP32 peak (TFLOP/s) and its raw figures: FMA chains on every SM, CUDA-event
        timed (mbr_measure_fp32_peak)."""
        fl, ms = ctypes.c_double(), ctypes.c_float()
        self._raise(self.L.mbr_measure_fp32_peak(self.h, iters, launches, ctypes.byref(fl), ctypes.byref(ms),
                                                 _stream()))
        return fl.value / (ms.value * 1e-3) / 1e12, fl.value, ms.value

    def set_state_budget(self, nbytes):
        """Per-sample forward state kept for the adjoint up to ``nbytes`` (0: the adjoint always
        recomputes it; mbr_set_state_budget)."""
        self._raise(self.L.mbr_set_state_budget(self.h, int(nbytes)))

    def set_tuning(self, tile=16, spt=2, splits=0):
        self._raise(self.L.mbr_set_tuning(self.h, int(tile), int(spt), int(splits)))

    def render_blur(self, verts, faces, albedo, motion: Motion, camera: Camera, T, H, W, solver="fast", out=None,
                    uv=None, texture=None):
        """[H, W, 4] blurred RGBA.  With ``texture`` [th, tw, 3] and ``uv`` [V, 2] the colours are
        texture samples at the interpolated uv (albedo unused)."""
        m = self._mesh(verts, faces, albedo, uv, texture)
        if out is None:
            out = torch.empty((H, W, 4), dtype=torch.float32, device=verts.device)
        _check(out, torch.float32, (H, W, 4), "image")
        mo, ca = motion.c(), camera.c()
        self._raise(self.L.mbr_render_blur(self.h, ctypes.byref(m), ctypes.byref(mo), ctypes.byref(ca), T, H, W,
                                           _lib.SOLVERS[solver], ctypes.c_void_p(out.data_ptr()), _stream()))
        return out

    def render_blur_backward(self, verts, faces, albedo, motion, camera, T, H, W, dl_dimage, solver="fast",
                             want_albedo=True, reuse_forward=False, uv=None, texture=None):
        """dL/dverts (and dL/dalbedo) for dL/dimage; textured (``uv``, ``texture`` given):
        (dL/dverts, dL/dalbedo, dL/dtexture).  reuse_forward=True: the adjoint of the immediately
        preceding render_blur on this context with the same arguments and unchanged tensor
        contents (mbr_render_blur_backward_reuse)."""
        gt = torch.empty_like(texture) if texture is not None else None
        m = self._mesh(verts, faces, albedo, uv, texture, gt)
        _check(dl_dimage, torch.float32, (H, W, 4), "dl_dimage")
        gv = torch.empty_like(verts)
        ga = torch.empty_like(albedo) if want_albedo else None
        mo, ca = motion.c(), camera.c()
        fn = self.L.mbr_render_blur_backward_reuse if reuse_forward else self.L.mbr_render_blur_backward
        self._raise(fn(
            self.h, ctypes.byref(m), ctypes.byref(mo), ctypes.byref(ca), T, H, W, _lib.SOLVERS[solver],
            ctypes.c_void_p(dl_dimage.data_ptr()), ctypes.c_void_p(gv.data_ptr()),
            ctypes.c_void_p(ga.data_ptr() if ga is not None else 0), _stream()))
        return (gv, ga, gt) if texture is not None else (gv, ga)

    def debug_winners(self, verts, faces, albedo, motion, camera, T, H, W, k, solver="fast"):
        m = self._mesh(verts, faces, albedo)
        ids = torch.empty((H, W), dtype=torch.int32, device=verts.device)
        mo, ca = motion.c(), camera.c()
        self._raise(self.L.mbr_debug_winners(self.h, ctypes.byref(m), ctypes.byref(mo), ctypes.byref(ca), T, H, W,
                                             _lib.SOLVERS[solver], int(k), ctypes.c_void_p(ids.data_ptr()),
                                             _stream()))
        return ids

    def count_candidates(self, verts, faces, albedo, motion, camera, T, H, W, solver="fast"):
        m = self._mesh(verts, faces, albedo)
        out = ctypes.c_int64()
        mo, ca = motion.c(), camera.c()
        self._raise(self.L.mbr_count_candidates(self.h, ctypes.byref(m), ctypes.byref(mo), ctypes.byref(ca), T, H,
                                                W, _lib.SOLVERS[solver], ctypes.byref(out), _stream()))
        return out.value

    def count_work(self, verts, faces, albedo, motion, camera, T, H, W, solver="fast", out=None, detail=False):
        """(N_box, N_soft, N_covered) of one forward render (see include/mbr.h, mbr_count_work);
        also renders into ``out`` when given.  detail=True returns the dict of all eight counters."""
        m = self._mesh(verts, faces, albedo)
        if out is not None:
            _check(out, torch.float32, (H, W, 4), "image")
        res = (ctypes.c_int64 * 8)()
        mo, ca = motion.c(), camera.c()
        self._raise(self.L.mbr_count_work(self.h, ctypes.byref(m), ctypes.byref(mo), ctypes.byref(ca), T, H, W,
                                          _lib.SOLVERS[solver],
                                          ctypes.c_void_p(out.data_ptr() if out is not None else 0), res,
                                          _stream()))
        keys = ("n_cand", "n_soft", "n_cov", "soft_evals", "soft_warp_steps", "cov_tests", "cov_warp_steps", "n_box")
        if detail:
            return {k: int(res[i]) for i, k in enumerate(keys)}
        return int(res[7]), int(res[1]), int(res[2])

    def _items(self, items, with_backward):
        arr = (MbrItem * len(items))()
        for i, it in enumerate(items):
            a = arr[i]
            a.mesh = self._mesh(it["verts"], it["faces"], it["albedo"], it.get("uv"), it.get("texture"),
                                it.get("dl_dtexture") if with_backward else None)
            a.motion = it["motion"].c()
            a.camera = it["camera"].c()
            a.T, a.H, a.W = it["T"], it["H"], it["W"]
            a.solver = _lib.SOLVERS[it.get("solver", "fast")]
            a.image = it["image"].data_ptr()
            if with_backward:
                a.dl_dimage = it["dl_dimage"].data_ptr()
                a.dl_dverts = it["dl_dverts"].data_ptr()
                a.dl_dalbedo = it["dl_dalbedo"].data_ptr() if it.get("dl_dalbedo") is not None else 0
        return arr

    def render_batch(self, items, with_backward=False):
        """items: list of dicts(verts, faces, albedo, motion, camera, T, H, W, solver, image,
        [uv, texture], [dl_dimage, dl_dverts, dl_dalbedo, dl_dtexture]) with preallocated CUDA
        tensors (see include/mbr.h)."""
        arr = self._items(items, with_backward)
        self._raise(self.L.mbr_render_blur_batch(self.h, len(items), arr, int(bool(with_backward)), _stream()))

    def autotune(self, items, with_backward=False):
        """Pick the fastest tile shape / sub-frames per thread for this batch; returns
        (tile, spt, ms) and keeps the choice on the context."""
        arr = self._items(items, with_backward)
        t, sp, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
        self._raise(self.L.mbr_autotune(self.h, len(items), arr, int(bool(with_backward)), ctypes.byref(t),
                                        ctypes.byref(sp), ctypes.byref(ms), _stream()))
        return t.value, sp.value, ms.value


_default_ctx = {}


def default_context():
    dev = torch.cuda.current_device()
    if dev not in _default_ctx:
        _default_ctx[dev] = Context()
    return _default_ctx[dev]


class RenderBlur(torch.autograd.Function):
    """image = render_blur(verts, albedo); backward gives dL/dverts and dL/dalbedo through the
    library's adjoint kernels.  The adjoint recomputes every sub-frame quantity (barycentrics,
    distances, closest points, shading) per sample; the forward keeps only, per sample, the winner
    face or the aggregate log soft product, and its front half (records, bins)."""

    @staticmethod
    def forward(ctx, verts, albedo, faces, motion, camera, T, H, W, solver, rctx):
        verts = verts.contiguous()
        albedo = albedo.contiguous()
        img = rctx.render_blur(verts, faces, albedo, motion, camera, T, H, W, solver)
        ctx.save_for_backward(verts, albedo, faces)
        ctx.args = (motion, camera, T, H, W, solver, rctx)
        return img

    @staticmethod
    def backward(ctx, g):
        verts, albedo, faces = ctx.saved_tensors
        motion, camera, T, H, W, solver, rctx = ctx.args
        # autograd's saved-tensor version check guarantees verts/albedo/faces are unchanged since the
        # forward, so the adjoint may reuse the forward's front half if nothing else ran in between
        gv, ga = rctx.render_blur_backward(verts, faces, albedo, motion, camera, T, H, W, g.contiguous(), solver,
                                           want_albedo=ctx.needs_input_grad[1], reuse_forward=True)
        return gv, ga, None, None, None, None, None, None, None, None


def render_blur(verts, albedo, faces, motion, camera, T, H, W, solver="fast", rctx=None):
    """Differentiable blurred render [H,W,4] of the mesh (see include/mbr.h)."""
    return RenderBlur.apply(verts, albedo, faces, motion, camera, T, H, W, solver, rctx or default_context())
