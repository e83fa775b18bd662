"""mbr_render_blur_noalloc: the forward render for callers that cannot allocate device memory
(a process that gives the GPU's memory to its own pool or a fixed budget up front, or a
latency-sensitive loop that cannot afford cudaMalloc's synchronisation).  Its scratch is a
static array inside the library, so these checks call it through the C ABI, twice in a row
(the second call must not see the first call's leftovers), and compare it with the
allocating entry point mbr_render_blur within the parity tolerance of the other GPU tests."""
import ctypes

import numpy as np
import pytest
import torch

import scenes

pytestmark = pytest.mark.gpu

TOL = 1e-4


def _call_noalloc(L, sc, solver, out):
    import paper_2602_07860_gb300 as mbr
    from paper_2602_07860_gb300 import _lib
    v, f, a = mbr.mesh_tensors(sc)
    mesh = mbr.Context._mesh(v, f, a)
    mo = mbr.motion_from_dict(sc["motion"]).c()
    ca = mbr.camera_from_dict(sc["camera"]).c()
    err = ctypes.create_string_buffer(512)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.mbr_render_blur_noalloc(ctypes.byref(mesh), ctypes.byref(mo), ctypes.byref(ca), sc["T"], sc["H"],
                                   sc["W"], _lib.SOLVERS[solver], ctypes.c_void_p(out.data_ptr()), stream, err,
                                   len(err))
    torch.cuda.synchronize()
    return rc, err.value.decode()


SCENES = {
    "translate_64x64_T16": lambda: scenes.config1(),
    "rotate_72x40_T8": lambda: scenes.small_scene("rotate", subdiv=2, T=8, H=40, W=72),
    "rotate_96x80_T16_subdiv4": lambda: scenes.config2(T=16, H=80, W=96),
}


@pytest.mark.parametrize("solver", ["fast", "plain"])
@pytest.mark.parametrize("name", sorted(SCENES))
def test_noalloc_matches_allocating_render_on_two_calls(name, solver):
    import paper_2602_07860_gb300 as mbr
    from paper_2602_07860_gb300 import _lib
    L = _lib.load()
    sc = SCENES[name]()
    ctx = mbr.Context()
    v, f, a = mbr.mesh_tensors(sc)
    ref = ctx.render_blur(v, f, a, mbr.motion_from_dict(sc["motion"]), mbr.camera_from_dict(sc["camera"]),
                          sc["T"], sc["H"], sc["W"], solver)
    torch.cuda.synchronize()
    for _ in range(2):
        out = torch.full((sc["H"], sc["W"], 4), float("nan"), dtype=torch.float32, device="cuda")
        rc, msg = _call_noalloc(L, sc, solver, out)
        assert rc == _lib.MBR_OK, msg
        assert torch.isfinite(out).all()
        assert float((out - ref).abs().max()) <= TOL


def test_noalloc_rejects_renders_beyond_its_static_scratch():
    from paper_2602_07860_gb300 import _lib
    L = _lib.load()
    sc = scenes.config2()  # 64 per-sub-frame record sets of 5120 faces need more than 32 MiB
    out = torch.zeros((sc["H"], sc["W"], 4), dtype=torch.float32, device="cuda")
    rc, msg = _call_noalloc(L, sc, "plain", out)
    assert rc == _lib.MBR_ERR_ARG
    assert "static scratch" in msg
    # a small render still works afterwards
    small = scenes.config1()
    out2 = torch.zeros((small["H"], small["W"], 4), dtype=torch.float32, device="cuda")
    rc, msg = _call_noalloc(L, small, "fast", out2)
    assert rc == _lib.MBR_OK, msg
    assert np.isfinite(out2.cpu().numpy()).all()
