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


def _call_noalloc(L, sc, solver, out, tensors=None):
    import paper_2602_07860_gb300 as mbr
    from paper_2602_07860_gb300 import _lib
    v, f, a = tensors if tensors is not None else mbr.mesh_tensors(sc)
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


def test_noalloc_allocates_no_device_memory():
    """The point of the entry point: after a first call (which looks up the static array's
    address), a call leaves the device's free memory exactly unchanged."""
    import paper_2602_07860_gb300 as mbr
    from paper_2602_07860_gb300 import _lib
    L = _lib.load()
    sc = scenes.config2(T=16, H=80, W=96)
    out = torch.zeros((sc["H"], sc["W"], 4), dtype=torch.float32, device="cuda")
    tensors = mbr.mesh_tensors(sc)  # every input exists before the measured calls
    rc, msg = _call_noalloc(L, sc, "fast", out, tensors)
    assert rc == _lib.MBR_OK, msg
    free0, _ = torch.cuda.mem_get_info()
    for solver in ("fast", "plain"):
        rc, msg = _call_noalloc(L, sc, solver, out, tensors)
        assert rc == _lib.MBR_OK, msg
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_reports_a_raster_wait_that_gave_up():
    """A bounded raster wait that gives up (forced by the test hook: claimed units are never
    published, so the waiting warps run out of polls) is reported as MBR_ERR_TIMEOUT by the same
    call when it checks at once, otherwise by the next call on the device; the call after that
    renders completely again."""
    from paper_2602_07860_gb300 import _lib
    L = _lib.load()
    sc = scenes.small_scene("rotate", subdiv=2, T=8, H=40, W=72)
    ref = torch.zeros((sc["H"], sc["W"], 4), dtype=torch.float32, device="cuda")
    assert _call_noalloc(L, sc, "fast", ref)[0] == _lib.MBR_OK
    out = torch.zeros_like(ref)
    try:
        assert L.mbr_debug_wait_limit(2000, 1, 1) == _lib.MBR_OK
        rc, msg = _call_noalloc(L, sc, "fast", out)
        assert rc == _lib.MBR_ERR_TIMEOUT, (rc, msg)
        assert L.mbr_debug_wait_limit(2000, 1, 0) == _lib.MBR_OK
        rc, msg = _call_noalloc(L, sc, "fast", out)
        assert rc == _lib.MBR_OK, msg  # nothing waited for the raster: the report comes next
    finally:
        L.mbr_debug_wait_limit(0, 0, 0)
    rc, msg = _call_noalloc(L, sc, "fast", out)
    assert rc == _lib.MBR_ERR_TIMEOUT and "bounded wait" in msg, (rc, msg)
    rc, msg = _call_noalloc(L, sc, "fast", out)
    assert rc == _lib.MBR_OK, msg
    assert float((out - ref).abs().max()) <= 2e-6


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
