"""Bounded device-side waits of the persistent raster (failure detection without a GPU fault).

The raster CTAs hand work units to their warps through shared-memory flags, and every wait on
such a flag gives up after a bounded number of polls.  The test hook mbr_debug_wait_limit makes
the CTAs never publish a claimed unit (a flag that nothing sets) with a short limit: every
waiting warp then gives up, sets the kernel's status word and returns, so the launch ends by
itself and the context stays usable.  The tests check the status reaches the caller as
MBR_ERR_TIMEOUT -- from the same call when asked to check at once, otherwise from the next call
-- and that the following renders are complete again."""
import numpy as np
import pytest
import torch

import scenes
from gpu_util import gpu_inputs

pytestmark = pytest.mark.gpu

POLLS = 2000  # about 0.13 ms per wait before it gives up


@pytest.fixture
def hook():
    from paper_2602_07860_gb300 import _lib
    L = _lib.load()

    def set_(polls, stall, check_now):
        assert L.mbr_debug_wait_limit(polls, stall, check_now) == _lib.MBR_OK
    yield set_
    L.mbr_debug_wait_limit(0, 0, 0)


def _render(ctx, sc, solver):
    v, f, a, mo, ca = gpu_inputs(sc)
    img = ctx.render_blur(v, f, a, mo, ca, sc["T"], sc["H"], sc["W"], solver)
    torch.cuda.synchronize()
    return img.clone()


def test_hook_rejects_unbounded_stall():
    from paper_2602_07860_gb300 import _lib
    L = _lib.load()
    assert L.mbr_debug_wait_limit(0, 1, 1) == _lib.MBR_ERR_ARG       # a stall needs a limit
    assert L.mbr_debug_wait_limit(1 << 21, 1, 1) == _lib.MBR_ERR_ARG  # and a short one
    assert L.mbr_debug_wait_limit(-1, 0, 0) == _lib.MBR_ERR_ARG
    assert L.mbr_debug_wait_limit(0, 0, 0) == _lib.MBR_OK


@pytest.mark.parametrize("solver", ["fast", "plain"])
def test_give_up_reported_by_the_same_call(hook, solver):
    import paper_2602_07860_gb300 as mbr
    from paper_2602_07860_gb300._lib import MBR_ERR_TIMEOUT, MbrError
    sc = scenes.small_scene("rotate", subdiv=2, T=8, H=48, W=64)
    ref = _render(mbr.Context(), sc, solver)
    ctx = mbr.Context()
    hook(POLLS, 1, 1)
    with pytest.raises(MbrError) as e:
        _render(ctx, sc, solver)
    assert e.value.code == MBR_ERR_TIMEOUT
    hook(0, 0, 0)
    img = _render(ctx, sc, solver)  # the report was consumed; the context works again
    assert float((img - ref).abs().max()) <= 2e-6


@pytest.mark.parametrize("solver", ["fast", "plain"])
def test_give_up_reported_by_the_next_call(hook, solver):
    import paper_2602_07860_gb300 as mbr
    from paper_2602_07860_gb300._lib import MBR_ERR_TIMEOUT, MbrError
    sc = scenes.small_scene("rotate", subdiv=2, T=8, H=48, W=64)
    ref = _render(mbr.Context(), sc, solver)
    ctx = mbr.Context()
    hook(POLLS, 1, 0)
    bad = _render(ctx, sc, solver)  # returns: the raster gave up, nothing waited for it
    hook(0, 0, 0)
    assert float(torch.nan_to_num(bad - ref, nan=1.0).abs().max()) > 1e-3  # most units were never drawn
    with pytest.raises(MbrError) as e:
        _render(ctx, sc, solver)
    assert e.value.code == MBR_ERR_TIMEOUT
    img = _render(ctx, sc, solver)
    assert float((img - ref).abs().max()) <= 2e-6


def test_adjoint_give_up_reported(hook):
    import paper_2602_07860_gb300 as mbr
    from paper_2602_07860_gb300._lib import MBR_ERR_TIMEOUT, MbrError
    sc = scenes.small_scene("rotate", subdiv=2, T=8, H=48, W=64)
    v, f, a, mo, ca = gpu_inputs(sc)
    G = torch.ones((sc["H"], sc["W"], 4), device="cuda")
    ref, _ = mbr.Context().render_blur_backward(v, f, a, mo, ca, sc["T"], sc["H"], sc["W"], G, "fast")
    ctx = mbr.Context()
    ctx.render_blur(v, f, a, mo, ca, sc["T"], sc["H"], sc["W"], "fast")
    hook(POLLS, 1, 1)
    with pytest.raises(MbrError) as e:
        ctx.render_blur_backward(v, f, a, mo, ca, sc["T"], sc["H"], sc["W"], G, "fast", reuse_forward=True)
    assert e.value.code == MBR_ERR_TIMEOUT
    hook(0, 0, 0)
    gv, _ = ctx.render_blur_backward(v, f, a, mo, ca, sc["T"], sc["H"], sc["W"], G, "fast")
    torch.cuda.synchronize()
    assert np.allclose(gv.cpu().numpy(), ref.cpu().numpy(), rtol=1e-4, atol=1e-5 * float(ref.abs().max()))
