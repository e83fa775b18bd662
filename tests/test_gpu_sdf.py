"""SDF -> mesh extraction on the GPU (mbr_sdf_extract, the rotational recovery's extractor)
against the FP64 oracle: the same triangles (as oriented triples of grid edges, bit-exact
topology), vertex positions within single-precision rounding, and the adjoint dL/dsdf."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2602_07860_gb300 as mbr
    return mbr.Context()


def _grid(n, lo=-1.2, hi=1.2):
    h = (hi - lo) / n
    ax = lo + h * np.arange(n + 1)
    Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
    return X, Y, Z, np.array([lo, lo, lo]), h


def _canon(faces, edges):
    """Each face as its three (a, b) grid-edge keys, rotated to start at the smallest key (the
    winding is kept), all faces sorted."""
    keys = [tuple(map(tuple, edges[f])) for f in faces]
    out = []
    for k in keys:
        r = min(range(3), key=lambda q: k[q])
        out.append(k[r:] + k[:r])
    return sorted(out)


def _gpu(ctx, s, lo, h):
    sd = torch.as_tensor(s.astype(np.float32), device="cuda")
    v, f, e = ctx.sdf_extract(sd, lo.astype(np.float32), np.float32(h))
    torch.cuda.synchronize()
    return sd, v, f, e


def _fields():
    rng = np.random.default_rng(11)
    X, Y, Z, lo, h = _grid(24)
    yield "sphere_24", np.sqrt(X ** 2 + Y ** 2 + Z ** 2) - 0.83, lo, h
    X, Y, Z, lo, h = _grid(17, -1.0, 1.0)
    yield "ellipsoid_inclined_17", (4 * X ** 2 + 2.5 * Y ** 2 + 2.5 * Z ** 2 - 3 * Y * Z - 1.0) / 4.0, lo, h
    for t in range(4):
        n = int(rng.integers(3, 10))
        X, Y, Z, lo, h = _grid(n, -1.0, 1.0)
        s = rng.normal(size=X.shape)
        if t % 2 == 0:
            s = np.round(s * 2) / 2  # exact zeros on the grid
        yield f"random_{t}_n{n}", s, lo, h


@pytest.mark.parametrize("case", list(range(6)))
def test_extraction_matches_oracle(ctx, case):
    name, s, lo, h = list(_fields())[case]
    s32 = s.astype(np.float32).astype(np.float64)  # both sides see the same samples
    lo32, h32 = lo.astype(np.float32).astype(np.float64), float(np.float32(h))
    sd, v, f, e = _gpu(ctx, s32, lo32, h32)
    ov, oe, of = oracle.sdf_extract(s32, lo32, h32)
    v, f, e = v.cpu().numpy(), f.cpu().numpy(), e.cpu().numpy().astype(np.int64)
    assert len(v) == len(ov) and len(f) == len(of), name
    assert _canon(f, e) == _canon(of, oe), name
    # positions: match vertices by their grid edge
    order = np.lexsort((e[:, 1], e[:, 0]))
    assert np.array_equal(e[order], oe)
    assert np.abs(v[order] - ov).max() <= 2e-6 * max(1.0, np.abs(ov).max()), name


def test_adjoint_matches_oracle(ctx):
    X, Y, Z, lo, h = _grid(20)
    s = (np.sqrt(X ** 2 + (1.3 * Y) ** 2 + Z ** 2) - 0.8 + 0.05 * np.sin(4 * X)).astype(np.float32).astype(np.float64)
    lo32, h32 = lo.astype(np.float32).astype(np.float64), float(np.float32(h))
    sd, v, f, e = _gpu(ctx, s, lo32, h32)
    rng = np.random.default_rng(2)
    g = rng.normal(size=tuple(v.shape)).astype(np.float32)
    gs = ctx.sdf_extract_backward(sd, np.float32(h32), e, torch.as_tensor(g, device="cuda")).cpu().numpy()
    ev = e.cpu().numpy().astype(np.int64)
    order = np.lexsort((ev[:, 1], ev[:, 0]))
    ov, oe, of = oracle.sdf_extract(s, lo32, h32)
    ref = oracle.sdf_extract_backward(s, lo32, h32, oe, g[order].astype(np.float64))
    scale = np.abs(ref).max()
    assert scale > 0
    assert np.abs(gs - ref).max() <= 1e-4 * scale


def test_empty_field_and_capacity_errors(ctx):
    from paper_2602_07860_gb300._lib import MbrError
    X, Y, Z, lo, h = _grid(6)
    sd, v, f, e = _gpu(ctx, np.ones_like(X), lo, h)
    assert v.shape == (0, 3) and f.shape == (0, 3)
    import ctypes
    counts = (ctypes.c_int32 * 2)()
    s = torch.as_tensor((np.sqrt(X ** 2 + Y ** 2 + Z ** 2) - 0.7).astype(np.float32), device="cuda")
    lo_c = (ctypes.c_float * 3)(*[float(x) for x in lo])
    out_v = torch.empty((4, 3), device="cuda")
    out_f = torch.empty((4, 3), dtype=torch.int32, device="cuda")
    rc = ctx.L.mbr_sdf_extract(ctx.h, 6, ctypes.c_void_p(s.data_ptr()), lo_c, float(h), 4, 4,
                               ctypes.c_void_p(out_v.data_ptr()), ctypes.c_void_p(out_f.data_ptr()), None, counts,
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc != 0 and counts[0] > 4 and counts[1] > 4  # sizes reported, nothing written
    with pytest.raises(ValueError):
        ctx.sdf_extract(s[:3], lo, h)  # not a cube of samples
    with pytest.raises(MbrError):
        ctx.sdf_extract(s, lo, -1.0)  # the library rejects a non-positive spacing
