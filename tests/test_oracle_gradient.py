"""The oracle's hand-derived FP64 adjoint against central finite differences of its own forward
(h = 1e-6), skipping coordinates where the +-h renders change any discrete choice (the oracle's
decision hash), plus rigid-shift and albedo-linearity checks."""
import numpy as np
import pytest

import oracle
import scenes


def _loss(sc, G, mode, **kw):
    r = oracle.render(sc, mode, **kw)
    return float(np.sum(r["rgba"] * G)), int(r["counters"][oracle.CNT_HASH])


def _scene(kind, delta, prob="exp", interp="screen"):
    sc = scenes.small_scene(kind, subdiv=1, T=4, H=22, W=26, lmax=3, sigma=0.08, d=(0.9, 0.2, 0.4))
    sc["camera"] = dict(sc["camera"], delta=delta, prob=prob, interp=interp)
    return sc


@pytest.mark.parametrize("mode,kind,delta,prob,interp",
                         [(m, k, d, "exp", "screen") for m in ("exact", "linear", "fast")
                          for k in ("rotate", "translate") for d in (1e-4, 2e-3)] +
                         [(m, k, 2e-3, "sigmoid", "screen") for m in ("exact", "fast") for k in ("rotate", "translate")] +
                         [(m, k, 1e-4, "exp", "perspective") for m in ("exact", "fast") for k in ("rotate", "translate")])
def test_adjoint_matches_central_differences(mode, kind, delta, prob, interp):
    """prob 'sigmoid' is the SoftRas probability map (dA/dd = -A (1 - A) / delta); interp
    'perspective' the perspective-correct attribute weights (gradients also reach the depths)."""
    _fd_check(_scene(kind, delta, prob, interp), mode)


@pytest.mark.parametrize("mode,kind", [("exact", "rotate"), ("fast", "rotate"), ("fast", "translate")])
def test_single_precision_truncated_adjoint_matches_central_differences(mode, kind):
    """With soft32 (factors with exp(-d/delta) <= 2^-25 dropped, the kernels' truncation) the
    adjoint is still the exact derivative of the truncated forward."""
    _fd_check(_scene(kind, 1e-4), mode, soft32=True)


def _fd_check(sc, mode, **kw):
    rng = np.random.default_rng(17)
    G = rng.normal(size=(sc["H"], sc["W"], 4))
    gv, ga, _ = oracle.render_backward(sc, G, mode, **kw)
    _, h0 = _loss(sc, G, mode, **kw)
    h = 1e-6
    V = len(sc["verts"])
    coords = [(int(v), int(c)) for v, c in zip(rng.integers(0, V, 40), rng.integers(0, 3, 40))]
    checked = 0
    scale = np.max(np.abs(gv))
    for v, c in coords:
        plus = dict(sc, verts=sc["verts"].copy())
        minus = dict(sc, verts=sc["verts"].copy())
        plus["verts"][v, c] += h
        minus["verts"][v, c] -= h
        lp, hp = _loss(plus, G, mode, **kw)
        lm, hm = _loss(minus, G, mode, **kw)
        if hp != h0 or hm != h0:
            continue  # a discrete choice changed inside [-h, h]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gv[v, c]) <= 1e-5 * abs(fd) + 1e-7 * scale + 1e-9, (v, c, fd, gv[v, c])
        checked += 1
    assert checked >= 25
    # albedo enters linearly: dL/dalbedo is exact
    for v, c in coords[:10]:
        plus = dict(sc, albedo=sc["albedo"].copy())
        plus["albedo"][v, c] += 1.0
        lp, _ = _loss(plus, G, mode, **kw)
        l0, _ = _loss(sc, G, mode, **kw)
        assert abs((lp - l0) - ga[v, c]) < 1e-9 * max(1.0, abs(ga[v, c]))


@pytest.mark.parametrize("mode", ["exact", "fast"])
def test_rigid_shift_gradient_sums(mode):
    """Moving every vertex by the same small offset c: dL/dc = sum_v dL/dv (normals unchanged)."""
    sc = _scene("translate", 2e-3)
    rng = np.random.default_rng(23)
    G = rng.normal(size=(sc["H"], sc["W"], 4))
    gv, _, _ = oracle.render_backward(sc, G, mode)
    h = 1e-7
    for axis in range(3):
        e = np.zeros(3)
        e[axis] = h
        lp, hp = _loss(dict(sc, verts=sc["verts"] + e), G, mode)
        lm, hm = _loss(dict(sc, verts=sc["verts"] - e), G, mode)
        _, h0 = _loss(sc, G, mode)
        if hp != h0 or hm != h0:
            continue
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gv[:, axis].sum()) <= 1e-5 * abs(fd) + 1e-6 * np.abs(gv).max()
