"""The SDF regularisers of the rotational recovery (loss-term appendix) on CPU tensors, against
closed forms: the Eikonal term vanishes on an exact distance field and is |c - 1| for a field
scaled by c; the singular-Hessian term vanishes on a linear field and is O(h) on a sphere's
distance (its Hessian is singular); the sign term of one sign-changing edge is
softplus(-s_a) + softplus(s_b) for s_a < 0 < s_b."""
import math

import numpy as np
import torch

from paper_2602_07860_gb300.sdf import eikonal_loss, grid_points, sign_loss, singular_hessian_loss


def _sphere(n, R=0.7, lo=-1.0, hi=1.0):
    h = (hi - lo) / n
    P = grid_points(n, (lo, lo, lo), h, device="cpu", dtype=torch.float64)
    return P.norm(dim=-1) - R, h


def test_eikonal_vanishes_on_a_distance_field_and_scales():
    s, h = _sphere(32)
    s = s + 0.0 * s  # exact distance away from the centre
    assert float(eikonal_loss(s, h)) < 0.01  # central differences miss only near the centre
    assert abs(float(eikonal_loss(3.0 * s, h)) - 2.0) < 0.03
    X = grid_points(8, (0.0, 0.0, 0.0), 0.25, device="cpu", dtype=torch.float64)
    plane = 0.6 * X[..., 0] + 0.8 * X[..., 2]  # unit gradient everywhere
    assert float(eikonal_loss(plane, 0.25)) < 1e-12


def test_singular_hessian_vanishes_on_linear_and_sphere_fields():
    X = grid_points(10, (-1.0, -1.0, -1.0), 0.2, device="cpu", dtype=torch.float64)
    lin = 0.3 * X[..., 0] - 0.5 * X[..., 1] + 0.2 * X[..., 2] + 0.05
    assert float(singular_hessian_loss(lin, 0.2)) < 1e-10
    s, h = _sphere(40)
    # det of the Hessian of |x| is 0; the differences leave an O(h^2 / r^3) remainder
    assert float(singular_hessian_loss(s, h)) < 0.05
    quad = (X ** 2).sum(-1) - 0.5  # Hessian 2 I: det 8 everywhere near the surface
    assert abs(float(singular_hessian_loss(quad, 0.2, band=5.0)) - 8.0) < 1e-9


def test_sign_loss_of_one_crossing_edge():
    s = torch.full((2, 2, 2), 1.0, dtype=torch.float64)
    s[0, 0, 0] = -0.3  # crosses to its three axis neighbours (values 1.0)
    sp = lambda x: math.log1p(math.exp(x))
    want = 3 * (sp(0.3) + sp(1.0))  # BCE(sigmoid(-0.3), 1) + BCE(sigmoid(1), 0) per edge
    assert abs(float(sign_loss(s)) - want) < 1e-12
    assert float(sign_loss(torch.ones(3, 3, 3, dtype=torch.float64))) == 0.0
