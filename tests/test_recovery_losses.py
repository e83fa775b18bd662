"""The regularisers of the translational recovery loss (loss-term appendix), on CPU: the
smoothness term is zero on a flat fold and (cos + 1)^2 on a folded one; the displacement Laplacian
vanishes for a rigid translation of the template; the edge-opposite table of a closed mesh has one
entry per edge."""
import math

import numpy as np
import torch

import scenes


def test_smoothness_flat_and_folded():
    from paper_2602_07860_gb300.recovery import edge_opposites, smoothness_loss
    faces = torch.tensor([[0, 1, 2], [1, 0, 3]], dtype=torch.int32)
    flat = torch.tensor([[0., 0, 0], [1, 0, 0], [0.5, 1, 0], [0.5, -1, 0]])
    q = edge_opposites(faces)
    assert q.shape == (4, 1)
    assert float(smoothness_loss(flat, q)) < 1e-12
    for ang in (math.pi / 2, math.pi / 3):
        folded = flat.clone()
        folded[3] = torch.tensor([0.5, -math.cos(math.pi - ang), math.sin(math.pi - ang)])  # dihedral angle ang
        cos = math.cos(ang)
        assert abs(float(smoothness_loss(folded, q)) - (cos + 1) ** 2) < 1e-6


def test_laplacian_of_rigid_translation_is_zero_and_edges_of_closed_mesh():
    from paper_2602_07860_gb300.recovery import edge_index, edge_opposites, laplacian_delta_loss
    v, f = scenes.uv_sphere()
    assert v.shape == (1352, 3) and f.shape == (2700, 3)
    V = torch.as_tensor(v, dtype=torch.float64)
    F = torch.as_tensor(f)
    e = edge_index(F, V.shape[0])
    assert float(laplacian_delta_loss(V + torch.tensor([0.3, -0.2, 0.1], dtype=torch.float64), V, e)) < 1e-20
    bump = V.clone()
    bump[0] += 0.1
    assert float(laplacian_delta_loss(bump, V, e)) > 0
    assert edge_opposites(F).shape[1] == 3 * f.shape[0] // 2  # closed: every edge has two faces


def test_laplacian_of_one_moved_vertex_on_a_tetrahedron():
    """Every vertex of a tetrahedron has the other three as neighbours.  Moving vertex 0 by e gives
    Laplacians e at vertex 0 and -e/3 at the others: |e|^2 (1 + 3/9) in total."""
    from paper_2602_07860_gb300.recovery import edge_index, laplacian_delta_loss
    V = torch.tensor([[1., 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=torch.float64)
    F = torch.tensor([[0, 1, 2], [0, 3, 1], [0, 2, 3], [1, 3, 2]])
    e = edge_index(F, 4)
    assert e.shape == (2, 12)
    moved = V.clone()
    step = torch.tensor([0.2, -0.1, 0.3], dtype=torch.float64)
    moved[0] += step
    expect = float((step * step).sum()) * (1.0 + 3.0 / 9.0)
    assert abs(float(laplacian_delta_loss(moved, V, e)) - expect) < 1e-14
