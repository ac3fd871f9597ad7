"""Host logic of training (no GPU): which parts of a packed grid
the optimiser updates and where the gradient's SDF entries sit, in every
FP32 grid layout."""
import torch

import paper_2412_10084_gb300 as ps
from paper_2412_10084_gb300.fit import trainable_grid


def buffers(gd):
    vb, gb = ps.grid_bytes(gd)
    return torch.zeros(vb // 16, 4), torch.ones(gb // 16, 4)


def test_node_records():
    gd = ps.grid_desc((4, 5, 6), (0, 0, 0), (1, 1, 1))
    values, grad = buffers(gd)
    v, g, sdf = trainable_grid(gd, values, grad)
    assert v.numel() == values.numel() and g.numel() == grad.numel()
    sdf.zero_()
    assert float(grad[:, 0].abs().sum()) == 0 and bool((grad[:, 1:] == 1).all())


def test_sparse_bricks_leave_the_table_alone():
    gd = ps.grid_desc((32, 16, 48), (0, 0, 0), (1, 1, 1), n_bricks=2, empty_sdf=1.0)
    values, grad = buffers(gd)
    w = ps.table_words(gd)
    v, g, sdf = trainable_grid(gd, values, grad)
    assert v.numel() == g.numel() == 2 * 4096 * 4
    assert g.data_ptr() == grad.data_ptr() + 4 * w and v.data_ptr() == values.data_ptr() + 4 * w
    assert sdf.numel() == 2 * 4096
    sdf.zero_()
    flat = grad.view(-1)
    assert bool((flat[:w] == 1).all())                       # the table
    rec = flat[w:].view(-1, 4)
    assert float(rec[:, 0].abs().sum()) == 0 and bool((rec[:, 1:] == 1).all())


def test_triplanes_sdf_array_first():
    gd = ps.grid_desc((9, 10, 11), (0, 0, 0), (1, 1, 1), feat_layout=ps.FEAT_TRIPLANE)
    values, grad = buffers(gd)
    v, g, sdf = trainable_grid(gd, values, grad)
    n = 9 * 10 * 11
    assert sdf.numel() == n and sdf.data_ptr() == grad.data_ptr()
    sdf.zero_()
    flat = grad.view(-1)
    assert float(flat[:n].abs().sum()) == 0 and bool((flat[n:] == 1).all())


def test_autograd_gives_a_sparse_brick_table_zero_gradient(monkeypatch):
    """The gradient buffer of a sparse grid starts with a copy of the table's
    bits (for unpacking); the autograd gradient of scene.grid must not carry
    them (as floats, a -1 entry is a NaN)."""
    import types
    gd = ps.grid_desc((32, 16, 16), (0, 0, 0), (1, 1, 1), n_bricks=1, empty_sdf=1.0)
    _, gb = ps.grid_bytes(gd)
    w = ps.table_words(gd)
    gg = torch.full((gb // 4,), float("nan"))
    monkeypatch.setattr(ps, "render_backward", lambda *a, **k: (gg, None, None))
    scene = types.SimpleNamespace(n_bricks=1, descs=lambda n_fresnel: (gd, None, None))
    empty = torch.empty(0)
    ctx = types.SimpleNamespace(saved_tensors=(empty,) * 6, storage=(None, None), has_t=False,
                                scene=scene, params=types.SimpleNamespace(n_fresnel=3))
    d_grid = ps.RenderFunction.backward(ctx, torch.zeros(0, 3), None, None)[0]
    assert bool((d_grid[:w] == 0).all()) and bool(d_grid[w:].isnan().all())
