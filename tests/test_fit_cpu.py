"""Host logic of training (no GPU): which parts of a packed grid
the optimiser updates and where the gradient's SDF entries sit, in every
FP32 grid layout."""
import pytest
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
                                scene=scene, params=types.SimpleNamespace(n_fresnel=3),
                                check_status=False)
    d_grid = ps.RenderFunction.backward(ctx, torch.zeros(0, 3), None, None)[0]
    assert bool((d_grid[:w] == 0).all()) and bool(d_grid[w:].isnan().all())


def test_autograd_backward_raises_when_a_kernel_stopped_early(monkeypatch):
    """With the status check on (the default), a nonzero device status word
    (a render kernel gave up waiting on its tensor-core work and returned with
    part of its gradients missing) raises instead of handing them on."""
    import types
    gd = ps.grid_desc((16, 16, 16), (0, 0, 0), (1, 1, 1))
    monkeypatch.setattr(ps, "render_backward", lambda *a, **k: (torch.zeros(4), None, None))
    monkeypatch.setattr(ps, "device_status", lambda stream=None: 1)
    scene = types.SimpleNamespace(n_bricks=0, descs=lambda n_fresnel: (gd, None, None))
    empty = torch.empty(0)
    ctx = types.SimpleNamespace(saved_tensors=(empty,) * 6, storage=(None, None), has_t=False,
                                scene=scene, params=types.SimpleNamespace(n_fresnel=3),
                                check_status=True)
    with pytest.raises(ps.LibraryError, match="stopped early"):
        ps.RenderFunction.backward(ctx, torch.zeros(0, 3), None, None)
    ctx.check_status = False
    assert ps.RenderFunction.backward(ctx, torch.zeros(0, 3), None, None)[0].numel() == 4


def test_pack_sparse_rejects_a_slot_named_twice():
    """Two table entries naming one slot would alias one record block; more
    named slots than stored bricks would index past the records."""
    gd = ps.grid_desc((32, 32, 16), (0, 0, 0), (1, 1, 1), n_bricks=2, empty_sdf=1.0)
    sdf, feat = torch.zeros(16, 32, 32), torch.zeros(16, 32, 32, 3)
    dup = torch.tensor([[[0, -1], [0, 1]]], dtype=torch.int32)
    with pytest.raises(ps.LibraryError, match="at most once"):
        ps.pack_sparse(gd, dup, sdf, feat)
    too_many = torch.tensor([[[0, 1], [2, -1]]], dtype=torch.int32)
    with pytest.raises(ps.LibraryError, match="at most once"):
        ps.pack_sparse(gd, too_many, sdf, feat)
    ok = torch.tensor([[[1, -1], [0, -1]]], dtype=torch.int32)
    with pytest.raises(ps.LibraryError, match="CUDA"):  # valid table: fails only on the CPU tensors
        ps.pack_sparse(gd, ok, sdf, feat)
