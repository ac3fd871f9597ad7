"""Grid-level training terms (Sec. 3.3, Eqs. 11-15) on the GPU against the FP64
oracle: the 5^3 Gaussian smoothing and its transpose, the per-voxel SDF terms,
the tri-plane and probe smoothness terms, in every grid layout."""
import numpy as np
import pytest
import torch

import synth
from helpers import log_errors, rel_err_tensor
from oracle import regularizers as R

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2412_10084_gb300 as ps

# FP32 against FP64.  A smoothed node is a convex combination of 125 inputs
# taken in three passes of 5 FMAs (<= 15 roundings of values bounded by
# max|in|); the transposed rows sum to at most 2.2 per axis.  The stencil
# gradients are short sums of terms of one scale (atomics in any order).
SMOOTH_ATOL = 4e-6       # x max|input|
SMOOTH_T_ATOL = 4e-5     # x max|input|
GRAD_RTOL = 1e-4         # x max|reference|, per tensor
LOSS_RTOL = 1e-4

# (name, feature dtype, feature layout): FP32 node records, BF16 node features
# (plain FP32 SDF array), tile tri-planes (plain FP32 SDF array)
LAYOUTS = [("nodes", 0, 0), ("bf16", 1, 0), ("triplane", 0, 1)]


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def fields(dims, seed, noise=0.02):
    """A sphere SDF with an off-node centre (|grad s| ~ 1 everywhere it is
    differenced) plus seeded noise, and a raw grid s_hat around it."""
    g = synth.rng(seed)
    bmin, bmax = (-1.0, -1.1, -0.9), (1.05, 1.0, 1.1)
    s = synth.sphere_sdf(dims, bmin, bmax, (0.113, -0.071, 0.052), 0.6).astype(np.float64)
    s = (s + noise * g.normal(size=s.shape)).astype(np.float32)
    s_hat = (s + 0.05 * g.normal(size=s.shape)).astype(np.float32)
    return s, s_hat, bmin, bmax


def make_grid(dims, bmin, bmax, s, feat_dtype, layout, seed):
    g = synth.rng(seed + 7)
    gd = ps.grid_desc(dims, bmin, bmax, 3, feat_dtype, layout)
    Rx, Ry, Rz = dims
    if layout == ps.FEAT_TRIPLANE:
        feat = synth.tile_planes(dims, 3, g)
    else:
        feat = g.normal(size=(Rz, Ry, Rx, 3)).astype(np.float32)
    return gd, ps.pack_grid(gd, dev(s), dev(feat)), feat


@pytest.mark.parametrize("dims", [(37, 29, 21), (2, 3, 5), (64, 8, 9)])
@pytest.mark.parametrize("layout", LAYOUTS, ids=lambda v: v[0])
def test_smooth_parity_and_features_untouched(dims, layout):
    _, fdt, lay = layout
    _, s_hat, bmin, bmax = fields(dims, 3)
    zero = np.zeros_like(s_hat)
    gd, values, feat = make_grid(dims, bmin, bmax, zero, fdt, lay, 3)
    ps.sdf_smooth(gd, dev(s_hat), values)
    sdf, f2 = ps.unpack_grid(gd, values, which=ps.GRID_VALUES)
    ref = R.smooth(s_hat)
    err = float(np.max(np.abs(sdf.cpu().numpy() - ref)))
    log_errors(f"smooth {layout[0]} {dims}", {"abs_over_max": float(err / np.max(np.abs(s_hat)))})
    assert err <= SMOOTH_ATOL * np.max(np.abs(s_hat)), err
    # the features are not touched (exact, in their storage precision)
    if fdt == ps.F32:
        assert np.array_equal(f2.cpu().numpy(), feat)
    else:
        f_once = ps.unpack_grid(gd, make_grid(dims, bmin, bmax, zero, fdt, lay, 3)[1],
                                which=ps.GRID_VALUES)[1]
        assert torch.equal(f2, f_once)


@pytest.mark.parametrize("dims", [(37, 29, 21), (2, 2, 2), (70, 5, 17)])
@pytest.mark.parametrize("layout", LAYOUTS, ids=lambda v: v[0])
def test_smooth_adjoint_parity(dims, layout):
    _, fdt, lay = layout
    g = synth.rng(11)
    gd = ps.grid_desc(dims, (0, 0, 0), (1, 1, 1), 3, fdt, lay)
    _, gbytes = ps.grid_bytes(gd)
    Rx, Ry, Rz = dims
    ds = g.normal(size=(Rz, Ry, Rx)).astype(np.float32)
    grad = torch.zeros(gbytes // 4, dtype=torch.float32, device="cuda")
    if lay == ps.FEAT_TRIPLANE:
        grad[:ds.size] = dev(ds.ravel())
    else:
        grad.view(-1, 4)[:ds.size, 0] = dev(ds.ravel())
        grad.view(-1, 4)[:ds.size, 1:] = 7.0  # other slots must not leak in
    out = dev(g.normal(size=ds.shape))
    base = out.clone()
    ps.sdf_smooth_adjoint(gd, grad, out, accumulate=True)
    ref = R.smooth_adjoint(ds)
    err_acc = float(np.max(np.abs(out.cpu().numpy() - base.cpu().numpy() - ref)))
    ps.sdf_smooth_adjoint(gd, grad, out, accumulate=False)
    err = float(np.max(np.abs(out.cpu().numpy() - ref)))
    scale = np.max(np.abs(ds))
    log_errors(f"smooth adjoint {layout[0]} {dims}", {"abs_over_max": float(err / scale)})
    assert err <= SMOOTH_T_ATOL * scale, err
    assert err_acc <= SMOOTH_T_ATOL * (scale + 4.0), err_acc


def test_smooth_adjoint_is_the_transpose_on_device():
    """<G x, y> = <x, G^T y> with both operators on the GPU (FP64 dot products
    of the FP32 results)."""
    dims = (45, 19, 33)
    g = synth.rng(5)
    gd = ps.grid_desc(dims, (0, 0, 0), (1, 1, 1), 3, ps.BF16, ps.FEAT_NODES)
    vb, gb = ps.grid_bytes(gd)
    Rx, Ry, Rz = dims
    x = g.normal(size=(Rz, Ry, Rx)).astype(np.float32)
    y = g.normal(size=(Rz, Ry, Rx)).astype(np.float32)
    values = torch.zeros(vb // 4, dtype=torch.float32, device="cuda")
    ps.sdf_smooth(gd, dev(x), values)
    gx = values[:x.size].cpu().numpy().astype(np.float64)
    grad = torch.zeros(gb // 4, dtype=torch.float32, device="cuda")
    grad.view(-1, 4)[:y.size, 0] = dev(y.ravel())
    gty = torch.zeros(x.shape, dtype=torch.float32, device="cuda")
    ps.sdf_smooth_adjoint(gd, grad, gty, accumulate=False)
    lhs = float(np.dot(gx, y.ravel().astype(np.float64)))
    rhs = float(np.dot(x.ravel().astype(np.float64), gty.cpu().numpy().ravel().astype(np.float64)))
    assert abs(lhs - rhs) <= 1e-5 * np.sqrt(x.size) * 2, (lhs, rhs)


def _sdf_terms_case(dims, layout, lam, seed, lam_features=0.0):
    _, fdt, lay = layout
    s, s_hat, bmin, bmax = fields(dims, seed)
    gd, values, feat = make_grid(dims, bmin, bmax, s, fdt, lay, seed)
    _, gbytes = ps.grid_bytes(gd)
    grad = torch.zeros(gbytes // 4, dtype=torch.float32, device="cuda")
    d_hat = torch.zeros(s.shape, dtype=torch.float32, device="cuda")
    loss = torch.zeros(4, dtype=torch.float32, device="cuda")
    ps.grid_regularizers(gd, dev(s_hat), values, grad, d_hat, *lam, lam_features=lam_features,
                         loss=loss)
    assert ps.device_status() == 0
    h = R.spacing(dims, np.float32(bmin), np.float32(bmax))
    vals, ds, ds_hat = R.sdf_terms(s_hat, s, h, *lam)
    gs, gf = ps.unpack_grid(gd, grad, which=ps.GRID_GRAD)
    return vals, ds, ds_hat, gs.cpu().numpy(), d_hat.cpu().numpy(), loss.cpu().numpy(), gf, feat


@pytest.mark.parametrize("dims", [(37, 29, 21), (3, 3, 3), (2, 2, 2), (16, 40, 9)])
@pytest.mark.parametrize("layout", LAYOUTS, ids=lambda v: v[0])
def test_sdf_terms_parity(dims, layout):
    lam = (1.0, 0.1, 0.02)
    vals, ds, ds_hat, gs, gh, loss, gf, _ = _sdf_terms_case(dims, layout, lam, 17)
    errs = {"ds": rel_err_tensor(gs, ds), "ds_hat": rel_err_tensor(gh, ds_hat)}
    for i, k in enumerate(("sdf", "eik", "normal")):
        errs[k] = abs(float(loss[i]) - vals[k]) / max(abs(vals[k]), 1e-30)
    log_errors(f"sdf terms {layout[0]} {dims}", errs)
    assert errs["ds"] <= GRAD_RTOL and errs["ds_hat"] <= GRAD_RTOL, errs
    for k in ("sdf", "eik", "normal"):
        if vals[k] == 0.0:
            assert float(loss[("sdf", "eik", "normal").index(k)]) == 0.0
        else:
            assert errs[k] <= LOSS_RTOL, (k, errs)
    # no interior node: only L_sdf; one interior node: no normal pairs
    if min(dims) == 2:
        assert vals["eik"] == 0.0 and vals["normal"] == 0.0
    if dims == (3, 3, 3):
        assert vals["eik"] > 0.0 and vals["normal"] == 0.0
    # the feature slots of the gradient stay zero
    assert float(gf.abs().max()) == 0.0


@pytest.mark.parametrize("term", ["sdf", "eik", "normal"])
def test_each_sdf_term_alone(term):
    """One weight at a time, so no term hides another's mistake."""
    lam = {"sdf": (1.0, 0.0, 0.0), "eik": (0.0, 1.0, 0.0), "normal": (0.0, 0.0, 1.0)}[term]
    vals, ds, ds_hat, gs, gh, loss, _, _ = _sdf_terms_case((33, 20, 18), LAYOUTS[0], lam, 29)
    assert np.abs(ds).max() > 0
    assert rel_err_tensor(gs, ds) <= GRAD_RTOL
    if term == "sdf":
        assert rel_err_tensor(gh, ds_hat) <= GRAD_RTOL
    else:
        assert float(np.abs(gh).max()) == 0.0


def test_plane_terms_parity():
    dims = (40, 33, 20)
    lam = (0.5, 0.05, 0.01)
    vals, ds, _, gs, _, loss, gf, feat = _sdf_terms_case(dims, LAYOUTS[2], lam, 41,
                                                         lam_features=0.3)
    ref_val, ref_g = R.plane_terms(feat, 0.3)
    err_g = rel_err_tensor(gf.cpu().numpy(), ref_g)
    err_v = abs(float(loss[3]) - ref_val) / ref_val
    log_errors("plane terms", {"grad": float(err_g), "value": float(err_v)})
    assert err_g <= GRAD_RTOL and err_v <= LOSS_RTOL
    assert rel_err_tensor(gs, ds) <= GRAD_RTOL


@pytest.mark.parametrize("pdims,n_a", [((7, 6, 5), 4), ((2, 2, 2), 8), ((33, 17, 9), 4)])
def test_probe_terms_parity(pdims, n_a):
    g = synth.rng(51)
    Px, Py, Pz = pdims
    b = g.normal(size=(Pz, Py, Px, 9, n_a)).astype(np.float32)
    pd = ps.ProbeDesc()
    pd.dims[:] = pdims
    pd.sh_l, pd.n_ang, pd.dtype = 3, n_a, ps.F32
    base = g.normal(size=b.shape).astype(np.float32)
    grad = dev(base)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    ps.probe_smoothness(pd, dev(b), grad, 0.7, loss=loss)
    ref_val, ref_g = R.probe_terms(b, 0.7)
    err_g = rel_err_tensor(grad.cpu().numpy() - base, ref_g)
    err_v = abs(float(loss[0]) - ref_val) / ref_val
    log_errors(f"probe terms {pdims} n_a={n_a}", {"grad": float(err_g), "value": float(err_v)})
    assert err_g <= GRAD_RTOL and err_v <= LOSS_RTOL


def test_regularizer_validation():
    s, s_hat, bmin, bmax = fields((9, 9, 9), 2)
    gd, values, _ = make_grid((9, 9, 9), bmin, bmax, s, ps.F32, ps.FEAT_NODES, 2)
    _, gb = ps.grid_bytes(gd)
    grad = torch.zeros(gb // 4, dtype=torch.float32, device="cuda")
    d_hat = torch.zeros(s.shape, dtype=torch.float32, device="cuda")
    with pytest.raises(ps.LibraryError, match="not compiled in"):
        ps.grid_regularizers(gd, dev(s_hat), values, grad, d_hat, 1, 1, 1, lam_features=0.1)
    with pytest.raises(ps.LibraryError):
        ps.grid_regularizers(gd, dev(s_hat), values, grad, d_hat, -1, 1, 1)
    pd = ps.ProbeDesc()
    pd.dims[:] = (3, 3, 3)
    pd.sh_l, pd.n_ang, pd.dtype = 3, 4, ps.F16
    b = torch.zeros(3, 3, 3, 9, 4, dtype=torch.float32, device="cuda")
    with pytest.raises(ps.LibraryError, match="dtype"):
        ps.probe_smoothness(pd, b, b.clone(), 1.0)
    pd.dtype, pd.n_ang = ps.F32, 3
    b3 = torch.zeros(3, 3, 3, 9, 3, dtype=torch.float32, device="cuda")
    with pytest.raises(ps.LibraryError, match="not compiled in"):
        ps.probe_smoothness(pd, b3, b3.clone(), 1.0)
    assert ps.device_status() == 0


def test_zero_weights_add_nothing_but_report_the_terms():
    """With every weight 0 the gradients are left as they were (bit for bit)
    and the unweighted loss values are still reported."""
    dims = (33, 20, 18)
    s, s_hat, bmin, bmax = fields(dims, 61)
    gd, values, _ = make_grid(dims, bmin, bmax, s, 0, 0, 61)
    _, gbytes = ps.grid_bytes(gd)
    g = synth.rng(62)
    grad = dev(g.normal(size=gbytes // 4))
    d_hat = dev(g.normal(size=s.shape))
    grad0, d_hat0 = grad.clone(), d_hat.clone()
    loss = torch.zeros(4, dtype=torch.float32, device="cuda")
    ps.grid_regularizers(gd, dev(s_hat), values, grad, d_hat, 0.0, 0.0, 0.0, loss=loss)
    assert torch.equal(grad, grad0) and torch.equal(d_hat, d_hat0)
    h = R.spacing(dims, np.float32(bmin), np.float32(bmax))
    vals, _, _ = R.sdf_terms(s_hat, s, h, 0.0, 0.0, 0.0)
    for i, k in enumerate(("sdf", "eik", "normal")):
        assert abs(float(loss[i]) - vals[k]) <= LOSS_RTOL * abs(vals[k])
