"""Sparse 16^3-node bricks on the GPU against the FP64 oracle.

A sparse grid stores only the bricks its table names; every other node reads
as SDF = empty_sdf with zero features.  The oracle therefore renders the dense
grid with those values written into the bricks that are not stored, and the
adjoints are compared on the stored nodes (the others have no storage)."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import (GRAD_RTOL, RGB_DEPTH_RTOL, clean_rays, log_errors, oracle_backward,
                     oracle_forward, rel_err_elementwise, rel_err_tensor)

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2412_10084_gb300 as ps

EMPTY = 1.0


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def brick_mask(sdf, thr):
    """Bricks whose nodes come within thr of the surface."""
    Rz, Ry, Rx = sdf.shape
    b = np.abs(sdf).reshape(Rz // 16, 16, Ry // 16, 16, Rx // 16, 16).min(axis=(1, 3, 5))
    return b < thr


def sparse_case(dims=(96, 80, 112), probe_dims=(4, 4, 5), thr=0.1, sh_l=3, seed=41, keep=None):
    """(dense-equivalent synth scene for the oracle, sparse ps.Scene, node mask):
    a sphere of radius 0.22 in the unit box, bricks within thr of its surface
    (or the given brick mask), MLP width 32 (the sparse shapes compiled in)."""
    sc = synth.make_scene("sphere64", dims=dims, probe_dims=probe_dims)
    g = synth.rng(seed)
    sdf = synth.sphere_sdf(dims, sc.box_min, sc.box_max, (0.45, 0.5, 0.55), 0.22)
    sc = dataclasses.replace(sc, sdf=(sdf + g.normal(0, 0.003, size=sdf.shape))
                             .astype(np.float32), width=32, mlp=synth.mlp_params(10, 32, g))
    if sh_l == 4:
        Px, Py, Pz = probe_dims
        sc = dataclasses.replace(sc, sh_l=4, probes=g.normal(0, 0.1, size=(Pz, Py, Px, 16, 4))
                                 .astype(np.float32))
    if keep is None:
        keep = brick_mask(sc.sdf, thr)
    assert keep.any() and (~keep).any()
    s = ps.Scene.from_host(sc, bricks=keep, empty_sdf=EMPTY)
    node_keep = np.repeat(np.repeat(np.repeat(keep, 16, 0), 16, 1), 16, 2)
    sdf = np.where(node_keep, sc.sdf, np.float32(EMPTY)).astype(np.float32)
    feat = np.where(node_keep[..., None], sc.feat, np.float32(0)).astype(np.float32)
    return dataclasses.replace(sc, sdf=sdf, feat=feat), s, node_keep


def test_sparse_pack_unpack_and_bytes():
    sc, s, node_keep = sparse_case()
    gd, _, _ = s.descs(3)
    n_b = int(node_keep.sum()) // 4096
    vb, gb = ps.grid_bytes(gd)
    assert gd.n_bricks == n_b and vb == gb == ps.table_words(gd) * 4 + 16 * 4096 * n_b
    sdf, feat = ps.unpack_grid(gd, s.grid, which=ps.GRID_VALUES)
    assert np.array_equal(sdf.cpu().numpy(), sc.sdf)
    assert np.array_equal(feat.cpu().numpy(), sc.feat)
    gg, _, _ = s.grad_buffers()
    gsdf, gfeat = ps.unpack_grid(gd, gg, which=ps.GRID_GRAD)
    assert float(gsdf.abs().max()) == 0.0 and float(gfeat.abs().max()) == 0.0


@pytest.mark.parametrize("sh_l,N", [(3, 96), (4, 64), (3, 33)])
def test_sparse_forward_parity(sh_l, N):
    sc, s, _ = sparse_case(sh_l=sh_l)
    rays = synth.make_rays("sphere64", n_rays=700, seed_offset=70 + N)
    params = ps.render_params(64.0, N, 0, sc.n_fresnel, (0.1, 0.2, 0.3))
    rgb, depth, wsum, logT = ps.render_forward(s, dev(rays.o), dev(rays.d), params)
    assert ps.device_status() == 0
    ref = oracle_forward(sc, rays.o, rays.d, 64.0, N, bg=(0.1, 0.2, 0.3))
    errs = {k: rel_err_elementwise(v.cpu().numpy(), ref[k])
            for k, v in (("rgb", rgb), ("depth", depth), ("wsum", wsum))}
    log_errors(f"sparse forward l={sh_l} N={N}", errs)
    for k, e in errs.items():
        assert e <= RGB_DEPTH_RTOL, (k, e)
    assert float(wsum.max()) > 0.5


@pytest.mark.parametrize("sh_l", [3, 4])
def test_sparse_backward_parity(sh_l):
    sc, s, node_keep = sparse_case(sh_l=sh_l, seed=43)
    rays = synth.make_rays("sphere64", n_rays=600, seed_offset=80 + sh_l)
    tau, N = 64.0, 64
    keep = clean_rays(sc, rays.o, rays.d, tau, N)
    o, d = rays.o[keep], rays.d[keep]
    n = o.shape[0]
    drgb = (synth.rng(9).normal(size=(n, 3)) / n).astype(np.float32)
    params = ps.render_params(tau, N, 0, sc.n_fresnel)
    o_, d_ = dev(o), dev(d)
    _, _, _, logT, live = ps.render_forward(s, o_, d_, params, want_live=True)
    gg, gp, gm = ps.render_backward(s, o_, d_, params, dev(drgb), logT, n_live=live)
    assert ps.device_status() == 0
    gd, _, _ = s.descs(3)
    gsdf, gfeat = ps.unpack_grid(gd, gg, which=ps.GRID_GRAD)
    ref = oracle_backward(sc, o, d, drgb.astype(np.float64), tau, N)
    ref_sdf = np.where(node_keep, ref["sdf"], 0.0)
    ref_feat = np.where(node_keep[..., None], ref["feat"], 0.0)
    errs = {"sdf": rel_err_tensor(gsdf.cpu().numpy(), ref_sdf),
            "feat": rel_err_tensor(gfeat.cpu().numpy(), ref_feat),
            "probes": rel_err_tensor(gp.cpu().numpy(), ref["probes"]),
            "mlp": rel_err_tensor(gm.cpu().numpy(), ref["mlp"])}
    log_errors(f"sparse backward l={sh_l}", errs)
    assert np.abs(ref_sdf).max() > 0
    for k, e in errs.items():
        assert e <= GRAD_RTOL, (k, e)


def test_empty_space_is_exactly_empty():
    """A ray that meets only bricks that are not stored has s = empty_sdf at
    every sample: zero weight, the background colour, exactly."""
    sc, s, _ = sparse_case()
    o = np.array([[0.03, 0.02, -1.0], [0.97, 0.03, 2.0]], np.float32)  # along two box edges
    d = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, -1.0]], np.float32)
    params = ps.render_params(64.0, 128, 0, sc.n_fresnel, (0.25, 0.5, 0.75))
    rgb, depth, wsum, _ = ps.render_forward(s, dev(o), dev(d), params)
    assert np.array_equal(rgb.cpu().numpy(), np.tile([0.25, 0.5, 0.75], (2, 1)).astype(np.float32))
    assert float(wsum.abs().max()) == 0.0 and float(depth.abs().max()) == 0.0


def test_sparse_weight_histogram_matches_oracle():
    sc, s, _ = sparse_case()
    rays = synth.make_rays("sphere64", n_rays=400, seed_offset=7)
    params = ps.render_params(64.0, 64, 0, sc.n_fresnel)
    h = ps.weight_histogram(s, dev(rays.o), dev(rays.d), params, n_bins=8)
    ref = oracle.weight_histogram(oracle.Model.from_scene(sc), rays.o, rays.d, 64.0, 64, 8)
    assert float(np.abs(h.cpu().numpy() - ref).max()) <= 2e-6


def test_sparse_table_out_of_range_reads_as_empty():
    """A table entry beyond n_bricks stores nothing: the brick reads as empty."""
    sc, s, node_keep = sparse_case()
    gd, _, _ = s.descs(3)
    bad = s.grid.clone()
    tab = bad.view(-1)[:ps.table_words(gd)].view(torch.int32)
    first = int(torch.nonzero(tab >= 0)[0])
    tab[first] = gd.n_bricks + 5
    sdf, _ = ps.unpack_grid(gd, bad, which=ps.GRID_VALUES)
    Bx, By = sc.dims[0] // 16, sc.dims[1] // 16
    bz, by, bx = first // (Bx * By), (first // Bx) % By, first % Bx
    blk = sdf.cpu().numpy()[bz * 16:(bz + 1) * 16, by * 16:(by + 1) * 16, bx * 16:(bx + 1) * 16]
    assert np.all(blk == EMPTY)
    s2 = dataclasses.replace(s, grid=bad)
    rays = synth.make_rays("sphere64", n_rays=64, seed_offset=2)
    rgb, _, _, _ = ps.render_forward(s2, dev(rays.o), dev(rays.d),
                                     ps.render_params(64.0, 32, 0, sc.n_fresnel))
    assert torch.isfinite(rgb).all() and ps.device_status() == 0


def test_sparse_validation():
    sc, s, _ = sparse_case()
    with pytest.raises(ps.LibraryError, match="shape"):
        ps.grid_bytes(ps.grid_desc((40, 32, 64), (0, 0, 0), (1, 1, 1), n_bricks=3))
    with pytest.raises(ps.LibraryError, match="compiled"):
        ps.grid_bytes(ps.grid_desc((48, 32, 64), (0, 0, 0), (1, 1, 1), feat_dtype=ps.BF16,
                                   n_bricks=3))
    with pytest.raises(ps.LibraryError, match="shape"):  # more bricks than the grid has
        ps.grid_bytes(ps.grid_desc((32, 32, 32), (0, 0, 0), (1, 1, 1), n_bricks=9))
    gd, _, _ = s.descs(3)
    hat = torch.zeros(tuple(reversed(sc.dims)), dtype=torch.float32, device="cuda")
    gg, _, _ = s.grad_buffers()
    with pytest.raises(ps.LibraryError, match="stored nodes"):  # s_hat holds the bricks
        ps.grid_regularizers(gd, hat, s.grid, gg, torch.zeros_like(hat), 1.0, 1.0, 1.0)
    hb = torch.zeros((s.n_bricks, 16, 16, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(ps.LibraryError, match="compiled"):  # L_features: tile tri-planes only
        ps.grid_regularizers(gd, hb, s.grid, gg, torch.zeros_like(hb), 1.0, 1.0, 1.0,
                             lam_features=1.0)
    with pytest.raises(ps.LibraryError, match="stored nodes"):  # s_hat holds the bricks
        ps.sdf_smooth(gd, hat, s.grid)


def test_sparse_scene_from_bricks_matches_packing_from_dense_arrays():
    """Assembling the packed buffer brick by brick gives the same bytes as
    packing the dense arrays with the same brick table."""
    keep, bsdf, bfeat, probes, mlp = synth.sparse_object(128, 0.01)
    assert 0 < keep.sum() < keep.size
    s1 = ps.sparse_scene(keep, bsdf, bfeat, probes, mlp, (128, 128, 128), (0, 0, 0), (1, 1, 1),
                         3, 32, empty_sdf=EMPTY)
    sdf = np.full((128, 128, 128), EMPTY, np.float32)
    feat = np.zeros((128, 128, 128, 3), np.float32)
    for k, (bz, by, bx) in enumerate(np.argwhere(keep)):
        sl = (slice(bz * 16, bz * 16 + 16), slice(by * 16, by * 16 + 16),
              slice(bx * 16, bx * 16 + 16))
        sdf[sl] = bsdf[k]
        feat[sl] = bfeat[k]
    sc = synth.Scene(sdf=sdf, feat=feat, probes=probes, mlp=mlp,
                     box_min=np.zeros(3, np.float32), box_max=np.ones(3, np.float32), sh_l=3,
                     width=32, n_fresnel=3)
    s2 = ps.Scene.from_host(sc, bricks=keep, empty_sdf=EMPTY)
    assert s1.n_bricks == s2.n_bricks
    assert torch.equal(s1.grid.view(torch.int32), s2.grid.view(torch.int32))  # bitwise


def test_sparse_colour_field_march_matches_oracle():
    """The colour-field march reads the SDF through the brick table too."""
    sc, s, _ = sparse_case()
    g = synth.rng(19)
    Rx, Ry, Rz = sc.dims
    c16 = np.zeros((Rz, Ry, Rx, 4), np.float16)
    c16[..., :3] = g.uniform(0.0, 1.0, size=(Rz, Ry, Rx, 3)).astype(np.float16)
    rays = synth.make_rays("sphere64", n_rays=600, seed_offset=23)
    params = ps.render_params(64.0, 80, 0, sc.n_fresnel, (0.2, 0.1, 0.4))
    rgb, depth, wsum = ps.render_colour_field(s, torch.as_tensor(c16, device="cuda"),
                                              dev(rays.o), dev(rays.d), params)
    ref = oracle.render_colour_field(oracle.Model.from_scene(sc),
                                     c16[..., :3].astype(np.float64), rays.o, rays.d, 64.0, 80,
                                     bg=(0.2, 0.1, 0.4))
    errs = {k: rel_err_elementwise(v.cpu().numpy(), ref[k])
            for k, v in (("rgb", rgb), ("depth", depth), ("wsum", wsum))}
    log_errors("sparse colour field", errs)
    for k, e in errs.items():
        assert e <= RGB_DEPTH_RTOL, (k, e)


def test_sparse_view_mode_background_and_explicit_distances():
    sc, s, _ = sparse_case(seed=47)
    rays = synth.make_rays("sphere64", n_rays=500, seed_offset=31)
    from helpers import box_interval
    g = synth.rng(13)
    N = 40
    tn, tf, hit = box_interval(rays.o, rays.d, sc.box_min, sc.box_max)
    u = np.sort(g.uniform(0.0, 1.0, size=(rays.o.shape[0], N + 1)), axis=1)
    t = (tn[:, None] + 1e-3 + u * np.maximum(tf - tn - 2e-3, 0.0)[:, None]).astype(np.float32)
    t[~hit] = 0.0
    bg = (0.4, 0.2, 0.6)
    params = ps.render_params(48.0, N, ps.DIR_VIEW, sc.n_fresnel, bg)
    rgb, depth, wsum, _ = ps.render_forward(s, dev(rays.o), dev(rays.d), params, dev(t))
    ref = oracle_forward(sc, rays.o, rays.d, 48.0, N, dir_mode=oracle.DIR_VIEW, bg=bg,
                         t_samples=t)
    for k, v in (("rgb", rgb), ("depth", depth), ("wsum", wsum)):
        assert rel_err_elementwise(v.cpu().numpy(), ref[k]) <= RGB_DEPTH_RTOL, k


# A node colour is FP16-rounded FP32 (as in the dense two-pass tests).
COLOUR_ATOL = 2.0 ** -12 + 2e-5
CAM = (1.9, -0.7, 1.4)


@pytest.mark.parametrize("res,thr", [((8, 8, 8), 0.8), ((7, 5, 9), 2.0 / 95), ((24, 20, 28), 1.0 / 95)])
def test_sparse_occupancy_exact(res, thr):
    """The occupancy build reads the nodes of bricks that are not stored as
    empty_sdf: bit-exact against the oracle on the dense-equivalent grid and
    against the dense kernel on that grid.  thr = 0.8 lies between the
    largest stored |s| and empty_sdf, so exactly the cells that reach a stored
    node are set."""
    sc, s, _ = sparse_case()
    thr = float(np.float32(thr))
    occ = ps.occupancy_unpack(ps.occupancy_build(s, res, thr), res).numpy()
    ref = oracle.occupancy(oracle.Model.from_scene(sc), res, thr)
    assert np.array_equal(occ, ref)
    assert 0 < occ.mean() < 1
    dense = ps.Scene.from_host(sc)
    assert np.array_equal(occ, ps.occupancy_unpack(ps.occupancy_build(dense, res, thr),
                                                   res).numpy())


@pytest.mark.parametrize("mode,band", [(0, 0.08), (1, 0.08), (0, float("inf"))])
def test_sparse_shade_parity(mode, band):
    """Node shading through the brick table: a node of a brick that is not
    stored has s = empty_sdf and zero features (band = inf shades them too);
    the colour field stays one record per node of the full grid."""
    sc, s, node_keep = sparse_case()
    params = ps.render_params(64.0, 64, mode, sc.n_fresnel)
    c16 = ps.shade_nodes(s, CAM, band, params)
    assert ps.device_status() == 0
    assert tuple(c16.shape) == tuple(reversed(sc.dims)) + (4,)
    ref = oracle.shade_nodes(oracle.Model.from_scene(sc), CAM, band, dir_mode=mode)
    got = c16.float().cpu().numpy()[..., :3]
    inside = np.abs(sc.sdf.astype(np.float64)) < band
    assert np.all(got[~inside] == 0.0)
    if np.isinf(band):
        assert (~node_keep).sum() > 0 and np.all(got[~node_keep] > 0.0)
    err = float(np.abs(got - ref).max())
    log_errors(f"sparse shade mode={mode} band={band}", {"abs": err})
    assert err <= COLOUR_ATOL, err


def test_sparse_two_pass_end_to_end():
    sc, s, _ = sparse_case(seed=45)
    band = 0.1
    params = ps.render_params(64.0, 96, 0, sc.n_fresnel)
    rays = synth.make_rays("sphere64", n_rays=600, seed_offset=79)
    o, d = rays.o, rays.d
    cam = tuple(float(v) for v in o[0])
    c16 = ps.shade_nodes(s, cam, band, params)
    rgb, _, wsum = ps.render_colour_field(s, c16, dev(o), dev(d), params)
    m = oracle.Model.from_scene(sc)
    col = oracle.shade_nodes(m, cam, band).astype(np.float16).astype(np.float64)
    ref = oracle.render_colour_field(m, col, o, d, 64.0, 96)
    err = float(np.abs(rgb.cpu().numpy() - ref["rgb"]).max())
    log_errors("sparse two-pass end to end", {"rgb_abs": err})
    assert err <= 2.0 ** -11 + 1e-5
    np.testing.assert_allclose(wsum.cpu().numpy(), ref["wsum"], rtol=0, atol=1e-5)
    assert float(wsum.max()) > 0.5


def test_sparse_proposal_drives_the_render():
    """Occupancy, proposal placement and the render, all on the sparse grid,
    against the oracle's render of the dense-equivalent grid at the placed
    distances."""
    sc, s, _ = sparse_case(seed=49)
    rays = synth.make_rays("sphere64", n_rays=400, seed_offset=93)
    res, n_out = (16, 16, 16), 32
    occ = ps.occupancy_build(s, res, float(np.float32(2.0 / 95)))
    prm = synth.proposal_params(synth.rng(3), n_bins=8).astype(np.float32)
    prm[-8 - 8 * 32:] *= 4.0
    desc = ps.proposal_desc(res, mix=0.1, theta=0.0)
    o_, d_ = dev(rays.o), dev(rays.d)
    t, _ = ps.proposal_forward(s, desc, dev(prm), occ, o_, d_, n_out, want_probs=False)
    hit = (t[:, -1] > t[:, 0]).cpu().numpy()
    assert hit.sum() > 100
    params = ps.render_params(64.0, n_out, n_fresnel=sc.n_fresnel)
    rgb, depth, wsum, _ = ps.render_forward(s, o_[hit], d_[hit], params, t[hit].contiguous())
    ref = oracle_forward(sc, rays.o[hit], rays.d[hit], 64.0, n_out,
                         t_samples=t[hit].cpu().numpy())
    for k, v in (("rgb", rgb), ("depth", depth), ("wsum", wsum)):
        assert rel_err_elementwise(v.cpu().numpy(), ref[k]) <= RGB_DEPTH_RTOL, k


def brick_array(dense, keep):
    """The stored bricks of a dense [Rz,Ry,Rx] array, [n,16,16,16] in slot order."""
    return np.stack([dense[bz * 16:bz * 16 + 16, by * 16:by * 16 + 16, bx * 16:bx * 16 + 16]
                     for bz, by, bx in np.argwhere(keep)])


def random_bricks(dims, seed):
    """About half the bricks, the grid's corner bricks always among them (so
    the replicated edges and absent neighbours both occur)."""
    Bx, By, Bz = (d // 16 for d in dims)
    keep = synth.rng(seed).uniform(size=(Bz, By, Bx)) < 0.5
    keep[0, 0, 0] = keep[-1, -1, -1] = True
    keep[0, -1, 0] = False
    return keep


@pytest.mark.parametrize("dims", [(96, 80, 112), (48, 32, 64)])
def test_sparse_smoothing_matches_the_full_grid(dims):
    """s = G(s_hat) on a sparse grid is the full grid's smoothing, absent bricks
    holding empty_sdf, at the stored nodes; the features are not touched and
    absent nodes still read as empty_sdf."""
    from oracle import regularizers as ORC
    sc, s, node_keep = sparse_case(dims=dims, probe_dims=(3, 3, 3),
                                   keep=random_bricks(dims, sum(dims)))
    keep = node_keep[::16, ::16, ::16]
    gd, _, _ = s.descs(3)
    g = synth.rng(61)
    hat = np.where(node_keep, sc.sdf + g.normal(0, 0.05, size=sc.sdf.shape),
                   EMPTY).astype(np.float32)
    values = s.grid.clone()
    ps.sdf_smooth(gd, dev(brick_array(hat, keep)), values)
    assert ps.device_status() == 0
    sdf, feat = ps.unpack_grid(gd, values, which=ps.GRID_VALUES)
    got = sdf.cpu().numpy()
    ref = ORC.smooth(hat.astype(np.float64))
    err = float(np.abs(got - ref)[node_keep].max())
    log_errors(f"sparse smoothing {dims}", {"abs": err})
    assert err <= 4e-6 * float(np.abs(hat).max())
    assert np.all(got[~node_keep] == EMPTY)
    assert np.array_equal(feat.cpu().numpy(), sc.feat)


@pytest.mark.parametrize("accumulate", [False, True])
def test_sparse_smoothing_adjoint_matches_the_full_grid(accumulate):
    """G^T on a sparse grid: the full grid's transposed smoothing of a gradient
    that is zero on absent bricks, at the stored nodes; the table comes from
    the gradient buffer and the feature slots are not read."""
    from oracle import regularizers as ORC
    dims = (64, 48, 80)
    sc, s, node_keep = sparse_case(dims=dims, probe_dims=(3, 3, 3), keep=random_bricks(dims, 5))
    keep = node_keep[::16, ::16, ::16]
    gd, _, _ = s.descs(3)
    g = synth.rng(67)
    ds = np.where(node_keep, g.normal(0, 1, size=sc.sdf.shape), 0.0).astype(np.float32)
    gg, _, _ = s.grad_buffers()
    rec = gg.view(-1)[ps.table_words(gd):].view(-1, 4)
    rec[:, 0] = dev(brick_array(ds, keep)).reshape(-1)
    rec[:, 1:] = 7.0
    n = int(keep.sum())
    base = g.normal(0, 1, size=(n, 16, 16, 16)).astype(np.float32)
    d_hat = dev(base) if accumulate else torch.full((n, 16, 16, 16), 123.0, device="cuda")
    ps.sdf_smooth_adjoint(gd, gg, d_hat, accumulate=accumulate)
    assert ps.device_status() == 0
    ref = brick_array(ORC.smooth_adjoint(ds.astype(np.float64)), keep)
    if accumulate:
        ref = ref + base
    err = float(np.abs(d_hat.cpu().numpy() - ref).max())
    log_errors(f"sparse smoothing adjoint acc={accumulate}", {"abs": err})
    assert err <= 4e-5 * float(np.abs(ds).max())


@pytest.mark.parametrize("dims", [(96, 80, 112), (48, 32, 64)])
def test_sparse_sdf_regularizers_match_the_full_grid(dims):
    """L_sdf, L_Eik and L_normal on a sparse grid against the oracle's terms
    of the stored nodes on the dense-equivalent grid (every node of an absent
    brick at empty_sdf, in s and s_hat): the three loss values, and the
    gradients w.r.t. s and s_hat at the stored nodes.  Random brick masks that
    keep the grid's corner bricks, so grid faces, absent neighbours across a
    brick face and stored neighbours across one all occur."""
    from oracle import regularizers as ORC
    sc, s, node_keep = sparse_case(dims=dims, probe_dims=(3, 3, 3),
                                   keep=random_bricks(dims, 3 * sum(dims)))
    keep = node_keep[::16, ::16, ::16]
    gd, _, _ = s.descs(3)
    g = synth.rng(71)
    hat = np.where(node_keep, sc.sdf + g.normal(0, 0.05, size=sc.sdf.shape),
                   EMPTY).astype(np.float32)
    # the smoothed SDF both sides read: the oracle's smoothing, rounded to FP32,
    # written into the stored records (absent nodes read empty_sdf)
    s_ref = np.where(node_keep, ORC.smooth(hat.astype(np.float64)), EMPTY).astype(np.float32)
    values = s.grid.clone()
    w = ps.table_words(gd)
    values.view(-1)[w:].view(-1, 4)[:, 0] = dev(brick_array(s_ref, keep)).reshape(-1)
    gg, _, _ = s.grad_buffers()
    gg.zero_()
    n = int(keep.sum())
    base = g.normal(0, 1, size=(n, 16, 16, 16)).astype(np.float32)
    d_hat = dev(base)
    loss = torch.zeros(4, dtype=torch.float32, device="cuda")
    lam = (1.0, 0.1, 0.02)
    ps.grid_regularizers(gd, dev(brick_array(hat, keep)), values, gg, d_hat, *lam, loss=loss)
    assert ps.device_status() == 0
    h = ORC.spacing(dims, sc.box_min, sc.box_max)
    vals, ds, ds_hat = ORC.sdf_terms(hat, s_ref, h, *lam, owner=node_keep)
    got_ds = gg.view(-1)[w:].view(-1, 4)[:, 0].reshape(n, 16, 16, 16).cpu().numpy()
    errs = {"ds": rel_err_tensor(got_ds, brick_array(ds, keep)),
            "ds_hat": rel_err_tensor(d_hat.cpu().numpy() - base, brick_array(ds_hat, keep))}
    lv = loss.cpu().numpy()
    for i, k in enumerate(("sdf", "eik", "normal")):
        errs[k] = abs(float(lv[i]) - vals[k]) / max(abs(vals[k]), 1e-30)
    log_errors(f"sparse sdf terms {dims}", errs)
    assert errs["ds"] <= GRAD_RTOL and errs["ds_hat"] <= GRAD_RTOL, errs
    for k in ("sdf", "eik", "normal"):
        assert vals[k] > 0.0 and errs[k] <= 1e-4, (k, errs)
    # the features' gradient slots stay zero
    assert float(gg.view(-1)[w:].view(-1, 4)[:, 1:].abs().max()) == 0.0
