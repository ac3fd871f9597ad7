"""Two-pass inference on the GPU against the FP64 oracle: per-view node
shading (FP16 colour records) and the colour-field march."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import RGB_DEPTH_RTOL, box_interval, log_errors, rel_err_elementwise

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2412_10084_gb300 as ps

# A node colour is FP16-rounded FP32: |gpu - ref| <= half an FP16 ulp below 1
# (2^-12) + the FP32 evaluation error (<= 2e-5 at the MLP's scale).
COLOUR_ATOL = 2.0 ** -12 + 2e-5
CAM = (1.9, -0.7, 1.4)


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def scene(kind="f32", width=16, dims=(40, 33, 37), probe_dims=(7, 6, 5), seed=31):
    """(synth scene as the GPU stores it, ps.Scene)."""
    sc = synth.make_scene("sphere64", dims=dims, probe_dims=probe_dims)
    g = synth.rng(seed)
    n_a = 8 if kind == "bf16" else 4
    if width != sc.width or n_a != sc.n_a:
        Pz, Py, Px = sc.probes.shape[:3]
        sc = dataclasses.replace(
            sc, width=width, probes=g.normal(0, 0.3, size=(Pz, Py, Px, 9, n_a)).astype(np.float32),
            mlp=synth.mlp_params(3 + n_a + 3, width, g))
    if kind == "triplane":
        sc = synth.with_triplanes(sc, seed)
    if kind == "bf16":
        # the oracle sees the features as they are stored
        feat = torch.as_tensor(sc.feat).to(torch.bfloat16).to(torch.float32).numpy()
        sc = dataclasses.replace(sc, feat=feat)
        return sc, ps.Scene.from_host(sc, feat_dtype=ps.BF16)
    return sc, ps.Scene.from_host(sc)


def colours_np(c16):
    return c16.float().cpu().numpy()[..., :3]


@pytest.mark.parametrize("kind,width,mode", [("f32", 16, 0), ("f32", 32, 1), ("bf16", 32, 0),
                                             ("triplane", 16, 0), ("triplane", 32, 1)])
def test_shade_parity(kind, width, mode):
    sc, s = scene(kind, width)
    band = 0.08
    params = ps.render_params(64.0, 64, mode, sc.n_fresnel)
    c16 = ps.shade_nodes(s, CAM, band, params)
    assert ps.device_status() == 0
    ref = oracle.shade_nodes(oracle.Model.from_scene(sc), CAM, band, dir_mode=mode)
    got = colours_np(c16)
    inside = np.abs(sc.sdf.astype(np.float64)) < band
    assert inside.sum() > 1000 and (~inside).sum() > 1000
    assert np.all(got[~inside] == 0.0) and np.all(c16.float().cpu().numpy()[..., 3] == 0.0)
    err = float(np.abs(got - ref).max())
    log_errors(f"shade {kind} W={width} mode={mode}", {"abs": err})
    assert err <= COLOUR_ATOL, err


@pytest.mark.parametrize("band", [0.0, float("inf")])
def test_shade_band_extremes(band):
    sc, s = scene(dims=(19, 21, 18), probe_dims=(3, 3, 3))
    params = ps.render_params(64.0, 64, 0, sc.n_fresnel)
    got = colours_np(ps.shade_nodes(s, CAM, band, params))
    if band == 0.0:
        assert np.all(got == 0.0)
    else:
        ref = oracle.shade_nodes(oracle.Model.from_scene(sc), CAM, band)
        assert np.all(got > 0.0) and float(np.abs(got - ref).max()) <= COLOUR_ATOL


def oracle_colour_field(sc, seed):
    """A colour field the oracle writes (shaded from another camera), rounded
    to the FP16 records both sides read."""
    col = oracle.shade_nodes(oracle.Model.from_scene(sc), (-1.2, 1.6, 0.9), 0.15)
    c16 = np.zeros(col.shape[:-1] + (4,), np.float16)
    c16[..., :3] = col.astype(np.float16)
    return c16


@pytest.mark.parametrize("N,explicit", [(64, False), (45, True), (1, False), (33, False)])
def test_colour_field_render_parity(N, explicit):
    sc, s = scene()
    c16 = oracle_colour_field(sc, 3)
    rays = synth.make_rays("sphere64", n_rays=700, seed_offset=60 + N)
    o, d = rays.o, rays.d
    t = None
    if explicit:
        # sorted random distances inside each ray's segment through the box
        g = synth.rng(7)
        tn, tf, hit = box_interval(o, d, sc.box_min, sc.box_max)
        u = np.sort(g.uniform(0.0, 1.0, size=(o.shape[0], N + 1)), axis=1)
        t = (tn[:, None] + 1e-3 + u * np.maximum(tf - tn - 2e-3, 0.0)[:, None]).astype(np.float32)
        t[~hit] = 0.0
        t[:40] = t[:40, ::-1]  # t_N < t_0: treated as misses
    bg = (0.2, 0.4, 0.1)
    params = ps.render_params(64.0, N, 0, sc.n_fresnel, bg=bg)
    rgb, depth, wsum = ps.render_colour_field(s, dev(c16, torch.float16), dev(o), dev(d), params,
                                              t_samples=None if t is None else dev(t))
    ref = oracle.render_colour_field(oracle.Model.from_scene(sc), c16[..., :3].astype(np.float64),
                                     o, d, 64.0, N, bg=bg, t_samples=t)
    errs = {k: rel_err_elementwise(v.cpu().numpy(), ref[k])
            for k, v in (("rgb", rgb), ("depth", depth), ("wsum", wsum))}
    log_errors(f"colour field N={N} explicit={explicit}", errs)
    for k, e in errs.items():
        assert e <= RGB_DEPTH_RTOL, (k, e)


def test_colour_field_render_with_bin_densities_matches_explicit_distances():
    """The march places samples from bin densities exactly as the proposal
    does, so the proposal's densities and its distances give the same bits."""
    sc, s = scene()
    c16 = dev(oracle_colour_field(sc, 4), torch.float16)
    rays = synth.make_rays("sphere64", n_rays=512, seed_offset=91)
    o, d = dev(rays.o), dev(rays.d)
    B, N, res = 16, 48, (16, 16, 16)
    thr = float(np.float32(2.0 * float(sc.box_max[0] - sc.box_min[0]) / (sc.dims[0] - 1)))
    occ = ps.occupancy_build(s, res, thr)
    desc = ps.proposal_desc(res, n_bins=B, mix=0.3, theta=0.0)
    prm = dev(synth.proposal_params(synth.rng(3), n_bins=B))
    t, probs = ps.proposal_forward(s, desc, prm, occ, o, d, N)
    pb = ps.render_params(64.0, N, 0, sc.n_fresnel, n_bins=B)
    pt = ps.render_params(64.0, N, 0, sc.n_fresnel)
    rgb_b, dep_b, w_b = ps.render_colour_field(s, c16, o, d, pb, t_samples=probs)
    rgb_t, dep_t, w_t = ps.render_colour_field(s, c16, o, d, pt, t_samples=t)
    assert torch.equal(rgb_b, rgb_t) and torch.equal(dep_b, dep_t) and torch.equal(w_b, w_t)
    assert float(w_b.max()) > 0.5


def test_two_pass_end_to_end():
    """GPU shading + GPU march against the oracle's two passes: the FP16
    roundings of the two sides may differ by one unit, so rgb may differ by
    up to 2^-11 per unit of weight."""
    sc, s = scene(width=32)
    band = 0.1
    params = ps.render_params(64.0, 96, 0, sc.n_fresnel)
    rays = synth.make_rays("sphere64", n_rays=600, seed_offset=77)
    o, d = rays.o, rays.d
    cam = tuple(float(v) for v in o[0])  # the rays of one camera
    c16 = ps.shade_nodes(s, cam, band, params)
    rgb, _, wsum = ps.render_colour_field(s, c16, dev(o), dev(d), params)
    m = oracle.Model.from_scene(sc)
    col = oracle.shade_nodes(m, cam, band).astype(np.float16).astype(np.float64)
    ref = oracle.render_colour_field(m, col, o, d, 64.0, 96)
    err = float(np.abs(rgb.cpu().numpy() - ref["rgb"]).max())
    log_errors("two-pass end to end", {"rgb_abs": err})
    assert err <= 2.0 ** -11 + 1e-5
    np.testing.assert_allclose(wsum.cpu().numpy(), ref["wsum"], rtol=0, atol=1e-5)


def test_two_pass_equals_fused_render_for_a_constant_colour():
    """Zero MLP weights: every colour is sigmoid(b3); the two passes then give
    the fused per-sample render up to the FP16 rounding of that colour."""
    sc, _ = scene(width=32)
    mlp = np.zeros_like(sc.mlp)
    mlp[-3:] = (0.3, -0.8, 1.6)
    sc = dataclasses.replace(sc, mlp=mlp)
    s = ps.Scene.from_host(sc)
    params = ps.render_params(64.0, 80, 0, sc.n_fresnel)
    rays = synth.make_rays("sphere64", n_rays=500, seed_offset=5)
    o, d = dev(rays.o), dev(rays.d)
    c16 = ps.shade_nodes(s, (2.0, 2.0, 2.0), float("inf"), params)
    c = 1.0 / (1.0 + np.exp(-np.array([0.3, -0.8, 1.6])))
    assert float(np.abs(colours_np(c16) - c).max()) <= 2.0 ** -12 + 1e-6
    rgb2, depth2, wsum2 = ps.render_colour_field(s, c16, o, d, params)
    rgb1, depth1, wsum1, _ = ps.render_forward(s, o, d, params)
    assert float((wsum2 - wsum1).abs().max()) <= 2e-6
    assert float((depth2 - depth1).abs().max()) <= 2e-5
    assert float((rgb2 - rgb1).abs().max()) <= 2.0 ** -12 + 2e-6


def test_full_size_shading_sampled_nodes():
    """256^3 object grid: the band mask is exact and 512 sampled band nodes
    match the oracle."""
    sc = synth.make_scene("object256")
    s = ps.Scene.from_host(sc)
    band = 0.02
    params = ps.render_params(64.0, 256, 0, sc.n_fresnel)
    c16 = ps.shade_nodes(s, (0.5, -1.5, 1.2), band, params)
    got = c16.float().cpu().numpy().reshape(-1, 4)
    inside = (np.abs(sc.sdf.astype(np.float64)) < band).ravel()
    assert np.all(got[~inside] == 0.0) and np.all(got[inside, :3] > 0.0)
    idx = synth.rng(3).choice(np.nonzero(inside)[0], 512, replace=False)
    ref = oracle.shade_node_list(oracle.Model.from_scene(sc), (0.5, -1.5, 1.2), band, idx)
    err = float(np.abs(got[idx, :3] - ref).max())
    log_errors("shade full size sampled", {"abs": err, "band_nodes": int(inside.sum())})
    assert err <= COLOUR_ATOL


def test_two_pass_validation():
    sc, s = scene(dims=(9, 9, 9), probe_dims=(3, 3, 3))
    params = ps.render_params(64.0, 16, 0, sc.n_fresnel)
    with pytest.raises(ps.LibraryError):
        ps.shade_nodes(s, CAM, -1.0, params)
    bad = torch.empty((9, 9, 9, 3), dtype=torch.float16, device="cuda")
    with pytest.raises(ps.LibraryError):
        ps.shade_nodes(s, CAM, 0.1, params, out=bad)
    with pytest.raises(ps.LibraryError):
        ps.render_colour_field(s, bad, dev(np.zeros((4, 3))), dev(np.ones((4, 3))), params)
    c16 = ps.shade_nodes(s, CAM, 0.1, params)
    rgb, _, _ = ps.render_colour_field(s, c16, dev(np.zeros((0, 3))), dev(np.zeros((0, 3))),
                                       params)
    assert rgb.shape == (0, 3)
    assert ps.device_status() == 0
