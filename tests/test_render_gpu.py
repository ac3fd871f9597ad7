"""Parity of the CUDA render and adjoint with the FP64 oracle (GPU only).

Every comparison calls the C ABI through the Python binding on cuda:0 and
the oracle on the same seeded FP32 inputs.
"""
import numpy as np
import pytest
import torch

import copy
import os

import oracle
import synth
from helpers import (GRAD_RTOL, KINK_MARGIN, REL_FLOOR_S32, RGB_DEPTH_RTOL, box_interval,
                     clean_rays, log_errors, oracle_backward, oracle_forward,
                     rel_err_elementwise, rel_err_tensor, worst)

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2412_10084_gb300 as ps


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def gpu_forward(scene, o, d, params, t_samples=None):
    rgb, depth, wsum, logT = ps.render_forward(scene, dev(o), dev(d), params,
                                               None if t_samples is None else dev(t_samples))
    assert ps.device_status() == 0
    return {k: v.cpu().numpy().astype(np.float64)
            for k, v in (("rgb", rgb), ("depth", depth), ("wsum", wsum), ("logT", logT))}


def gpu_backward(scene, o, d, params, drgb, ddepth=None, dwsum=None, t_samples=None,
                 use_live=True):
    o_, d_ = dev(o), dev(d)
    ts = None if t_samples is None else dev(t_samples)
    _, _, _, logT, live = ps.render_forward(scene, o_, d_, params, ts, want_live=True)
    gg, gp, gm = ps.render_backward(scene, o_, d_, params, dev(drgb), logT,
                                    d_depth=None if ddepth is None else dev(ddepth),
                                    d_wsum=None if dwsum is None else dev(dwsum), t_samples=ts,
                                    n_live=live if use_live else None)
    gd, _, _ = scene.descs(params.n_fresnel)
    gsdf, gfeat = ps.unpack_grid(gd, gg)
    assert ps.device_status() == 0
    return {"sdf": gsdf.cpu().numpy(), "feat": gfeat.cpu().numpy(),
            "probes": gp.cpu().numpy(), "mlp": gm.cpu().numpy()}


def check_forward(sc, o, d, tau, N, dir_mode=0, bg=(0, 0, 0), t_samples=None):
    scene = ps.Scene.from_host(sc)
    params = ps.render_params(tau, N, dir_mode, sc.n_fresnel, bg)
    g = gpu_forward(scene, o, d, params, t_samples)
    r = oracle_forward(sc, o, d, tau, N, dir_mode=dir_mode, bg=bg, t_samples=t_samples)
    errs = {k: rel_err_elementwise(g[k], r[k]) for k in ("rgb", "depth", "wsum")}
    errs["logT"] = float(np.max(np.abs(g["logT"] - r["logT"]) /
                                np.maximum(np.abs(r["logT"]), 1.0)))
    detail = {k: worst(g[k], r[k]) for k in ("rgb", "depth", "wsum")}
    # against the oracle with FP32-rounded SDF values, at the 1e-3 floor
    r32 = oracle_forward(sc, o, d, tau, N, dir_mode=dir_mode, bg=bg, t_samples=t_samples,
                         sdf_fp32=True)
    for k in ("rgb", "depth", "wsum"):
        errs[k + "_s32"] = rel_err_elementwise(g[k], r32[k], floor=REL_FLOOR_S32)
        detail[k + "_s32"] = worst(g[k], r32[k], floor=REL_FLOOR_S32)
    log_errors(os.environ.get("PYTEST_CURRENT_TEST", "?") + " forward", errs)
    for k, e in errs.items():
        assert e <= RGB_DEPTH_RTOL, (k, e, detail)
    return g, r


def check_backward(sc, o, d, tau, N, dir_mode=0, bg=(0, 0, 0), seed=5, with_depth=False,
                   t_samples=None, min_kept=0.5):
    keep = clean_rays(sc, o, d, tau, N, dir_mode=dir_mode, bg=bg, t_samples=t_samples)
    assert keep.size >= min_kept * o.shape[0], (keep.size, o.shape[0])
    o, d = o[keep], d[keep]
    if t_samples is not None:
        t_samples = t_samples[keep]
    g = synth.rng(seed)
    n = o.shape[0]
    drgb = (g.normal(size=(n, 3)) / n).astype(np.float32)
    ddepth = (g.normal(size=n) / n).astype(np.float32) if with_depth else None
    dwsum = (g.normal(size=n) / n).astype(np.float32) if with_depth else None
    scene = ps.Scene.from_host(sc)
    params = ps.render_params(tau, N, dir_mode, sc.n_fresnel, bg)
    gg = gpu_backward(scene, o, d, params, drgb, ddepth, dwsum, t_samples)
    gr = oracle_backward(sc, o, d, drgb.astype(np.float64), tau, N, dir_mode=dir_mode, bg=bg,
                         d_depth=ddepth, d_wsum=dwsum, t_samples=t_samples)
    errs = {k: rel_err_tensor(gg[k], gr[k]) for k in ("sdf", "feat", "probes", "mlp")}
    errs["rays_kept"] = int(keep.size)
    log_errors(os.environ.get("PYTEST_CURRENT_TEST", "?") + " backward", errs)
    errs.pop("rays_kept")
    for k, e in errs.items():
        assert e <= GRAD_RTOL, (k, e, errs)
    return errs


# ---------------------------------------------------------------------------
# The small configuration: 64^3 sphere + noise, 4096 rays x 128 samples
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def sphere64():
    sc = synth.make_scene("sphere64")
    rays = synth.make_rays("sphere64")
    return sc, rays


def test_forward_parity_sphere64(sphere64):
    sc, rays = sphere64
    g, r = check_forward(sc, rays.o, rays.d, 64.0, 128)
    assert np.sum(r["wsum"] > 0.5) > 200  # the batch does hit the surface


def test_backward_parity_sphere64(sphere64):
    sc, rays = sphere64
    check_backward(sc, rays.o, rays.d, 64.0, 128)


def test_backward_parity_with_depth_and_wsum_cotangents(sphere64):
    sc, rays = sphere64
    check_backward(sc, rays.o[:1500], rays.d[:1500], 64.0, 128, bg=(0.2, 0.5, 0.9),
                   with_depth=True)


# ---------------------------------------------------------------------------
# Ragged shapes, modes and edge cases
# ---------------------------------------------------------------------------

def test_ragged_samples_and_rays_view_mode():
    sc = synth.make_scene("sphere64", dims=(40, 33, 37), probe_dims=(7, 6, 5))
    rays = synth.make_rays("sphere64", n_rays=777, seed_offset=3)
    check_forward(sc, rays.o, rays.d, 48.0, 100, dir_mode=1, bg=(0.3, 0.1, 0.7))
    check_backward(sc, rays.o, rays.d, 48.0, 100, dir_mode=1, bg=(0.3, 0.1, 0.7),
                   with_depth=True)


@pytest.mark.parametrize("N", [1, 31, 32, 33, 64])
def test_sample_counts_around_chunk_boundaries(N):
    sc = synth.make_scene("sphere64", dims=(24, 24, 24), probe_dims=(6, 6, 6))
    rays = synth.make_rays("sphere64", n_rays=300, seed_offset=N)
    check_forward(sc, rays.o, rays.d, 32.0, N)
    check_backward(sc, rays.o, rays.d, 32.0, N, with_depth=True)


def test_width32_and_eight_channels():
    spec = dict(synth.WORKLOADS["stress512"])
    g = synth.rng(77)
    sc = synth.make_scene("sphere64", dims=(30, 30, 30), probe_dims=(5, 5, 5))
    sc.probes = g.normal(0, 0.1, size=(5, 5, 5, 9, 8)).astype(np.float32)
    sc.width = 32
    sc.mlp = synth.mlp_params(3 + 8 + 3, 32, g)
    rays = synth.make_rays("sphere64", n_rays=600, seed_offset=9)
    check_forward(sc, rays.o, rays.d, 64.0, 96)
    check_backward(sc, rays.o, rays.d, 64.0, 96)
    assert spec["n_a"] == 8


@pytest.mark.parametrize("triplane", [False, True])
def test_sh_order_four(triplane):
    """l = 4 (16 SH coefficients per probe, Sec. 4), width 32, node features or
    tile tri-planes: forward and adjoint against the oracle."""
    g = synth.rng(78)
    sc = synth.make_scene("sphere64", dims=(34, 30, 33), probe_dims=(5, 4, 6))
    sc.probes = g.normal(0, 0.1, size=(6, 4, 5, 16, 4)).astype(np.float32)
    sc.sh_l = 4
    sc.width = 32
    sc.mlp = synth.mlp_params(3 + 4 + 3, 32, g)
    if triplane:
        sc = synth.with_triplanes(sc, 79)
    rays = synth.make_rays("sphere64", n_rays=500, seed_offset=19)
    check_forward(sc, rays.o, rays.d, 64.0, 80)
    check_backward(sc, rays.o, rays.d, 64.0, 80)


def test_explicit_sample_distances():
    sc = synth.make_scene("sphere64", dims=(32, 32, 32), probe_dims=(8, 8, 8))
    rays = synth.make_rays("sphere64", n_rays=256, seed_offset=11)
    g = synth.rng(12)
    N = 48
    # sorted random distances inside each ray's segment through the box
    tn, tf, hit = box_interval(rays.o, rays.d, sc.box_min, sc.box_max)
    u = np.sort(g.uniform(0.0, 1.0, size=(256, N + 1)), axis=1)
    t = (tn[:, None] + 1e-3 + u * np.maximum(tf - tn - 2e-3, 0.0)[:, None]).astype(np.float32)
    t[~hit] = 0.0
    t[:5] = 0.0  # treated as misses
    check_forward(sc, rays.o, rays.d, 64.0, N, t_samples=t)
    check_backward(sc, rays.o, rays.d, 64.0, N, t_samples=t)


@pytest.mark.parametrize("case", ["uniform", "explicit", "view_bg", "bf16", "triplane", "l4",
                                  "n33"])
def test_live_extent_in_every_layout_and_placement(case):
    """Asking the forward for the live extents changes no output bit, in each
    grid layout and sample placement, and the extents equal the oracle's
    (1 + the last sample with a nonzero weight) on rays away from the kinks."""
    sc = synth.make_scene("sphere64", dims=(40, 36, 44), probe_dims=(6, 5, 7))
    rays = synth.make_rays("sphere64", n_rays=900, seed_offset=41)
    N, mode, bg, ts = 96, 0, (0.0, 0.0, 0.0), None
    kw = {}
    if case == "explicit":
        tn, tf, hit = box_interval(rays.o, rays.d, sc.box_min, sc.box_max)
        u = np.sort(synth.rng(42).uniform(0.0, 1.0, size=(900, N + 1)), axis=1)
        ts = dev((tn[:, None] + 1e-3 + u * np.maximum(tf - tn - 2e-3, 0.0)[:, None])
                 .astype(np.float32) * hit[:, None])
    elif case == "view_bg":
        mode, bg = 1, (0.3, 0.6, 0.9)
    elif case == "bf16":  # BF16 features with FP32 probes: 8 channels, width 32 compiled in
        g = synth.rng(45)
        sc.width = 32
        sc.probes = g.normal(0, 0.1, size=(7, 5, 6, 9, 8)).astype(np.float32)
        sc.mlp = synth.mlp_params(3 + 8 + 3, 32, g)
        kw = dict(feat_dtype=ps.BF16)
    elif case == "triplane":
        sc = synth.with_triplanes(sc, 43)
    elif case == "l4":
        g = synth.rng(44)
        sc.sh_l, sc.width = 4, 32
        sc.probes = g.normal(0, 0.1, size=(7, 5, 6, 16, 4)).astype(np.float32)
        sc.mlp = synth.mlp_params(10, 32, g)
    elif case == "n33":
        N = 33
    scene = ps.Scene.from_host(sc, **kw)
    params = ps.render_params(64.0, N, mode, 3, bg)
    o, d = dev(rays.o), dev(rays.d)
    a = ps.render_forward(scene, o, d, params, ts)
    b = ps.render_forward(scene, o, d, params, ts, want_live=True)
    assert ps.device_status() == 0
    for x, y in zip(a, b[:4]):
        assert torch.equal(x, y)
    r = oracle_forward(sc if case != "bf16" else stored_values(sc, feat_bf16=True),
                       rays.o, rays.d, 64.0, N, dir_mode=mode, bg=bg,
                       t_samples=None if ts is None else ts.cpu().numpy(), margin=True)
    keep = r["margin"] > KINK_MARGIN
    m = oracle.Model.from_scene(sc)
    live = b[4].cpu().numpy()
    for i in np.nonzero(keep)[0][:40]:
        tr = oracle.render_trace(m, rays.o[i], rays.d[i], 64.0, N, dir_mode=mode,
                                 t_samples=None if ts is None else ts[i].cpu().numpy())
        ref = int(np.nonzero(tr["w"] > 0)[0].max() + 1) if tr["hit"] and np.any(tr["w"] > 0) \
            else 0
        assert live[i] == ref, (i, live[i], ref)


def test_empty_batch_and_misses():
    sc = synth.make_scene("sphere64", dims=(16, 16, 16), probe_dims=(4, 4, 4))
    scene = ps.Scene.from_host(sc)
    params = ps.render_params(64.0, 32, 0, 3, (0.25, 0.5, 0.75))
    e = torch.empty((0, 3), dtype=torch.float32, device="cuda")
    rgb, depth, wsum, logT = ps.render_forward(scene, e, e, params)
    assert rgb.shape == (0, 3)
    gg, gp, gm = ps.render_backward(scene, e, e, params, e, logT)
    assert float(gg.abs().sum()) == 0.0
    o = np.array([[2.0, 2.0, 2.0], [-1.0, 0.5, 0.5], [0.5, 0.5, 3.0]], np.float32)
    d = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]], np.float32)
    out = gpu_forward(scene, o, d, params)
    np.testing.assert_array_equal(out["rgb"], np.tile([0.25, 0.5, 0.75], (3, 1)))
    assert np.all(out["wsum"] == 0) and np.all(out["depth"] == 0)


def test_per_ray_results_do_not_depend_on_the_batch(sphere64):
    """A CTA's warps take its rays from a counter, so which warp renders a ray
    depends on timing: every ray's outputs must still be the same bits in a
    batch of any size (1, 3, 6, 37 rays: fewer rays than warps, CTAs with some
    warps idle) as in the full batch, and the adjoint of a small batch must
    match the oracle."""
    sc, rays = sphere64
    scene = ps.Scene.from_host(sc)
    params = ps.render_params(64.0, 128, 0, 3)
    full = ps.render_forward(scene, dev(rays.o), dev(rays.d), params, want_live=True)
    assert ps.device_status() == 0
    idx = np.nonzero(full[2].cpu().numpy() > 0.5)[0]  # rays that reach the surface first
    for n in (1, 3, 6, 37):
        part = ps.render_forward(scene, dev(rays.o[idx[:n]]), dev(rays.d[idx[:n]]), params,
                                 want_live=True)
        assert ps.device_status() == 0
        for x, y in zip(part, full):
            assert torch.equal(x, y[torch.as_tensor(idx[:n], device="cuda")]), n
    check_backward(sc, rays.o[idx[:37]], rays.d[idx[:37]], 64.0, 128, min_kept=0.3)


def test_host_validation_errors():
    sc = synth.make_scene("sphere64", dims=(16, 16, 16), probe_dims=(4, 4, 4))
    scene = ps.Scene.from_host(sc)
    o = dev(np.zeros((4, 3)))
    with pytest.raises(ps.LibraryError, match="shape"):
        ps.render_forward(scene, o, o, ps.render_params(64.0, 0))
    with pytest.raises(ps.LibraryError, match="shape"):
        ps.render_forward(scene, o, o, ps.render_params(-1.0, 8))
    with pytest.raises(ps.LibraryError):
        ps.render_forward(scene, o, o, ps.render_params(64.0, 8, n_fresnel=2))
    with pytest.raises(ps.LibraryError, match="CPU"):
        ps.render_forward(scene, o.cpu(), o.cpu(), ps.render_params(64.0, 8))


def test_launch_occupancy():
    """The launcher fills every SM to the kernels' resident-CTA limit."""
    sc = synth.make_scene("sphere64", dims=(16, 16, 16), probe_dims=(4, 4, 4))
    scene = ps.Scene.from_host(sc)
    f, b = ps.render_occupancy(scene, ps.render_params(64.0, 32, 0, 3))
    assert f >= 2 and b >= 2, (f, b)


# ---------------------------------------------------------------------------
# Reduced-precision storage and arithmetic
# ---------------------------------------------------------------------------

RP_RGB_ABS = 2e-3      # reduced precision: |rgb - ref| <= 2e-3 (absolute)
RP_GRAD_RTOL = 2e-2    # reduced precision: per tensor max|g - g_ref| <= 2e-2 max|g_ref|
# Against the oracle whose MLP layer inputs are rounded to FP16 as the tensor
# cores read them (both sides then take the same ReLU decisions), what is left
# is the FP16 storage of the adjoint's dz rows (unit roundoff 2^-11 ~ 4.9e-4,
# two roundings on the path to dx) and FP32 accumulation: gradients within
# 2e-3 of each tensor's largest magnitude, colours within 1e-5 absolute.
RP16_GRAD_RTOL = 2e-3
RP16_RGB_ABS = 1e-5


def stored_values(sc, feat_bf16=False, probe_f16=False, mlp_f16=False):
    """The scene with features / probes rounded to their storage precision:
    the values the kernels read, given to the oracle.  mlp_f16: W1 and W2 (the
    tensor-core operands of the reduced-precision MLP) rounded to FP16; the
    biases and the output layer stay FP32."""
    out = copy.copy(sc)
    if feat_bf16:
        out.feat = torch.as_tensor(sc.feat).bfloat16().float().numpy()
    if probe_f16:
        out.probes = sc.probes.astype(np.float16).astype(np.float32)
    if mlp_f16:
        W = sc.width
        mlp = np.asarray(sc.mlp, np.float32).copy()
        nin = (mlp.size - W * W - 5 * W - 3) // W
        o2 = W * nin + W
        for lo, hi in ((0, W * nin), (o2, o2 + W * W)):
            mlp[lo:hi] = mlp[lo:hi].astype(np.float16).astype(np.float32)
        out.mlp = mlp
    return out


def l2_rel(gpu, ref):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    nr = float(np.linalg.norm(ref))
    return float(np.linalg.norm(gpu - ref)) / nr if nr > 0 else float(np.linalg.norm(gpu))


def psnr(a, b):
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return float("inf") if mse == 0 else 10.0 * np.log10(1.0 / mse)


def test_reduced_precision_human_shape():
    """BF16 features, FP16 probes, FP16 MLP on the tensor cores (FP32 accumulation)
    on a human-capture shaped scene, against the FP64 oracle of the stored values."""
    sc = synth.make_scene("human384", dims=(48, 96, 48), probe_dims=(6, 12, 6))
    rays = synth.make_rays("human384", n_rays=1024)
    ref_sc = stored_values(sc, feat_bf16=True, probe_f16=True)
    scene = ps.Scene.from_host(sc, feat_dtype=ps.BF16, probe_dtype=ps.F16, mlp_dtype=ps.F16)
    params = ps.render_params(64.0, 128, 0, 3)
    g = gpu_forward(scene, rays.o, rays.d, params)
    r = oracle_forward(ref_sc, rays.o, rays.d, 64.0, 128)
    err = float(np.max(np.abs(g["rgb"] - r["rgb"])))
    assert np.sum(r["wsum"] > 0.5) > 50
    assert err <= RP_RGB_ABS, err
    log_errors("reduced precision forward", {"rgb_max_abs": err, "psnr_vs_oracle": psnr(g["rgb"], r["rgb"]),
                                             "depth_rel": rel_err_elementwise(g["depth"], r["depth"])})
    keep = clean_rays(ref_sc, rays.o, rays.d, 64.0, 128)[:600]
    o, d = rays.o[keep], rays.d[keep]
    n = o.shape[0]
    drgb = (synth.rng(5).normal(size=(n, 3)) / n).astype(np.float32)
    gg = gpu_backward(scene, o, d, params, drgb)
    gr = oracle_backward(ref_sc, o, d, drgb.astype(np.float64), 64.0, 128)
    errs = {k: rel_err_tensor(gg[k], gr[k]) for k in ("sdf", "feat", "probes", "mlp")}
    log_errors("reduced precision backward", errs)
    for k, e in errs.items():
        assert e <= RP_GRAD_RTOL, (k, e, errs)


def test_bf16_features_with_fp32_mlp():
    """BF16 feature storage with FP32 probes and the FP32-equivalent MLP (the
    adjoint-stress configuration) meets the FP32 tolerances on the stored values."""
    g = synth.rng(78)
    sc = synth.make_scene("sphere64", dims=(30, 30, 30), probe_dims=(5, 5, 5))
    sc.probes = g.normal(0, 0.1, size=(5, 5, 5, 9, 8)).astype(np.float32)
    sc.width = 32
    sc.mlp = synth.mlp_params(3 + 8 + 3, 32, g)
    rays = synth.make_rays("sphere64", n_rays=600, seed_offset=19)
    ref_sc = stored_values(sc, feat_bf16=True)
    scene = ps.Scene.from_host(sc, feat_dtype=ps.BF16)
    params = ps.render_params(64.0, 96, 0, 3)
    gf = gpu_forward(scene, rays.o, rays.d, params)
    rf = oracle_forward(ref_sc, rays.o, rays.d, 64.0, 96)
    for k in ("rgb", "depth", "wsum"):
        assert rel_err_elementwise(gf[k], rf[k]) <= RGB_DEPTH_RTOL, k
    keep = clean_rays(ref_sc, rays.o, rays.d, 64.0, 96)
    o, d = rays.o[keep], rays.d[keep]
    n = o.shape[0]
    drgb = (synth.rng(6).normal(size=(n, 3)) / n).astype(np.float32)
    gg = gpu_backward(scene, o, d, params, drgb)
    gr = oracle_backward(ref_sc, o, d, drgb.astype(np.float64), 64.0, 96)
    for k in ("sdf", "feat", "probes", "mlp"):
        assert rel_err_tensor(gg[k], gr[k]) <= GRAD_RTOL, k


def test_bf16_pack_roundtrip():
    sc = synth.make_scene("sphere64", dims=(19, 17, 23), probe_dims=(4, 4, 4))
    scene = ps.Scene.from_host(sc, feat_dtype=ps.BF16)
    gd, _, _ = scene.descs(3)
    sdf, feat = ps.unpack_grid(gd, scene.grid)
    np.testing.assert_array_equal(sdf.cpu().numpy(), sc.sdf)
    np.testing.assert_array_equal(feat.cpu().numpy(),
                                  torch.as_tensor(sc.feat).bfloat16().float().numpy())


def test_pack_unpack_roundtrip_exact():
    sc = synth.make_scene("sphere64", dims=(19, 17, 23), probe_dims=(4, 4, 4))
    scene = ps.Scene.from_host(sc)
    gd, _, _ = scene.descs(3)
    sdf, feat = ps.unpack_grid(gd, scene.grid)
    np.testing.assert_array_equal(sdf.cpu().numpy(), sc.sdf)
    np.testing.assert_array_equal(feat.cpu().numpy(), sc.feat)


# ---------------------------------------------------------------------------
# Invariants and determinism at the full object-capture size
# (256^3 grid, 32^3 probes, W = 32, 2^18 rays x 256 samples: the benchmark's launch)
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def object256():
    sc = synth.make_scene("object256")
    rays = synth.make_rays("object256")
    return sc, rays


def test_full_size_forward_sampled_parity_and_invariants(object256):
    sc, rays = object256
    scene = ps.Scene.from_host(sc)
    params = ps.render_params(64.0, 256, 0, 3)
    o, d = dev(rays.o), dev(rays.d)
    rgb, depth, wsum, logT = ps.render_forward(scene, o, d, params)
    rgb2, depth2, wsum2, logT2 = ps.render_forward(scene, o, d, params)
    torch.cuda.synchronize()
    assert torch.equal(rgb, rgb2) and torch.equal(depth, depth2) and torch.equal(wsum, wsum2)
    # asking for the live extents changes no output bit
    rgb3, depth3, wsum3, logT3, live = ps.render_forward(scene, o, d, params, want_live=True)
    assert torch.equal(rgb, rgb3) and torch.equal(depth, depth3) and torch.equal(wsum, wsum3)
    assert torch.equal(logT, logT3)
    assert 0 < float(live.float().mean()) < 256
    for t in (rgb, depth, wsum, logT):
        assert torch.isfinite(t).all()
    assert float(wsum.min()) >= 0.0 and float(wsum.max()) <= 1.0 + 1e-6
    assert float(rgb.min()) >= 0.0 and float(rgb.max()) <= 1.0 + 1e-6
    idx = synth.rng(3).choice(rays.o.shape[0], 256, replace=False)
    r = oracle_forward(sc, rays.o[idx], rays.d[idx], 64.0, 256)
    r32 = oracle_forward(sc, rays.o[idx], rays.d[idx], 64.0, 256, sdf_fp32=True)
    for k, v in (("rgb", rgb), ("depth", depth), ("wsum", wsum)):
        e = rel_err_elementwise(v.cpu().numpy()[idx], r[k])
        assert e <= RGB_DEPTH_RTOL, (k, e)
        e32 = rel_err_elementwise(v.cpu().numpy()[idx], r32[k], floor=REL_FLOOR_S32)
        assert e32 <= RGB_DEPTH_RTOL, (k + " (FP32-rounded s, 1e-3 floor)", e32)


def test_full_size_backward_subset_parity(object256):
    sc, rays = object256
    idx = synth.rng(4).choice(rays.o.shape[0], 384, replace=False)
    check_backward(sc, rays.o[idx], rays.d[idx], 64.0, 256, min_kept=0.3)


def test_full_batch_adjoint_parity_at_the_bench_launch(object256):
    """The adjoint of the benchmark's whole launch (2^18 rays x 256 samples,
    its kernel configuration and live extents) against the FP64 oracle's over
    the same rays: all four gradient tensors at the FP32 bar, with every
    CTA-level probe / MLP reduction and the contention of the grid reductions
    of the timed launch.  The cotangent is the L1 loss gradient of the
    oracle's colours against the targets, zeroed on the rays that pass within
    the kink margin of a ReLU or alpha-clip decision (the launch keeps its
    shape; those rays add exactly nothing on either side)."""
    sc, rays = object256
    n = rays.o.shape[0]
    tau, N = 64.0, 256
    r = oracle_forward(sc, rays.o, rays.d, tau, N, margin=True)
    keep = r["margin"] > KINK_MARGIN
    assert keep.mean() > 0.5, keep.mean()
    drgb = (np.sign(r["rgb"] - rays.target) / (3.0 * n) * keep[:, None]).astype(np.float32)
    scene = ps.Scene.from_host(sc)
    params = ps.render_params(tau, N, 0, 3)
    gg = gpu_backward(scene, rays.o, rays.d, params, drgb)
    gr = oracle_backward(sc, rays.o, rays.d, drgb.astype(np.float64), tau, N)
    errs = {k: rel_err_tensor(gg[k], gr[k]) for k in ("sdf", "feat", "probes", "mlp")}
    errs["rays_kept"] = int(keep.sum())
    log_errors("full-batch adjoint object256", errs)
    errs.pop("rays_kept")
    for k, e in errs.items():
        assert e <= GRAD_RTOL, (k, e, errs)


def test_full_size_backward_runs_and_is_finite(object256):
    sc, rays = object256
    scene = ps.Scene.from_host(sc)
    params = ps.render_params(64.0, 256, 0, 3)
    o, d = dev(rays.o), dev(rays.d)
    target = dev(rays.target)
    scene.grid.requires_grad_(True)
    scene.probes.requires_grad_(True)
    scene.mlp.requires_grad_(True)
    rgb, depth, wsum = ps.render(scene, o, d, params)
    loss = (rgb - target).abs().mean()
    loss.backward()
    torch.cuda.synchronize()
    for p in (scene.grid, scene.probes, scene.mlp):
        assert p.grad is not None and torch.isfinite(p.grad).all()
        assert float(p.grad.abs().max()) > 0.0


# ---------------------------------------------------------------------------
# Autograd wrapper and FP32 finite differences on the GPU itself
# ---------------------------------------------------------------------------

def test_autograd_function_matches_direct_backward(sphere64):
    sc, rays = sphere64
    scene = ps.Scene.from_host(sc)
    params = ps.render_params(64.0, 128, 0, 3)
    o, d = dev(rays.o), dev(rays.d)
    drgb = dev(synth.rng(8).normal(size=(rays.o.shape[0], 3)) / 4096)
    grid = scene.grid.clone().requires_grad_(True)
    probes = scene.probes.clone().requires_grad_(True)
    mlp = scene.mlp.clone().requires_grad_(True)
    rgb, _, _ = ps.RenderFunction.apply(grid, probes, mlp, o, d, None, scene, params)
    (rgb * drgb).sum().backward()
    _, _, _, logT = ps.render_forward(scene, o, d, params)
    gg, gp, gm = ps.render_backward(scene, o, d, params, drgb, logT)
    for a, b in ((grid.grad, gg), (probes.grad, gp), (mlp.grad, gm)):
        scale = float(b.abs().max())
        assert float((a - b).abs().max()) <= 1e-5 * scale


def test_gpu_central_differences():
    """FP32 gradients against central differences of the FP32 forward on the GPU,
    h = 1e-3 on 64 random parameters with significant gradients: spatial
    features, probe coefficients and MLP weights (an SDF value moved by 1e-3
    shifts the alpha-clip kinks of Eq. 9 under nearby samples, so SDF values
    are checked against the FP64 oracle's finite differences instead).  FP32
    forward noise divided by 2h limits each difference to a few percent, so
    every parameter is held to 10% and the 64 together to 2.5% in the L2 sense;
    the strict check is the FP64-oracle comparison above."""
    sc = synth.make_scene("sphere64", dims=(20, 20, 20), probe_dims=(5, 5, 5))
    rays = synth.make_rays("sphere64", n_rays=512, seed_offset=21)
    keep = clean_rays(sc, rays.o, rays.d, 16.0, 48, margin=3e-4)
    o, d = dev(rays.o[keep]), dev(rays.d[keep])
    n = o.shape[0]
    scene = ps.Scene.from_host(sc)
    params = ps.render_params(16.0, 48, 0, 3)
    wts = dev(synth.rng(22).normal(size=(n, 3)))

    def loss():
        rgb, _, _, _ = ps.render_forward(scene, o, d, params)
        return float((rgb.double() * wts.double()).sum())

    _, _, _, logT = ps.render_forward(scene, o, d, params)
    gg, gp, gm = ps.render_backward(scene, o, d, params, wts, logT)
    g = synth.rng(23)
    h = 1e-3
    fds, ans = [], []
    for tensor, grad, count in ((scene.grid, gg, 22), (scene.probes, gp, 21),
                                (scene.mlp, gm, 21)):
        flat, gflat = tensor.view(-1), grad.view(-1)
        eligible = torch.ones_like(gflat, dtype=torch.bool)
        if tensor is scene.grid:  # feature components only: {sdf, f0, f1, f2} records
            eligible = (torch.arange(gflat.numel(), device=gflat.device) % 4) != 0
        mag = torch.where(eligible, gflat.abs(), torch.zeros_like(gflat))
        nz = torch.nonzero(mag > 0.1 * mag.max()).view(-1).cpu().numpy()
        for i in g.choice(nz, min(count, nz.size), replace=False):
            old = float(flat[i])
            flat[i] = old + h
            lp = loss()
            flat[i] = old - h
            lm = loss()
            flat[i] = old
            fd, an = (lp - lm) / (2 * h), float(gflat[i])
            assert abs(fd - an) <= 1e-1 * abs(an), (i, fd, an)
            fds.append(fd)
            ans.append(an)
    fds, ans = np.array(fds), np.array(ans)
    assert fds.size == 64
    assert np.linalg.norm(fds - ans) <= 2.5e-2 * np.linalg.norm(ans)


def test_tensor_core_waits_that_run_out_are_reported_and_the_gpu_stays_usable(sphere64):
    """With the wait limit at 0 polls every tensor-core completion wait runs out
    at once (no tensor core can answer that fast): the forward, the adjoint
    and node shading stop early, set bit 0 of the device status word, free
    their tensor memory and return, without a trap or a hang.  With the
    default limit restored, the next launches (which allocate tensor memory
    again) match the oracle."""
    sc, rays = sphere64
    o, d = rays.o[:512], rays.d[:512]
    tau, N = 64.0, 128
    scene = ps.Scene.from_host(sc)
    params = ps.render_params(tau, N, 0, 3)
    o_, d_ = dev(o), dev(d)
    _, _, _, logT, live = ps.render_forward(scene, o_, d_, params, want_live=True)
    assert ps.device_status() == 0
    drgb = dev(synth.rng(31).normal(size=(512, 3)) / 512)
    ps.set_wait_polls(0)
    try:
        assert ps.wait_polls() == 0
        ps.render_forward(scene, o_, d_, params)
        assert ps.device_status() & 1
        gg, gp, gm = scene.grad_buffers()
        ps.render_backward(scene, o_, d_, params, drgb, logT, grads=(gg, gp, gm), n_live=live)
        assert ps.device_status() & 1
        ps.shade_nodes(scene, (2.0, 0.5, 0.5), 0.1, params)
        assert ps.device_status() & 1
    finally:
        ps.set_wait_polls(None)
    assert ps.wait_polls() == 1 << 24
    assert ps.device_status() == 0
    check_forward(sc, o, d, tau, N)
    check_backward(sc, o, d, tau, N)


def test_live_extent_matches_oracle_and_skipping_is_exact(sphere64):
    """n_live (1 + the last sample with a nonzero opacity) equals the oracle's
    on rays away from the clip kink, and the adjoint that skips the samples
    after it gives the gradients of the one that visits every sample."""
    sc, rays = sphere64
    o, d = rays.o[:600], rays.d[:600]
    tau, N = 64.0, 128
    scene = ps.Scene.from_host(sc)
    params = ps.render_params(tau, N, n_fresnel=sc.n_fresnel)
    out = ps.render_forward(scene, dev(o), dev(d), params, want_live=True)
    live = out[4].cpu().numpy()
    keep = clean_rays(sc, o, d, tau, N)
    m = oracle.Model.from_scene(sc)
    for i in keep[:120]:
        tr = oracle.render_trace(m, o[i], d[i], tau, N)
        ref = 0 if not tr["hit"] else int(np.nonzero(tr["w"] > 0)[0].max() + 1) \
            if np.any(tr["w"] > 0) else 0
        assert live[i] == ref, (i, live[i], ref)
    assert 0 < np.mean(live[live > 0]) < N  # samples are actually skipped
    g = synth.rng(17)
    drgb = (g.normal(size=(600, 3)) / 600).astype(np.float32)
    a = gpu_backward(scene, o, d, params, drgb, use_live=True)
    b = gpu_backward(scene, o, d, params, drgb, use_live=False)
    # equal up to FP32 summation order: the grid and probe entries sum a few
    # samples each; an MLP entry sums every sample of the batch through
    # tensor-memory tiles, shared-memory and global atomics whose order differs
    # between launches (the skipped chunks change which rows share a tile)
    for k in a:
        bar = 1e-5 if k == "mlp" else 1e-6
        assert rel_err_tensor(a[k], b[k]) <= bar, (k, rel_err_tensor(a[k], b[k]))


# ---------------------------------------------------------------------------
# The adjoint-stress configuration: 512^3 FP32 SDF + 3 BF16 features per node,
# probes 64^3 x 9 SH x 8 channels FP32, MLP 14 -> 32 -> 32 -> 3 (FP32-equivalent
# on the tensor cores), 2^20 rays x 512 samples, activations recomputed
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def stress512():
    sc = synth.make_scene("stress512")
    rays = synth.make_rays("stress512")
    return sc, rays


def test_adjoint_stress_oracle_subset(stress512):
    """The full 2^20 x 512 launch with a cotangent that is nonzero on 1024
    random rays only (rays away from the ReLU / alpha-clip kinks): its
    gradients are those rays' alone, and equal the FP64 oracle's on them (on
    the BF16-rounded feature values the kernels read) at the FP32 bar."""
    sc, rays = stress512
    tau, N = 64.0, 512
    n = rays.o.shape[0]
    ref_sc = stored_values(sc, feat_bf16=True)
    cand = synth.rng(91).choice(n, 2048, replace=False)
    clean = clean_rays(ref_sc, rays.o[cand], rays.d[cand], tau, N)
    assert clean.size >= 1024, clean.size
    sub = np.sort(cand[clean[:1024]])
    drgb = np.zeros((n, 3), np.float32)
    drgb[sub] = (synth.rng(92).normal(size=(sub.size, 3)) / sub.size).astype(np.float32)
    scene = ps.Scene.from_host(sc, feat_dtype=ps.BF16)
    params = ps.render_params(tau, N, 0, 3)
    gg = gpu_backward(scene, rays.o, rays.d, params, drgb)
    gr = oracle_backward(ref_sc, rays.o[sub], rays.d[sub], drgb[sub].astype(np.float64), tau, N)
    errs = {k: rel_err_tensor(gg[k], gr[k]) for k in ("sdf", "feat", "probes", "mlp")}
    log_errors("adjoint stress oracle subset", errs)
    for k, e in errs.items():
        assert e <= GRAD_RTOL, (k, e, errs)


def test_adjoint_stress_central_differences(stress512):
    """torch.autograd.Function gradients of L = sum(wts * rgb) over all 2^20
    rays x 512 samples against central differences of the FP32 forward,
    h = 1e-3, on 64 random parameters with significant gradients: probe
    coefficients and MLP weights (the BF16 feature storage cannot represent a
    1e-3 step, and an SDF step moves the alpha-clip kinks of Eq. 9; both are
    held to the oracle above).  Bars as the small-scene test: 10% per
    parameter, 2.5% over the 64 in the L2 sense."""
    sc, rays = stress512
    tau, N = 64.0, 512
    scene = ps.Scene.from_host(sc, feat_dtype=ps.BF16)
    gd32 = ps.grid_desc(sc.dims, sc.box_min, sc.box_max, 3, ps.F32)
    grid_master = ps.pack_grid(gd32, torch.as_tensor(sc.sdf, device="cuda"),
                               torch.as_tensor(sc.feat, device="cuda")).requires_grad_(True)
    probes = scene.probes.requires_grad_(True)
    mlp = scene.mlp.requires_grad_(True)
    params = ps.render_params(tau, N, 0, 3)
    o, d = dev(rays.o), dev(rays.d)
    wts = dev(synth.rng(93).normal(size=(rays.o.shape[0], 3)))
    rgb, _, _ = ps.render(scene, o, d, params, masters=(grid_master, probes))
    (rgb * wts).sum().backward()
    gp, gm = probes.grad.detach(), mlp.grad.detach()
    probes.requires_grad_(False)
    mlp.requires_grad_(False)

    def loss():
        out, _, _, _ = ps.render_forward(scene, o, d, params)
        return float((out.double() * wts.double()).sum())

    g = synth.rng(94)
    h = 1e-3
    fds, ans = [], []
    for tensor, grad, count in ((scene.probes, gp, 32), (scene.mlp, gm, 32)):
        flat, gflat = tensor.view(-1), grad.reshape(-1)
        nz = torch.nonzero(gflat.abs() > 0.1 * gflat.abs().max()).view(-1).cpu().numpy()
        for i in g.choice(nz, min(count, nz.size), replace=False):
            old = float(flat[i])
            flat[i] = old + h
            lp = loss()
            flat[i] = old - h
            lm = loss()
            flat[i] = old
            fd, an = (lp - lm) / (2 * h), float(gflat[i])
            assert abs(fd - an) <= 1e-1 * abs(an), (i, fd, an)
            fds.append(fd)
            ans.append(an)
    fds, ans = np.array(fds), np.array(ans)
    assert fds.size == 64
    rel = float(np.linalg.norm(fds - ans) / np.linalg.norm(ans))
    log_errors("adjoint stress central differences", {"l2_rel": rel})
    assert rel <= 2.5e-2, rel


# ---------------------------------------------------------------------------
# The human-capture configuration in reduced precision at its full size:
# 384 x 768 x 384 FP32 SDF + 3 BF16 features per node, probes 48 x 96 x 48 x
# 9 SH x 4 channels FP16, MLP FP16 on the tensor cores, 2^19 rays x 256
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def human384():
    sc = synth.make_scene("human384")
    rays = synth.make_rays("human384")
    return sc, rays


def test_reduced_precision_full_launch_sampled_parity(human384):
    """The benchmark's reduced-precision launch (2^19 rays x 256 samples on the
    full human-capture grid).  Forward: the colours of 256 random rays against
    the FP64 oracle on the stored values (BF16 features, FP16 probes, FP16 W1
    and W2), at the reduced-precision bar.  Adjoint: the whole launch with a
    cotangent that is nonzero on 512 random rays, against the oracle's
    gradients over those rays with the MLP's layer inputs rounded to FP16 as the
    tensor-core path stores them, so that both sides take the ReLU decisions on
    the same values (rays within the kink margin left out, as everywhere).
    Against the oracle with FP64 layer inputs the ReLU decisions of a few
    samples differ (FP16 rounding moves pre-activations by ~1e-3 of their
    scale, far beyond the kink margin); those errors are logged, not held to
    a bar."""
    sc, rays = human384
    tau, N = 64.0, 256
    n = rays.o.shape[0]
    ref_sc = stored_values(sc, feat_bf16=True, probe_f16=True, mlp_f16=True)
    scene = ps.Scene.from_host(sc, feat_dtype=ps.BF16, probe_dtype=ps.F16, mlp_dtype=ps.F16)
    params = ps.render_params(tau, N, 0, 3)
    g = gpu_forward(scene, rays.o, rays.d, params)
    for k in ("rgb", "depth", "wsum", "logT"):
        assert np.isfinite(g[k]).all(), k
    idx = np.sort(synth.rng(101).choice(n, 256, replace=False))
    r = oracle_forward(ref_sc, rays.o[idx], rays.d[idx], tau, N)
    assert np.sum(r["wsum"] > 0.5) > 20
    err = float(np.max(np.abs(g["rgb"][idx] - r["rgb"])))
    r16 = oracle_forward(ref_sc, rays.o[idx], rays.d[idx], tau, N, mlp_f16=True)
    err16 = float(np.max(np.abs(g["rgb"][idx] - r16["rgb"])))
    log_errors("reduced precision full launch forward",
               {"rgb_max_abs": err, "psnr_vs_oracle": psnr(g["rgb"][idx], r["rgb"]),
                "depth_rel": rel_err_elementwise(g["depth"][idx], r["depth"]),
                "rgb_max_abs_f16_inputs": err16})
    assert err <= RP_RGB_ABS, err
    assert err16 <= RP16_RGB_ABS, err16
    cand = synth.rng(102).choice(n, 1024, replace=False)
    clean = clean_rays(ref_sc, rays.o[cand], rays.d[cand], tau, N, mlp_f16=True)
    assert clean.size >= 512, clean.size
    sub = np.sort(cand[clean[:512]])
    drgb = np.zeros((n, 3), np.float32)
    drgb[sub] = (synth.rng(103).normal(size=(sub.size, 3)) / sub.size).astype(np.float32)
    gg = gpu_backward(scene, rays.o, rays.d, params, drgb)
    gr = oracle_backward(ref_sc, rays.o[sub], rays.d[sub], drgb[sub].astype(np.float64), tau, N,
                         mlp_f16=True)
    errs = {k: rel_err_tensor(gg[k], gr[k]) for k in ("sdf", "feat", "probes", "mlp")}
    errs.update({k + "_l2": l2_rel(gg[k], gr[k]) for k in ("sdf", "feat", "probes", "mlp")})
    gp = oracle_backward(ref_sc, rays.o[sub], rays.d[sub], drgb[sub].astype(np.float64), tau, N)
    errs.update({k + "_plain": rel_err_tensor(gg[k], gp[k]) for k in ("sdf", "feat", "probes", "mlp")})
    errs["rays_hit"] = int(np.sum(oracle_forward(ref_sc, rays.o[sub], rays.d[sub], tau, N)["wsum"] > 0.5))
    log_errors("reduced precision full launch backward", errs)
    for k in ("sdf", "feat", "probes", "mlp"):
        assert errs[k] <= RP16_GRAD_RTOL, (k, errs)


# ---------------------------------------------------------------------------
# The 1080p inference launch: 8 novel 1920 x 1080 views of the object-capture
# scene per launch (16.6 M rays)
# ---------------------------------------------------------------------------

def test_inference_launch_sampled_parity(object256):
    """Both forms of the 1080p inference comparison at the benchmark's launch
    size: the FP32 uniform 256-sample render at the FP32 bars, and the BF16 /
    FP16 render placed by 16 per-bin densities (N' = 128) at the
    reduced-precision bar, on 256 random pixels against the FP64 oracle.  The
    densities are seeded FP32 inputs given to both sides."""
    sc, _ = object256
    tau = 64.0
    spec = synth.WORKLOADS["object256"]
    views = [synth.image_rays(c, 1920, 1080, spec["fov"])
             for c in synth.novel_cameras("object256", 8)]
    o = np.concatenate([v[0] for v in views])
    d = np.concatenate([v[1] for v in views])
    n = o.shape[0]
    assert n == 8 * 1920 * 1080
    idx = np.sort(synth.rng(104).choice(n, 256, replace=False))

    scene = ps.Scene.from_host(sc)
    g = gpu_forward(scene, o, d, ps.render_params(tau, 256, 0, 3))
    r = oracle_forward(sc, o[idx], d[idx], tau, 256)
    r32 = oracle_forward(sc, o[idx], d[idx], tau, 256, sdf_fp32=True)
    assert np.sum(r["wsum"] > 0.5) > 20
    for k in ("rgb", "depth", "wsum"):
        e = rel_err_elementwise(g[k][idx], r[k])
        assert e <= RGB_DEPTH_RTOL, (k, e)
        e32 = rel_err_elementwise(g[k][idx], r32[k], floor=REL_FLOOR_S32)
        assert e32 <= RGB_DEPTH_RTOL, (k + " (FP32-rounded s, 1e-3 floor)", e32)
    del g, scene
    torch.cuda.empty_cache()

    B, n_out = 16, 128
    q = (0.2 + 0.8 * synth.rng(105).random(size=(n, B), dtype=np.float32)) ** 3
    q /= q.sum(1, keepdims=True)
    fast = ps.Scene.from_host(sc, feat_dtype=ps.BF16, probe_dtype=ps.F16, mlp_dtype=ps.F16)
    params = ps.render_params(tau, n_out, n_fresnel=sc.n_fresnel, n_bins=B)
    rgb, depth, wsum, _ = ps.render_forward(fast, dev(o), dev(d), params, dev(q))
    assert ps.device_status() == 0
    rgb, depth = rgb.cpu().numpy()[idx], depth.cpu().numpy()[idx]
    m = oracle.Model.from_scene(stored_values(sc, feat_bf16=True, probe_f16=True))
    t_ref = oracle.place_samples(m, o[idx], d[idx], q[idx].astype(np.float64), n_out)
    ref = oracle.render_forward(m, o[idx], d[idx], tau, n_out, t_samples=t_ref)
    err = float(np.max(np.abs(rgb - ref["rgb"])))
    log_errors("inference launch reduced precision + bin densities",
               {"rgb_max_abs": err, "psnr_vs_oracle": psnr(rgb, ref["rgb"]),
                "depth_rel": rel_err_elementwise(depth, ref["depth"])})
    assert err <= RP_RGB_ABS, err
