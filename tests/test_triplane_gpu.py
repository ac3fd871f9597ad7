"""Tile tri-plane spatial features (Sec. 3.1, Sec. 4) on the GPU against the
FP64 oracle: forward, adjoint, pack/unpack, host validation."""
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


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def tri_scene(dims=(40, 33, 37), probe_dims=(7, 6, 5), seed=21, width=16):
    sc = synth.make_scene("sphere64", dims=dims, probe_dims=probe_dims)
    if width != sc.width:
        g = synth.rng(seed + 1)
        import dataclasses
        sc = dataclasses.replace(sc, width=width, mlp=synth.mlp_params(10, width, g))
    return synth.with_triplanes(sc, seed)


@pytest.mark.parametrize("width,N", [(16, 64), (32, 45)])
def test_triplane_forward_parity(width, N):
    sc = tri_scene(width=width)
    rays = synth.make_rays("sphere64", n_rays=600, seed_offset=40 + N)
    scene = ps.Scene.from_host(sc)
    assert scene.feat_layout == ps.FEAT_TRIPLANE
    params = ps.render_params(64.0, N, n_fresnel=sc.n_fresnel)
    rgb, depth, wsum, logT = ps.render_forward(scene, dev(rays.o), dev(rays.d), params)
    ref = oracle_forward(sc, rays.o, rays.d, 64.0, N)
    errs = {k: rel_err_elementwise(v.cpu().numpy(), ref[k])
            for k, v in (("rgb", rgb), ("depth", depth), ("wsum", wsum))}
    log_errors(f"triplane forward W={width} N={N}", errs)
    for k, e in errs.items():
        assert e <= RGB_DEPTH_RTOL, (k, e)
    assert ps.device_status() == 0


@pytest.mark.parametrize("width", [16, 32])
def test_triplane_backward_parity(width):
    sc = tri_scene(width=width, seed=23)
    rays = synth.make_rays("sphere64", n_rays=500, seed_offset=50 + width)
    tau, N = 64.0, 64
    keep = clean_rays(sc, rays.o, rays.d, tau, N)
    o, d = rays.o[keep], rays.d[keep]
    n = o.shape[0]
    drgb = (synth.rng(9).normal(size=(n, 3)) / n).astype(np.float32)
    scene = ps.Scene.from_host(sc)
    params = ps.render_params(tau, N, n_fresnel=sc.n_fresnel)
    o_, d_ = dev(o), dev(d)
    _, _, _, logT, live = ps.render_forward(scene, o_, d_, params, want_live=True)
    gg, gp, gm = ps.render_backward(scene, o_, d_, params, dev(drgb), logT, n_live=live)
    gd, _, _ = scene.descs(params.n_fresnel)
    gsdf, gplanes = ps.unpack_grid(gd, gg, which=ps.GRID_GRAD)
    assert ps.device_status() == 0
    ref = oracle_backward(sc, o, d, drgb.astype(np.float64), tau, N)
    errs = {"sdf": rel_err_tensor(gsdf.cpu().numpy(), ref["sdf"]),
            "planes": rel_err_tensor(gplanes.cpu().numpy(), ref["feat"]),
            "probes": rel_err_tensor(gp.cpu().numpy(), ref["probes"]),
            "mlp": rel_err_tensor(gm.cpu().numpy(), ref["mlp"])}
    log_errors(f"triplane backward W={width}", errs)
    assert np.abs(ref["feat"]).max() > 0
    for k, e in errs.items():
        assert e <= GRAD_RTOL, (k, e)


def test_triplane_pack_roundtrip_and_validation():
    sc = tri_scene(dims=(19, 34, 17))
    gd = ps.grid_desc(sc.dims, sc.box_min, sc.box_max, 3, ps.F32, ps.FEAT_TRIPLANE)
    vb, gb = ps.grid_bytes(gd)
    tx, ty, tz = ps.tri_tiles(sc.dims)
    assert (tx, ty, tz) == (2, 3, 1)
    n = int(np.prod(sc.dims))
    assert vb == gb == ((4 * n + 15) // 16) * 16 + 16 * tx * ty * tz * 3 * 256
    packed = ps.pack_grid(gd, dev(sc.sdf), dev(sc.planes))
    sdf, planes = ps.unpack_grid(gd, packed, which=ps.GRID_VALUES)
    assert np.array_equal(sdf.cpu().numpy(), sc.sdf)
    assert np.array_equal(planes.cpu().numpy(), sc.planes)
    bad = ps.grid_desc(sc.dims, sc.box_min, sc.box_max, 3, ps.BF16, ps.FEAT_TRIPLANE)
    with pytest.raises(ps.LibraryError):
        ps.grid_bytes(bad)
