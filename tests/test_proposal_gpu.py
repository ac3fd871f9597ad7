"""Parity of the learned-proposal kernels with the FP64 oracle (GPU only):
coarse occupancy, the uniform render's weight histogram, the proposal's
density and sample placement, and its cross-entropy gradient."""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import log_errors, rel_err_tensor

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2412_10084_gb300 as ps

MIX = 0.1


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def scene_and_rays(dims=(32, 32, 32), probe_dims=(8, 8, 8), n_rays=700, seed_offset=41,
                   name="sphere64"):
    sc = synth.make_scene(name, dims=dims, probe_dims=probe_dims)
    rays = synth.make_rays(name, n_rays=n_rays, seed_offset=seed_offset)
    return sc, rays.o, rays.d


def proposal_params(seed=3, logit_scale=4.0, B=8):
    p = synth.proposal_params(synth.rng(seed), n_bins=B).astype(np.float32)
    p[-B - B * 32:] *= logit_scale  # spread the initial logits past the fallback
    return p


def threshold_f32(sc, voxels=2.0):
    ext = float(sc.box_max[0] - sc.box_min[0]) / (sc.dims[0] - 1)
    return float(np.float32(voxels * ext))


@pytest.mark.parametrize("res", [(8, 8, 8), (32, 32, 32), (7, 5, 9), (64, 2, 33)])
def test_occupancy_exact(res):
    sc, _, _ = scene_and_rays(dims=(40, 33, 37), probe_dims=(5, 5, 5))
    scene = ps.Scene.from_host(sc)
    thr = threshold_f32(sc)
    bits = ps.occupancy_build(scene, res, thr)
    occ = ps.occupancy_unpack(bits, res).numpy()
    ref = oracle.occupancy(oracle.Model.from_scene(sc), res, thr)
    assert occ.shape == ref.shape
    assert np.array_equal(occ, ref)
    assert 0 < occ.mean() < 1
    # padding bits of the last word stay clear
    n = res[0] * res[1] * res[2]
    if n % 32:
        last = int(bits[-1].item()) & 0xFFFFFFFF
        assert last >> (n % 32) == 0


def test_occupancy_bf16_grid_reads_fp32_sdf():
    sc, _, _ = scene_and_rays(dims=(24, 24, 24), probe_dims=(4, 4, 4))
    scene = ps.Scene.from_host(sc, feat_dtype=ps.BF16)
    thr = threshold_f32(sc)
    occ = ps.occupancy_unpack(ps.occupancy_build(scene, (12, 12, 12), thr), (12, 12, 12)).numpy()
    assert np.array_equal(occ, oracle.occupancy(oracle.Model.from_scene(sc), (12, 12, 12), thr))


@pytest.mark.parametrize("N,B", [(64, 8), (256, 8), (48, 8), (96, 32)])
def test_weight_histogram(N, B):
    sc, o, d = scene_and_rays(n_rays=500, seed_offset=N + B)
    scene = ps.Scene.from_host(sc)
    tau = 64.0
    params = ps.render_params(tau, N, n_fresnel=sc.n_fresnel)
    h = ps.weight_histogram(scene, dev(o), dev(d), params, B).cpu().numpy().astype(np.float64)
    ref = oracle.weight_histogram(oracle.Model.from_scene(sc), o, d, tau, N, B)
    err = np.max(np.abs(h - ref))
    log_errors("weight_histogram", {"abs": float(err)})
    assert err <= 2e-6, err
    # bins add up to the render's weight sum
    _, _, wsum, _ = ps.render_forward(scene, dev(o), dev(d), params)
    assert np.max(np.abs(h.sum(1) - wsum.cpu().numpy())) <= 2e-6


def _forward_pair(sc, o, d, prm, n_out, theta, res=(16, 16, 16), n_sub=8, B=8):
    scene = ps.Scene.from_host(sc)
    thr = threshold_f32(sc)
    occ = ps.occupancy_build(scene, res, thr)
    desc = ps.proposal_desc(res, n_bins=B, mix=MIX, theta=theta, n_sub=n_sub)
    t, probs = ps.proposal_forward(scene, desc, dev(prm), occ, dev(o), dev(d), n_out)
    m = oracle.Model.from_scene(sc)
    prop = oracle.Proposal(oracle.occupancy(m, res, thr), prm, n_bins=B, mix=MIX, theta=theta,
                           n_sub=n_sub)
    ref = oracle.proposal_forward(m, prop, o, d, n_out)
    return t.cpu().numpy().astype(np.float64), probs.cpu().numpy().astype(np.float64), ref


@pytest.mark.parametrize("n_out,theta,n_sub,res,B", [(32, 0.0, 8, (16, 16, 16), 8),
                                                     (17, 0.2, 3, (9, 16, 7), 8),
                                                     (64, "median", 8, (32, 32, 32), 8),
                                                     (1, 0.0, 1, (64, 64, 64), 8),
                                                     (48, 0.1, 4, (32, 32, 32), 16),
                                                     (7, "median", 8, (20, 24, 28), 16)])
def test_proposal_forward(n_out, theta, n_sub, res, B):
    sc, o, d = scene_and_rays(n_rays=900, seed_offset=n_out)
    prm = proposal_params(B=B)
    if theta == "median":  # half the rays fall back to uniform placement
        _, _, ref = _forward_pair(sc, o, d, prm, n_out, 0.0, res, n_sub, B)
        theta = float(np.float32(np.median(ref["probs"].max(1))))
    t, probs, ref = _forward_pair(sc, o, d, prm, n_out, theta, res, n_sub, B)
    # rays whose fallback decision sits at the threshold may go either way
    qmax = ref["probs"].max(1)
    settled = np.abs(qmax - theta) > 1e-4
    perr = np.max(np.abs(probs - ref["probs"])[settled])
    tn, tf = ref["t"][:, 0], ref["t"][:, -1]
    span = (tf - tn)[:, None]
    # t = t_n + (b + (u - c_b) / q_b) span / B, c_b the density summed over the
    # bins before b.  An error in c_b, u or q_b moves t by at most
    # (|dc_b| + |du| + |dq_b|) / q_b bin widths, and q_b >= mix / (4 B), so
    # |dt| <= 4 (sum_b |dq_b| + FP32 rounding of the running sum) / mix x span,
    # plus the rounding of t itself.
    dq = np.abs(probs - ref["probs"]).sum(1)[:, None]
    bound = 4 * (dq + 2e-6) / MIX * span + 2 * np.spacing(np.float32(np.abs(ref["t"]).max()))
    ratio = np.max((np.abs(t - ref["t"]) / bound)[settled])
    terr = np.max((np.abs(t - ref["t"]) / np.maximum(span, 1e-6))[settled])
    log_errors(f"proposal_forward n_out={n_out} theta={theta} n_sub={n_sub} res={res} B={B}",
               {"probs_abs": float(perr), "t_rel_span": float(terr), "t_over_bound": float(ratio)})
    assert perr <= 2e-6, perr
    assert ratio <= 1.0, (ratio, terr)
    hit = tf > tn
    assert hit.any() and (~hit).any()
    assert np.all(t[~hit] == 0)
    assert np.all(np.diff(t[hit], axis=1) >= 0)
    assert probs.shape == (o.shape[0], B)
    assert np.array_equal(t[hit, 0], ref["t"][hit, 0]) and np.array_equal(t[hit, -1],
                                                                          ref["t"][hit, -1])


def test_proposal_fallback_is_uniform():
    sc, o, d = scene_and_rays(n_rays=300, seed_offset=77)
    prm = proposal_params()
    t, probs, ref = _forward_pair(sc, o, d, prm, 24, theta=1.0)
    np.testing.assert_array_equal(probs, 0.125)
    hit = ref["t"][:, -1] > ref["t"][:, 0]
    tn, tf = ref["t"][hit, :1], ref["t"][hit, -1:]
    uniform = tn + (tf - tn) * np.arange(25)[None] / 24
    # exact up to the rounding of the FP32 bin width and of t itself
    tol = 1e-6 * (tf - tn) + 2 * np.spacing(np.float32(np.abs(uniform).max()))
    assert np.all(np.abs(t[hit] - uniform) <= tol)


def test_proposal_samples_drive_the_render():
    """Proposal-placed distances go straight into the render's explicit-t mode
    and reproduce the oracle's render at those distances."""
    sc, o, d = scene_and_rays(n_rays=400, seed_offset=91)
    prm = proposal_params()
    n_out = 32
    scene = ps.Scene.from_host(sc)
    res = (16, 16, 16)
    occ = ps.occupancy_build(scene, res, threshold_f32(sc))
    desc = ps.proposal_desc(res, mix=MIX, theta=0.0)
    o_, d_ = dev(o), dev(d)
    t, _ = ps.proposal_forward(scene, desc, dev(prm), occ, o_, d_, n_out, want_probs=False)
    hit = (t[:, -1] > t[:, 0]).cpu().numpy()
    params = ps.render_params(64.0, n_out, n_fresnel=sc.n_fresnel)
    rgb, depth, wsum, _ = ps.render_forward(scene, o_[hit], d_[hit], params, t[hit].contiguous())
    ref = oracle.render_forward(oracle.Model.from_scene(sc), o[hit], d[hit], 64.0, n_out,
                                t_samples=t[hit].cpu().numpy())
    assert np.max(np.abs(rgb.cpu().numpy() - ref["rgb"])) <= 1e-5
    assert np.max(np.abs(wsum.cpu().numpy() - ref["wsum"])) <= 1e-5


@pytest.mark.parametrize("B", [8, 16])
def test_proposal_backward(B):
    sc, o, d = scene_and_rays(n_rays=1500, seed_offset=5 + B)
    prm = proposal_params(seed=8, logit_scale=1.0, B=B)
    res = (16, 16, 16)
    thr = threshold_f32(sc)
    m = oracle.Model.from_scene(sc)
    prop = oracle.Proposal(oracle.occupancy(m, res, thr), prm, n_bins=B, mix=MIX, theta=0.2)
    # keep rays at least 1e-4 from a ReLU kink (both precisions switch alike)
    keep = oracle.proposal_forward(m, prop, o, d, 8)["margin"] > 1e-4
    o, d = o[keep], d[keep]
    # both sides see the same FP32-rounded targets
    hist = oracle.weight_histogram(m, o, d, 64.0, 64, B).astype(np.float32).astype(np.float64)
    assert np.mean(hist.sum(1) >= 1e-3) > 0.3
    g_ref, loss_ref = oracle.proposal_backward(m, prop, o, d, hist, 1e-3, 1.0 / len(o))
    scene = ps.Scene.from_host(sc)
    occ = ps.occupancy_build(scene, res, thr)
    desc = ps.proposal_desc(res, n_bins=B, mix=MIX, theta=0.2)
    grad, loss = ps.proposal_backward(scene, desc, dev(prm), occ, dev(o), dev(d), dev(hist),
                                      1e-3, 1.0 / len(o))
    grad, loss = grad.cpu().numpy(), loss.cpu().numpy()
    assert np.max(np.abs(loss - loss_ref) / np.maximum(loss_ref, 1e-2)) <= 1e-5
    W, nin = 32, 7 + 2 * B
    cuts = np.cumsum([W * nin, W, W * W, W, B * W, B])
    names = ["W1", "b1", "W2", "b2", "W3", "b3"]
    errs = {n: rel_err_tensor(gp, gr) for n, gp, gr in
            zip(names, np.split(grad, cuts[:-1]), np.split(g_ref, cuts[:-1]))}
    log_errors(f"proposal_backward B={B}", errs)
    for n, e in errs.items():
        assert e <= 1e-4, (n, e)
    # ACCUMULATE semantics: a second call adds the same gradient again
    g2 = torch.tensor(grad, device="cuda")
    ps.proposal_backward(scene, desc, dev(prm), occ, dev(o), dev(d), dev(hist), 1e-3,
                         1.0 / len(o), grad=g2, want_loss=False)
    assert rel_err_tensor(g2.cpu().numpy(), 2 * g_ref) <= 1e-4


def test_proposal_host_validation():
    sc, o, d = scene_and_rays(dims=(16, 16, 16), probe_dims=(4, 4, 4), n_rays=8)
    scene = ps.Scene.from_host(sc)
    occ = ps.occupancy_build(scene, (8, 8, 8), 0.1)
    prm = dev(proposal_params())
    with pytest.raises(ps.LibraryError):
        ps.proposal_forward(scene, ps.proposal_desc((8, 8, 8), n_bins=12), prm, occ, dev(o),
                            dev(d), 8)
    with pytest.raises(ps.LibraryError):
        ps.proposal_forward(scene, ps.proposal_desc((8, 8, 8), mix=1.0), prm, occ, dev(o),
                            dev(d), 8)
    with pytest.raises(ps.LibraryError):
        ps.proposal_forward(scene, ps.proposal_desc((8, 8, 8)), prm, occ, dev(o), dev(d), 0)
    with pytest.raises(ps.LibraryError):
        ps.proposal_forward(scene, ps.proposal_desc((8, 8, 8), n_sub=0), prm, occ, dev(o),
                            dev(d), 8)
    with pytest.raises(ps.LibraryError):
        ps.occupancy_build(scene, (65, 8, 8), 0.1)
    with pytest.raises(ps.LibraryError):
        ps.weight_histogram(scene, dev(o), dev(d), ps.render_params(64.0, 60), 8)
    t, _ = ps.proposal_forward(scene, ps.proposal_desc((8, 8, 8)), prm, occ, dev(o[:0]),
                               dev(d[:0]), 8)
    assert t.shape == (0, 9)


@pytest.mark.parametrize("B", [8, 16])
def test_bin_density_render_equals_explicit_distances(B):
    """The render placing samples from the proposal's bin densities uses the
    very distances the proposal writes: forward outputs are bit-identical and
    the adjoints agree to summation order."""
    sc, o, d = scene_and_rays(n_rays=700, seed_offset=30 + B)
    scene = ps.Scene.from_host(sc)
    res = (16, 16, 16)
    occ = ps.occupancy_build(scene, res, threshold_f32(sc))
    desc = ps.proposal_desc(res, n_bins=B, mix=0.3, theta=0.0)
    o_, d_ = dev(o), dev(d)
    n_out = 45
    t, q = ps.proposal_forward(scene, desc, dev(proposal_params(B=B)), occ, o_, d_, n_out)
    pe = ps.render_params(64.0, n_out, n_fresnel=sc.n_fresnel)
    pb = ps.render_params(64.0, n_out, n_fresnel=sc.n_fresnel, n_bins=B)
    a = ps.render_forward(scene, o_, d_, pe, t, want_live=True)
    b = ps.render_forward(scene, o_, d_, pb, q, want_live=True)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    drgb = dev(synth.rng(5).normal(size=(700, 3)) / 700)
    ga = ps.render_backward(scene, o_, d_, pe, drgb, a[3], t_samples=t, n_live=a[4])
    gb = ps.render_backward(scene, o_, d_, pb, drgb, b[3], t_samples=q, n_live=b[4])
    for x, y in zip(ga, gb):
        assert rel_err_tensor(x.cpu().numpy(), y.cpu().numpy()) <= 1e-6


def test_bin_density_render_parity_with_oracle():
    sc, o, d = scene_and_rays(n_rays=500, seed_offset=77)
    B, n_out = 16, 40
    g = synth.rng(12)
    q = g.uniform(0.2, 1.0, size=(500, B)) ** 3
    q = (q / q.sum(1, keepdims=True)).astype(np.float32)  # the same FP32 densities both sides
    scene = ps.Scene.from_host(sc)
    params = ps.render_params(64.0, n_out, n_fresnel=sc.n_fresnel, n_bins=B)
    rgb, depth, wsum, _ = ps.render_forward(scene, dev(o), dev(d), params, dev(q))
    m = oracle.Model.from_scene(sc)
    t_ref = oracle.place_samples(m, o, d, q.astype(np.float64), n_out)
    ref = oracle.render_forward(m, o, d, 64.0, n_out, t_samples=t_ref)
    for name, x in (("rgb", rgb), ("depth", depth), ("wsum", wsum)):
        err = np.max(np.abs(x.cpu().numpy() - ref[name]) / np.maximum(np.abs(ref[name]), 1e-2))
        assert err <= 1e-5, (name, err)
