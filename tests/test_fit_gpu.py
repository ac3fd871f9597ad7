"""Training on the library's kernels (GPU only): the Adam update against its
textbook definition, appearance fitting, and the learned proposal's gain over
uniform marching at an equal sample count."""
import math

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2412_10084_gb300 as ps
    from paper_2412_10084_gb300 import fit


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def adam_reference(p, grads, lr, b1, b2, eps):
    """Kingma & Ba (2015), Algorithm 1, in FP64."""
    p = p.astype(np.float64).copy()
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for t, g in enumerate(grads, start=1):
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        p -= lr * mh / (np.sqrt(vh) + eps)
    return p


@pytest.mark.parametrize("n", [1, 4, 1003, 1 << 16])
def test_adam_matches_definition(n):
    g = synth.rng(n)
    p0 = g.normal(size=n).astype(np.float32)
    grads = [g.normal(size=n).astype(np.float32) * 10.0 ** g.uniform(-3, 1) for _ in range(5)]
    p, m, v = dev(p0), torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    for t, gr in enumerate(grads, start=1):
        gt = dev(gr)
        ps.adam_step(p, gt, m, v, t, 1e-2, 0.9, 0.99, 1e-8)
        assert float(gt.abs().max()) == 0.0  # cleared in the same pass
    ref = adam_reference(p0, [gr.astype(np.float64) for gr in grads], 1e-2, 0.9, 0.99, 1e-8)
    # each update moves a parameter by at most lr (times a bounded ratio):
    # FP32 rounding of the five updates stays within 1e-6 of lr
    assert np.max(np.abs(p.cpu().numpy() - ref)) <= 1e-6 * 5


@pytest.fixture(scope="module")
def fitted_scene():
    """object-capture scene at 128^3 with its appearance fitted (150 steps)
    to teacher colours; returns (host scene, device scene, fit log)."""
    sc = synth.make_scene("object256", dims=(128, 128, 128), probe_dims=(16, 16, 16))
    pool = synth.training_pool("object256", 1 << 15, seed_offset=7)
    scene = ps.Scene.from_host(sc)
    params = ps.render_params(64.0, 128, n_fresnel=sc.n_fresnel)
    sdf_before = scene.grid[:, 0].clone()
    log = fit.fit_appearance(scene, dev(pool.o), dev(pool.d), dev(pool.target), params,
                             steps=150, batch=1 << 13, log_every=25)
    return sc, scene, log, sdf_before


def psnr_inside(rgb, ref_rgb, ref_wsum):
    mask = ref_wsum > 0.5
    mse = float(((rgb[mask] - ref_rgb[mask]) ** 2).mean())
    return 10 * math.log10(1.0 / max(mse, 1e-20)), int(mask.sum())


def test_fit_appearance_reduces_loss(fitted_scene):
    _, scene, log, sdf_before = fitted_scene
    assert ps.device_status() == 0
    first, last = log[0][1], log[-1][1]
    assert math.isfinite(last) and last < 0.5 * first, log
    assert torch.equal(scene.grid[:, 0], sdf_before)  # geometry frozen


def test_trained_proposal_beats_uniform_at_equal_samples(fitted_scene):
    """What the learned proposal gains: at the same sample count, its placement
    renders closer to the uniform 1024-sample reference than uniform marching
    (PSNR inside the silhouette and depth error), on held-out rays."""
    _, scene, _, _ = fitted_scene
    tau = 64.0
    B, R = 16, (64, 64, 64)
    prop = fit.Proposal.create(scene, synth.proposal_params(synth.rng(11), n_bins=B),
                               occ_res=R, n_bins=B, mix=0.25, theta=0.0)
    train = synth.make_rays("object256", n_rays=1 << 19, seed_offset=8)
    log = fit.train_proposal(scene, prop, dev(train.o), dev(train.d), tau, n_uniform=256,
                             steps=1000, batch=1 << 15, log_every=100)
    assert ps.device_status() == 0
    assert log[-1][1] < log[0][1], log
    test = synth.make_rays("object256", n_rays=1 << 16, seed_offset=99)
    to, td = dev(test.o), dev(test.d)
    ref = ps.render_forward(scene, to, td, ps.render_params(tau, 1024, n_fresnel=3))
    ref_rgb, ref_depth, ref_w = (x.cpu().numpy() for x in ref[:3])
    mask = ref_w > 0.5
    results = {}
    for n in (32, 64, 128):
        p = ps.render_params(tau, n, n_fresnel=3)
        uni = ps.render_forward(scene, to, td, p)
        pro = fit.render_proposed(scene, prop, to, td, n, p)
        pu, cnt = psnr_inside(uni[0].cpu().numpy(), ref_rgb, ref_w)
        pp, _ = psnr_inside(pro[0].cpu().numpy(), ref_rgb, ref_w)
        du = float(np.abs(uni[1].cpu().numpy() - ref_depth)[mask].mean())
        dp = float(np.abs(pro[1].cpu().numpy() - ref_depth)[mask].mean())
        results[n] = (round(pu, 2), round(pp, 2), du, dp)
        assert cnt > 2000
    print("uniform vs proposal PSNR / depth error:", results)
    for n, (pu, pp, du, dp) in results.items():
        assert pp > pu + 3.0, (n, results)
        assert dp < du, (n, results)
