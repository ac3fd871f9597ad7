"""Training loops on the library's kernels.

fit_appearance: the scene's features, probes and MLP (optionally the SDF)
are fitted to target colours with an L2 photometric loss, the render's
forward and adjoint kernels and the library's Adam (Sec. 3.4; the paper's
regularisers and coarse-to-fine schedule are left out: the loop exists to
give synthetic scenes a non-trivial appearance).

train_proposal: the learned sample proposal is trained on rays the method
itself renders: its target is the per-bin histogram of the uniform march's
weights w_k (Eqs. 8-10), its loss the cross-entropy against its softmax, its
gradient the library's proposal adjoint, its optimiser the library's Adam.

render_proposed: proposal placement followed by the render at those
distances (inference).

Torch supplies device memory, random batch indices and the loss's
elementwise gradient; every render, adjoint, histogram and update step runs
in the library.
"""
from __future__ import annotations

import dataclasses

import torch

from . import (F32, FEAT_TRIPLANE, Adam, LibraryError, RenderParams, Scene, device_status,
               grid_regularizers, occupancy_build, probe_smoothness, proposal_backward,
               proposal_desc, proposal_forward, proposal_param_count, render_backward,
               render_forward, render_params, table_words, weight_histogram)


def _check_device(what: str, step: int):
    """Raises if a kernel since the last check gave up waiting on its
    tensor-core work (it then returned with part of its rays or gradients
    missing, so the parameters updated from them are not to be trusted)."""
    flags = device_status()
    if flags:
        raise LibraryError(f"{what}: a render kernel stopped early (device status {flags:#x}) "
                           f"before step {step}")


def _batch(gen, n_pool, batch, device):
    return torch.randint(0, n_pool, (batch,), generator=gen, device=device)


def trainable_grid(gd, values, grad):
    """Flat views of an FP32-stored grid's values and gradient that an
    optimiser may update (a sparse grid's brick table left out), and the view
    of the gradient's SDF entries: column 0 of the {sdf, f0, f1, f2} records,
    or the leading FP32 SDF array of the tri-plane layout."""
    vals, grads = values.view(-1), grad.view(-1)
    if gd.n_bricks > 0:
        w = table_words(gd)
        vals, grads = vals[w:], grads[w:]
    if gd.feat_layout == FEAT_TRIPLANE:
        sdf = grads[:int(gd.dims[0]) * int(gd.dims[1]) * int(gd.dims[2])]
    else:
        sdf = grads.view(-1, 4)[:, 0]
    return vals, grads, sdf


def fit_appearance(scene: Scene, rays_o, rays_d, target, params: RenderParams, steps=200,
                   batch=1 << 14, lr_grid=1e-2, lr_probes=1e-2, lr_mlp=2e-3, train_sdf=False,
                   seed=0, log_every=50, lam_features=0.0, lam_probes=0.0):
    """Fits an FP32-stored scene in place; returns [(step, mean L2 loss)].

    lam_features (tile tri-plane grids) and lam_probes add the paper's
    smoothness terms L_features (Eq. 14) and L_probes (Eq. 15), with their
    gradients from the library's kernels, to the photometric objective."""
    if (scene.feat_dtype, scene.probe_dtype, scene.mlp_dtype) != (F32, F32, F32):
        raise LibraryError("fit_appearance trains FP32 storage; convert afterwards")
    dev = scene.grid.device
    gg, gp, gm = scene.grad_buffers()
    gd, pd, _ = scene.descs(3)
    grid_vals, grid_grads, sdf_grads = trainable_grid(gd, scene.grid, gg)
    if lam_features > 0.0:
        if gd.feat_layout != FEAT_TRIPLANE:
            raise LibraryError("fit_appearance: lam_features needs tile tri-plane features")
        # the regulariser call takes the raw SDF; with zero SDF weights it adds
        # nothing to the SDF gradients (which this loop zeroes anyway)
        n_nodes = int(gd.dims[0]) * int(gd.dims[1]) * int(gd.dims[2])
        s_hat = sdf_grads.new_zeros(n_nodes)
        d_hat = sdf_grads.new_zeros(n_nodes)
    opt = Adam([(grid_vals, grid_grads, lr_grid),
                (scene.probes.view(-1), gp.view(-1), lr_probes),
                (scene.mlp.view(-1), gm.view(-1), lr_mlp)])
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    n_pool = rays_o.shape[0]
    log = []
    for step in range(1, steps + 1):
        idx = _batch(gen, n_pool, batch, dev)
        o, d, tgt = rays_o[idx], rays_d[idx], target[idx]
        rgb, _, _, logT, live = render_forward(scene, o, d, params, want_live=True)
        diff = rgb - tgt
        d_rgb = (2.0 / batch) * diff
        render_backward(scene, o, d, params, d_rgb.contiguous(), logT, grads=(gg, gp, gm),
                        n_live=live)
        if lam_features > 0.0:
            grid_regularizers(gd, s_hat, scene.grid, gg, d_hat, 0.0, 0.0, 0.0, lam_features)
        if lam_probes > 0.0:
            probe_smoothness(pd, scene.probes, gp, lam_probes)
        if not train_sdf:
            sdf_grads.zero_()
        opt.step()
        if step % log_every == 0 or step == steps:
            _check_device("fit_appearance", step)
            log.append((step, float((diff * diff).sum(1).mean())))
    return log


@dataclasses.dataclass
class Proposal:
    """A learned sample proposal: its descriptor, FP32 parameters and the
    coarse occupancy it reads."""
    desc: object
    params: torch.Tensor
    occ: torch.Tensor

    @classmethod
    def create(cls, scene: Scene, init_params, occ_res=(32, 32, 32), voxels=2.0, mix=0.1,
               theta=0.2, n_sub=8, n_bins=8):
        """Occupancy from the scene's SDF with a threshold of `voxels` fine
        voxel sizes; parameters copied from init_params (host or device)."""
        desc = proposal_desc(occ_res, n_bins=n_bins, mix=mix, theta=theta, n_sub=n_sub)
        n = proposal_param_count(desc)
        p = torch.as_tensor(init_params, dtype=torch.float32).to(scene.grid.device).contiguous()
        if p.numel() != n:
            raise LibraryError(f"proposal parameters: expected {n}, got {p.numel()}")
        vox = min((scene.box_max[a] - scene.box_min[a]) / (scene.dims[a] - 1) for a in range(3))
        occ = occupancy_build(scene, occ_res, voxels * vox)
        return cls(desc=desc, params=p, occ=occ)


def train_proposal(scene: Scene, prop: Proposal, rays_o, rays_d, tau, n_uniform=256, steps=500,
                   batch=1 << 14, lr=1e-2, lr_final=5e-4, min_mass=1e-3, seed=1, log_every=50):
    """Trains prop.params in place on random batches of the ray pool (Adam,
    cosine decay of the rate from lr to lr_final); returns [(step, mean of
    the rays' normalised cross-entropy, mean over rays with mass)]."""
    import math
    dev = scene.grid.device
    grad = torch.zeros_like(prop.params)
    opt = Adam([(prop.params, grad, lr)])
    params = render_params(tau, n_uniform)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    n_pool = rays_o.shape[0]
    log = []
    for step in range(1, steps + 1):
        idx = _batch(gen, n_pool, batch, dev)
        o, d = rays_o[idx], rays_d[idx]
        hist = weight_histogram(scene, o, d, params, prop.desc.n_bins)
        _, loss = proposal_backward(scene, prop.desc, prop.params, prop.occ, o, d, hist,
                                    min_mass, 1.0 / batch, grad=grad,
                                    want_loss=(step % log_every == 0 or step == steps))
        rate = lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * (step - 1) / steps))
        opt.groups[0] = opt.groups[0][:2] + (rate,) + opt.groups[0][3:]
        opt.step()
        if loss is not None:
            mass = hist.sum(1)
            valid = mass >= min_mass
            ce = (loss[valid] / mass[valid]).mean() if bool(valid.any()) else torch.zeros(())
            log.append((step, float(ce)))
    return log


def render_proposed(scene: Scene, prop: Proposal, rays_o, rays_d, n_out, params: RenderParams):
    """(rgb, depth, wsum, logT) of the render at proposal-placed distances
    (n_out colour samples per ray; params.n_samples is replaced by n_out).
    The proposal returns its per-bin densities and the render places the
    samples at their quantiles itself."""
    _, q = proposal_forward(scene, prop.desc, prop.params, prop.occ, rays_o, rays_d, n_out,
                            want_probs=True, want_t=False)
    p = render_params(params.tau, n_out, params.dir_mode, params.n_fresnel, tuple(params.bg),
                      n_bins=prop.desc.n_bins)
    return render_forward(scene, rays_o, rays_d, p, q)


def reduced_copy(scene: Scene, feat_dtype, probe_dtype, mlp_dtype) -> Scene:
    """The same parameters in reduced-precision storage (BF16 features,
    FP16 probes, FP16 MLP arithmetic), converted once on the device."""
    from . import grid_desc, pack_grid, unpack_grid
    gd32 = grid_desc(scene.dims, scene.box_min, scene.box_max, scene.n_feat, scene.feat_dtype)
    sdf, feat = unpack_grid(gd32, scene.grid)
    gd = grid_desc(scene.dims, scene.box_min, scene.box_max, scene.n_feat, feat_dtype)
    grid = pack_grid(gd, sdf, feat)
    probes = scene.probes.half() if probe_dtype != F32 else scene.probes.float()
    return dataclasses.replace(scene, grid=grid, probes=probes.contiguous(),
                               mlp=scene.mlp.clone(), feat_dtype=feat_dtype,
                               probe_dtype=probe_dtype, mlp_dtype=mlp_dtype)
