"""Seeded synthetic inputs for the ProbeSDF render: scenes, cameras, rays,
parameters and targets.

This module holds no arithmetic of the method itself (no interpolation,
spherical harmonics, MLP or compositing): it only builds inputs.  Both the
CUDA path and the FP64 oracle read the arrays it returns, so they see the
identical FP32 bytes.

Workload recipes (shapes of the paper's object- and human-capture setups,
ProbeSDF Sec. 5; no dataset content is used):

* ``sphere64``   64^3 grid on [0,1]^3, SDF of a radius-0.5 sphere plus N(0,0.01)
  noise, 3 features/node ~N(0,0.1), probes 16^3 x 9 SH x 4 ch ~N(0,0.1), MLP
  10->16->16->3 Xavier-uniform with zero biases, 8 pinhole cameras on a
  radius-2 sphere, 128x128 px, 512 random pixels each (4096 rays), 128 samples.
* ``object256``  256^3 grid on [0,1]^3, smooth-min union of 32 random spheres and
  superquadrics, probes 32^3 x 9 x 4, MLP 10->32->32->3, 49 cameras at
  1600x1200 on a radius-2 hemisphere, 2^18 random pixels, 256 samples.
* ``human384``   384x768x384 grid on [0,1]x[0,2]x[0,1], a posed chain of 15
  capsules, probes 48x96x48 x 9 x 4, 64 cameras at 2048^2 on a ring, 2^19
  rays, 256 samples.
* ``stress512``  512^3 object-style grid, probes 64^3 x 9 x 8, MLP
  14->32->32->3, 2^20 rays, 512 samples.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


def rng(seed: int) -> np.random.Generator:
    """Counter-based generator (Philox) so every recipe is reproducible."""
    return np.random.Generator(np.random.Philox(int(seed)))


@dataclasses.dataclass
class Scene:
    sdf: np.ndarray          # float32 [Rz, Ry, Rx]
    feat: np.ndarray         # float32 [Rz, Ry, Rx, n_s]
    probes: np.ndarray       # float32 [Pz, Py, Px, l*l, n_a]
    mlp: np.ndarray          # float32 flat: W1[W][n_in] b1 W2[W][W] b2 W3[3][W] b3
    box_min: np.ndarray      # float32 [3]
    box_max: np.ndarray      # float32 [3]
    sh_l: int
    width: int
    n_fresnel: int
    planes: np.ndarray | None = None  # float32 [tz][ty][tx][3][16][16][n_s] (tile tri-planes)

    @property
    def dims(self):
        Rz, Ry, Rx = self.sdf.shape
        return (Rx, Ry, Rz)

    @property
    def probe_dims(self):
        Pz, Py, Px = self.probes.shape[:3]
        return (Px, Py, Pz)

    @property
    def n_s(self):
        return self.feat.shape[-1] if self.planes is None else self.planes.shape[-1]

    @property
    def n_a(self):
        return self.probes.shape[-1]


@dataclasses.dataclass
class Rays:
    o: np.ndarray            # float32 [n, 3]
    d: np.ndarray            # float32 [n, 3], unit length
    target: np.ndarray       # float32 [n, 3] in [0, 1]


# ----------------------------------------------------------------------------
# Parameters
# ----------------------------------------------------------------------------

def mlp_params(n_in: int, width: int, g: np.random.Generator, n_out: int = 3) -> np.ndarray:
    """Xavier-uniform weights, zero biases, packed W1 b1 W2 b2 W3 b3."""
    def xavier(fo, fi):
        a = math.sqrt(6.0 / (fi + fo))
        return g.uniform(-a, a, size=(fo, fi))
    parts = [xavier(width, n_in).ravel(), np.zeros(width),
             xavier(width, width).ravel(), np.zeros(width),
             xavier(n_out, width).ravel(), np.zeros(n_out)]
    return np.concatenate(parts).astype(np.float32)


def mlp_param_count(n_in: int, width: int, n_out: int = 3) -> int:
    return width * n_in + width + width * width + width + n_out * width + n_out


# ----------------------------------------------------------------------------
# Scene SDFs (scene construction only)
# ----------------------------------------------------------------------------

def _node_coords(dims, box_min, box_max, zslice):
    Rx, Ry, Rz = dims
    xs = np.linspace(box_min[0], box_max[0], Rx)
    ys = np.linspace(box_min[1], box_max[1], Ry)
    zs = np.linspace(box_min[2], box_max[2], Rz)[zslice]
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    return X, Y, Z


def _smin(a, b, k):
    h = np.maximum(k - np.abs(a - b), 0.0) / k
    return np.minimum(a, b) - h * h * k * 0.25


def sphere_sdf(dims, box_min, box_max, center, radius):
    X, Y, Z = _node_coords(dims, box_min, box_max, slice(None))
    return np.sqrt((X - center[0]) ** 2 + (Y - center[1]) ** 2 + (Z - center[2]) ** 2) - radius


def _random_rotation(g):
    q = g.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                     [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                     [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])


def object_shapes(g, n_shapes=32):
    shapes = []
    for i in range(n_shapes):
        c = g.uniform(0.25, 0.75, size=3)
        if i % 2 == 0:
            shapes.append(("sphere", c, g.uniform(0.05, 0.2)))
        else:
            radii = g.uniform(0.04, 0.16, size=3)
            expo = g.uniform(1.5, 6.0)
            shapes.append(("superquadric", c, (radii, expo, _random_rotation(g))))
    return shapes


def _torch_coords(dims, box_min, box_max, z0, z1):
    import torch
    Rx, Ry, Rz = dims
    xs = torch.linspace(float(box_min[0]), float(box_max[0]), Rx, dtype=torch.float64)
    ys = torch.linspace(float(box_min[1]), float(box_max[1]), Ry, dtype=torch.float64)
    zs = torch.linspace(float(box_min[2]), float(box_max[2]), Rz, dtype=torch.float64)[z0:z1]
    Z, Y, X = torch.meshgrid(zs, ys, xs, indexing="ij")
    return torch.stack([X, Y, Z], -1)


def _torch_smin(a, b, k):
    import torch
    h = torch.clamp(k - (a - b).abs(), min=0.0) / k
    return torch.minimum(a, b) - h * h * k * 0.25


def _object_dist(P, shapes, k=0.05):
    """Smooth-min union distance at points P [..., 3] (torch FP64)."""
    import torch
    acc = None
    for kind, c, prm in shapes:
        q = P - torch.as_tensor(c, dtype=torch.float64, device=P.device)
        if kind == "sphere":
            dist = q.norm(dim=-1) - prm
        else:
            radii, e, Rm = prm
            ql = (q @ torch.as_tensor(Rm, dtype=torch.float64, device=P.device)) / \
                torch.as_tensor(radii, device=P.device)
            f = ql.abs().pow(e).sum(-1).pow(1.0 / e)
            dist = (f - 1.0) * float(radii.min())
        acc = dist if acc is None else _torch_smin(acc, dist, k)
    return acc


def object_sdf(dims, box_min, box_max, shapes, k=0.05, slab=16):
    """Smooth-min (polynomial, k) union of spheres and superquadrics.  The
    superquadric uses the usual implicit-function distance approximation.
    Evaluated with torch on the host (multithreaded), FP64, stored FP32."""
    Rx, Ry, Rz = dims
    out = np.empty((Rz, Ry, Rx), np.float32)
    for z0 in range(0, Rz, slab):
        z1 = min(Rz, z0 + slab)
        P = _torch_coords(dims, box_min, box_max, z0, z1)
        out[z0:z1] = _object_dist(P, shapes, k).numpy().astype(np.float32)
    return out


def capsule_body(g):
    """A 15-capsule articulated figure in a seeded random pose, in a
    [0,1] x [0,2] x [0,1] box (y up)."""
    def rot(axis, ang):
        axis = np.asarray(axis, float)
        axis /= np.linalg.norm(axis)
        K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
        return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K

    def jitter(scale=0.35):
        return rot(g.normal(size=3), g.uniform(-scale, scale))

    caps = []
    pelvis = np.array([0.5, 0.95, 0.5]) + g.uniform(-0.03, 0.03, size=3)
    up = np.array([0.0, 1.0, 0.0])
    chest = pelvis + jitter(0.2) @ up * 0.45
    caps.append((pelvis, chest, 0.13))
    neck = chest + jitter(0.2) @ up * 0.12
    caps.append((chest, neck, 0.05))
    head = neck + jitter(0.3) @ up * 0.14
    caps.append((neck + up * 0.03, head, 0.085))
    for side in (-1.0, 1.0):
        sh = chest + np.array([0.17 * side, -0.04, 0.0])
        caps.append((chest, sh, 0.06))
        elbow = sh + jitter(0.8) @ np.array([0.12 * side, -0.25, 0.0])
        caps.append((sh, elbow, 0.045))
        wrist = elbow + jitter(0.8) @ np.array([0.05 * side, -0.24, 0.05])
        caps.append((elbow, wrist, 0.038))
        hip = pelvis + np.array([0.09 * side, -0.03, 0.0])
        knee = hip + jitter(0.4) @ np.array([0.0, -0.42, 0.03])
        caps.append((hip, knee, 0.07))
        ankle = knee + jitter(0.4) @ np.array([0.0, -0.40, -0.03])
        caps.append((knee, ankle, 0.055))
    caps.append((pelvis + np.array([-0.1, 0.0, 0.0]), pelvis + np.array([0.1, 0.0, 0.0]), 0.11))
    caps.append((chest + np.array([-0.13, -0.03, 0.0]), chest + np.array([0.13, -0.03, 0.0]), 0.09))
    assert len(caps) == 15
    return caps


def capsule_sdf(dims, box_min, box_max, caps, k=0.04, slab=16):
    import torch
    Rx, Ry, Rz = dims
    out = np.empty((Rz, Ry, Rx), np.float32)
    for z0 in range(0, Rz, slab):
        z1 = min(Rz, z0 + slab)
        P = _torch_coords(dims, box_min, box_max, z0, z1)
        acc = None
        for a, b, rad in caps:
            a_ = torch.as_tensor(a, dtype=torch.float64)
            ab = torch.as_tensor(b - a, dtype=torch.float64)
            h = torch.clamp(((P - a_) @ ab) / float(ab @ ab), 0.0, 1.0)
            q = P - a_ - h[..., None] * ab
            dist = q.norm(dim=-1) - rad
            acc = dist if acc is None else _torch_smin(acc, dist, k)
        out[z0:z1] = acc.numpy().astype(np.float32)
    return out


# ----------------------------------------------------------------------------
# Cameras and rays
# ----------------------------------------------------------------------------

def fibonacci_sphere(n, hemisphere=False):
    i = np.arange(n) + 0.5
    z = 1.0 - i / n if hemisphere else 1.0 - 2.0 * i / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = math.pi * (3.0 - math.sqrt(5.0)) * i
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], -1)


def look_at_cameras(positions, target, up=(0.0, 0.0, 1.0)):
    cams = []
    up = np.asarray(up, float)
    for p in positions:
        fwd = target - p
        fwd /= np.linalg.norm(fwd)
        u = up if abs(fwd @ up) < 0.99 else np.array([1.0, 0.0, 0.0])
        right = np.cross(fwd, u)
        right /= np.linalg.norm(right)
        cup = np.cross(right, fwd)
        cams.append((np.asarray(p, float), fwd, right, cup))
    return cams


def pixel_rays(cams, width, height, fov_deg, n_rays, g, per_camera=None):
    """Random pixel rays: uniform camera choice (or a fixed count per camera),
    uniform pixel; origins at the camera centre, FP64 unit directions rounded
    to FP32."""
    tan_half = math.tan(math.radians(fov_deg) * 0.5)
    aspect = width / height
    if per_camera is not None:
        cam_idx = np.repeat(np.arange(len(cams)), per_camera)
    else:
        cam_idx = g.integers(0, len(cams), size=n_rays)
    px = g.integers(0, width, size=cam_idx.size)
    py = g.integers(0, height, size=cam_idx.size)
    o = np.empty((cam_idx.size, 3))
    d = np.empty((cam_idx.size, 3))
    for ci, (p, fwd, right, cup) in enumerate(cams):
        sel = cam_idx == ci
        sx = (2.0 * (px[sel] + 0.5) / width - 1.0) * tan_half * aspect
        sy = (1.0 - 2.0 * (py[sel] + 0.5) / height) * tan_half
        dd = fwd[None] + sx[:, None] * right[None] + sy[:, None] * cup[None]
        dd /= np.linalg.norm(dd, axis=1, keepdims=True)
        o[sel] = p
        d[sel] = dd
    return o.astype(np.float32), d.astype(np.float32)


def image_rays(cam, width, height, fov_deg):
    """Every pixel of one camera, row-major."""
    p, fwd, right, cup = cam
    tan_half = math.tan(math.radians(fov_deg) * 0.5)
    aspect = width / height
    jj, ii = np.meshgrid(np.arange(height), np.arange(width), indexing="ij")
    sx = (2.0 * (ii + 0.5) / width - 1.0) * tan_half * aspect
    sy = (1.0 - 2.0 * (jj + 0.5) / height) * tan_half
    dd = fwd + sx[..., None] * right + sy[..., None] * cup
    dd /= np.linalg.norm(dd, axis=-1, keepdims=True)
    o = np.broadcast_to(p, dd.shape)
    return (np.ascontiguousarray(o.reshape(-1, 3), dtype=np.float32),
            np.ascontiguousarray(dd.reshape(-1, 3), dtype=np.float32))


# ----------------------------------------------------------------------------
# Recipes
# ----------------------------------------------------------------------------

WORKLOADS = {
    "sphere64": dict(seed=1235, R=(64, 64, 64), P=(16, 16, 16), box=((0, 0, 0), (1, 1, 1)),
                     n_s=3, n_a=4, sh_l=3, width=16, K=3, n_samples=128, tau=64.0,
                     n_rays=4096, cams=8, res=(128, 128), fov=50.0, cam_r=2.0),
    "object256": dict(seed=1236, R=(256, 256, 256), P=(32, 32, 32), box=((0, 0, 0), (1, 1, 1)),
                      n_s=3, n_a=4, sh_l=3, width=32, K=3, n_samples=256, tau=64.0,
                      n_rays=1 << 18, cams=49, res=(1600, 1200), fov=45.0, cam_r=2.0),
    "human384": dict(seed=1237, R=(384, 768, 384), P=(48, 96, 48), box=((0, 0, 0), (1, 2, 1)),
                     n_s=3, n_a=4, sh_l=3, width=32, K=3, n_samples=256, tau=64.0,
                     n_rays=1 << 19, cams=64, res=(2048, 2048), fov=45.0, cam_r=2.5),
    "stress512": dict(seed=1239, R=(512, 512, 512), P=(64, 64, 64), box=((0, 0, 0), (1, 1, 1)),
                      n_s=3, n_a=8, sh_l=3, width=32, K=3, n_samples=512, tau=64.0,
                      n_rays=1 << 20, cams=49, res=(1600, 1200), fov=45.0, cam_r=2.0),
}


def _make_scene_arrays(name, g, spec, dims=None, probe_dims=None):
    dims = tuple(dims or spec["R"])
    probe_dims = tuple(probe_dims or spec["P"])
    bmin = np.array(spec["box"][0], np.float64)
    bmax = np.array(spec["box"][1], np.float64)
    Rx, Ry, Rz = dims
    if name == "sphere64":
        sdf = sphere_sdf(dims, bmin, bmax, (0.5, 0.5, 0.5), 0.5)
        sdf = sdf + g.normal(0.0, 0.01, size=sdf.shape)
    elif name in ("object256", "stress512"):
        sdf = object_sdf(dims, bmin, bmax, object_shapes(g, 32))
    elif name == "human384":
        sdf = capsule_sdf(dims, bmin, bmax, capsule_body(g))
    else:
        raise KeyError(name)
    sdf = sdf.astype(np.float32)
    feat = g.normal(0.0, 0.1, size=(Rz, Ry, Rx, spec["n_s"])).astype(np.float32)
    Px, Py, Pz = probe_dims
    probes = g.normal(0.0, 0.1, size=(Pz, Py, Px, spec["sh_l"] ** 2, spec["n_a"]))
    n_in = spec["n_s"] + spec["n_a"] + spec["K"]
    mlp = mlp_params(n_in, spec["width"], g)
    return Scene(sdf=sdf, feat=feat, probes=probes.astype(np.float32), mlp=mlp,
                 box_min=bmin.astype(np.float32), box_max=bmax.astype(np.float32),
                 sh_l=spec["sh_l"], width=spec["width"], n_fresnel=spec["K"])


def sparse_object(R, band, seed=1240, probe_every=16, n_s=3, n_a=4, sh_l=3, width=32, K=3,
                  chunk=1 << 21, device="cpu"):
    """An object-capture scene (smooth-min union of 16 spheres and 16
    superquadrics, as object256) sampled on an R^3 node grid over [0,1]^3 and
    stored sparsely: only the 16^3-node bricks that come within `band` of the
    surface.  The bricks are chosen from the SDF at the brick's nodes on a
    4x coarser lattice, widened by that lattice's half diagonal.  Returns
    (keep [Bz,By,Bx] bool, brick SDF [n,16,16,16] FP32, brick features
    [n,16,16,16,n_s] FP32, probes [P,P,P,l*l,n_a], MLP parameters), bricks in
    x-fastest brick order and nodes x fastest inside a brick.  `device` is
    where torch evaluates the shapes (FP64)."""
    import torch
    g = rng(seed)
    shapes = object_shapes(g, 32)
    B = R // 16
    h = 1.0 / (R - 1)
    # coarse test: every 4th node of every brick (5 per axis incl. the far face)
    lo = torch.arange(B, dtype=torch.float64) * 16 * h
    off = torch.arange(5, dtype=torch.float64) * 4 * h
    keep = np.zeros((B, B, B), bool)
    for bz in range(B):
        zs = (lo[bz] + off).clamp(max=1.0)
        ys = (lo[:, None] + off[None]).clamp(max=1.0)          # [B, 5]
        xs = (lo[:, None] + off[None]).clamp(max=1.0)
        Z = zs[None, None, :, None, None].expand(B, B, 5, 5, 5)
        Y = ys[:, None, None, :, None].expand(B, B, 5, 5, 5)
        X = xs[None, :, None, None, :].expand(B, B, 5, 5, 5)
        P = torch.stack([X, Y, Z], -1).to(device)               # [by, bx, z, y, x, 3]
        d = _object_dist(P, shapes).abs().amin(dim=(2, 3, 4))
        keep[bz] = (d < band + 2.0 * 3 ** 0.5 * h * 2).cpu().numpy()
    idx = np.argwhere(keep)                                     # (bz, by, bx), x fastest
    n = idx.shape[0]
    local = torch.arange(16, dtype=torch.float64) * h
    Z, Y, X = torch.meshgrid(local, local, local, indexing="ij")
    base = torch.stack([X, Y, Z], -1).reshape(-1, 3).to(device)  # [4096, 3]
    sdf = np.empty((n, 16, 16, 16), np.float32)
    per = max(1, chunk // 4096)
    corner = torch.as_tensor(idx[:, ::-1].copy() * 16 * h, dtype=torch.float64,
                             device=device)                     # brick origins (x, y, z)
    for i in range(0, n, per):
        P = corner[i:i + per, None, :] + base[None]
        sdf[i:i + per] = _object_dist(P, shapes).reshape(-1, 16, 16, 16).cpu().numpy()
    feat = g.normal(0.0, 0.1, size=(n, 16, 16, 16, n_s)).astype(np.float32)
    Pn = (R - 1) // probe_every + 1
    probes = g.normal(0.0, 0.1, size=(Pn, Pn, Pn, sh_l * sh_l, n_a)).astype(np.float32)
    mlp = mlp_params(n_s + n_a + K, width, g)
    return keep, sdf, feat, probes, mlp


def smooth_features(dims, n_s, g: np.random.Generator, sigma_vox=3.0, std=0.1) -> np.ndarray:
    """Spatial features [Rz,Ry,Rx,n_s] drawn as white noise filtered by a
    Gaussian of sigma_vox nodes (in Fourier space, periodic) and rescaled to
    the given standard deviation: features that vary over a few voxels, like
    those of a scene trained with a smoothness term, instead of per-node
    noise."""
    Rx, Ry, Rz = (int(v) for v in dims)
    out = np.empty((Rz, Ry, Rx, n_s), np.float32)
    kz = np.fft.fftfreq(Rz)[:, None, None]
    ky = np.fft.fftfreq(Ry)[None, :, None]
    kx = np.fft.rfftfreq(Rx)[None, None, :]
    filt = np.exp(-2.0 * (np.pi * sigma_vox) ** 2 * (kx ** 2 + ky ** 2 + kz ** 2))
    for c in range(n_s):
        f = np.fft.irfftn(np.fft.rfftn(g.normal(size=(Rz, Ry, Rx))) * filt, s=(Rz, Ry, Rx),
                          axes=(0, 1, 2))
        out[..., c] = (f * (std / f.std())).astype(np.float32)
    return out


def inference_scene(name: str) -> Scene:
    """The workload's scene with smooth spatial features (the starting point of
    the real-time inference workload's appearance fit)."""
    sc = make_scene(name)
    spec = WORKLOADS[name]
    return dataclasses.replace(sc, feat=smooth_features(sc.dims, spec["n_s"],
                                                        rng(spec["seed"] + 29)))


def make_scene(name: str, dims=None, probe_dims=None) -> Scene:
    spec = WORKLOADS[name]
    return _make_scene_arrays(name, rng(spec["seed"]), spec, dims, probe_dims)


def make_rays(name: str, n_rays: int | None = None, seed_offset: int = 0) -> Rays:
    spec = WORKLOADS[name]
    g = rng(spec["seed"] * 7919 + 17 + seed_offset)
    n = int(n_rays if n_rays is not None else spec["n_rays"])
    bmin = np.array(spec["box"][0], float)
    bmax = np.array(spec["box"][1], float)
    center = 0.5 * (bmin + bmax)
    W, H = spec["res"]
    if name == "human384":
        ang = 2 * math.pi * (np.arange(spec["cams"]) + 0.5) / spec["cams"]
        pos = np.stack([center[0] + spec["cam_r"] * np.cos(ang),
                        np.full_like(ang, center[1]),
                        center[2] + spec["cam_r"] * np.sin(ang)], -1)
        cams = look_at_cameras(pos, center, up=(0.0, 1.0, 0.0))
    else:
        hemi = name != "sphere64"
        pos = center + spec["cam_r"] * fibonacci_sphere(spec["cams"], hemisphere=hemi)
        cams = look_at_cameras(pos, center)
    if name == "sphere64" and n_rays is None:
        o, d = pixel_rays(cams, W, H, spec["fov"], n, g, per_camera=n // spec["cams"])
    else:
        o, d = pixel_rays(cams, W, H, spec["fov"], n, g)
    target = g.uniform(0.0, 1.0, size=(o.shape[0], 3)).astype(np.float32)
    return Rays(o=o, d=d, target=target)


def random_unit_vectors(n, g):
    v = g.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def proposal_params(g: np.random.Generator, width: int = 32, n_bins: int = 8) -> np.ndarray:
    """Xavier-uniform initial parameters of the proposal MLP (7 + 2B -> W -> W -> B)."""
    return mlp_params(7 + 2 * n_bins, width, g, n_out=n_bins)


# ----------------------------------------------------------------------------
# Teacher images and novel views (appearance fitting and the inference test)
# ----------------------------------------------------------------------------

def workload_shapes(name: str):
    """The procedural shapes of an object-style workload (the first draws of
    its scene generator)."""
    spec = WORKLOADS[name]
    if name not in ("object256", "stress512"):
        raise KeyError(f"{name} has no object shapes")
    return object_shapes(rng(spec["seed"]), 32)


_ALBEDO_FREQ = np.array([[3.1, -1.7, 2.3], [-2.2, 2.9, 1.3], [1.4, 2.1, -3.3]])
_ALBEDO_PHASE = np.array([0.3, 1.9, 4.1])
_LIGHT = np.array([0.48, 0.36, 0.8]) / np.linalg.norm([0.48, 0.36, 0.8])


def teacher_colors(name: str, rays_o, rays_d, max_iter=160, chunk=1 << 16):
    """Teacher RGB of each ray: the first hit of the workload's analytic SDF
    (sphere tracing at 0.8 of the distance, inside the box), shaded by a
    procedural 3D albedo x (ambient + Lambert) plus a white Phong lobe; rays
    that miss get 0 (the render's black background).  FP64 on the host."""
    import torch
    spec = WORKLOADS[name]
    shapes = workload_shapes(name)
    bmin = np.array(spec["box"][0], float)
    bmax = np.array(spec["box"][1], float)
    o_all = np.asarray(rays_o, np.float64).reshape(-1, 3)
    d_all = np.asarray(rays_d, np.float64).reshape(-1, 3)
    out = np.zeros((o_all.shape[0], 3))
    for c0 in range(0, o_all.shape[0], chunk):
        o = o_all[c0:c0 + chunk]
        d = d_all[c0:c0 + chunk]
        with np.errstate(divide="ignore", invalid="ignore"):
            inv = 1.0 / d
            t0 = (bmin - o) * inv
            t1 = (bmax - o) * inv
        tn = np.maximum(np.nanmax(np.minimum(t0, t1), axis=1), 0.0)
        tf = np.nanmin(np.maximum(t0, t1), axis=1)
        t = tn.copy()
        active = tf > tn
        hit = np.zeros(o.shape[0], bool)
        for _ in range(max_iter):
            idx = np.nonzero(active)[0]
            if idx.size == 0:
                break
            P = torch.as_tensor(o[idx] + t[idx, None] * d[idx])
            s = _object_dist(P, shapes).numpy()
            done = s < 1e-5
            hit[idx[done]] = True
            t[idx] += np.where(done, 0.0, 0.8 * np.maximum(s, 1e-5))
            active[idx[done]] = False
            active[idx[t[idx] > tf[idx]]] = False
        idx = np.nonzero(hit)[0]
        if idx.size == 0:
            continue
        x = o[idx] + t[idx, None] * d[idx]
        h = 1e-5
        n = np.zeros_like(x)
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            n[:, a] = (_object_dist(torch.as_tensor(x + e), shapes).numpy() -
                       _object_dist(torch.as_tensor(x - e), shapes).numpy())
        n /= np.maximum(np.linalg.norm(n, axis=1, keepdims=True), 1e-12)
        albedo = 0.5 + 0.4 * np.sin(2 * math.pi * x @ _ALBEDO_FREQ.T + _ALBEDO_PHASE)
        lam = np.maximum(n @ _LIGHT, 0.0)
        v = -d[idx]
        r = 2 * np.sum(n * v, 1, keepdims=True) * n - v
        spec_ = 0.25 * np.maximum(r @ _LIGHT, 0.0) ** 16
        out[c0 + idx] = np.clip(albedo * (0.25 + 0.75 * lam[:, None]) + spec_[:, None], 0.0, 1.0)
    return out.astype(np.float32)


def novel_cameras(name: str, n_views: int = 8):
    """Views off the training rig: a ring at 30 degrees elevation, radius
    1.15x the training radius, rotated half a step from the training
    azimuths."""
    spec = WORKLOADS[name]
    bmin = np.array(spec["box"][0], float)
    bmax = np.array(spec["box"][1], float)
    center = 0.5 * (bmin + bmax)
    r = 1.15 * spec["cam_r"]
    el = math.radians(30.0)
    az = 2 * math.pi * (np.arange(n_views) + 0.37) / n_views
    pos = center + r * np.stack([math.cos(el) * np.cos(az), math.cos(el) * np.sin(az),
                                 np.full(n_views, math.sin(el))], -1)
    return look_at_cameras(pos, center)


def training_pool(name: str, n_rays: int, seed_offset: int = 0):
    """Random pixel rays of the workload's training cameras with their
    teacher colours (Rays with target = teacher RGB)."""
    r = make_rays(name, n_rays=n_rays, seed_offset=seed_offset)
    return Rays(o=r.o, d=r.d, target=teacher_colors(name, r.o, r.d))


TILE = 16


def tile_planes(dims, n_s, g: np.random.Generator, mean=1.0, std=0.3) -> np.ndarray:
    """Seeded tile tri-planes [tz][ty][tx][3][16][16][n_s] for a grid of `dims`
    nodes (16^3-cell tiles): N(mean, std) texels, so that the product of the
    three lookups stays of order one."""
    nt = [(int(r) - 1 + TILE - 1) // TILE for r in dims]
    return g.normal(mean, std, size=(nt[2], nt[1], nt[0], 3, TILE, TILE, n_s)).astype(np.float32)


def with_triplanes(sc: Scene, seed: int, **kw) -> Scene:
    """The scene with tile tri-plane spatial features instead of node features."""
    return dataclasses.replace(sc, planes=tile_planes(sc.dims, sc.feat.shape[-1], rng(seed), **kw),
                               feat=np.zeros(sc.feat.shape[:-1] + (0,), np.float32))
