"""FP64 oracle of the grid-level training terms of ProbeSDF (Sec. 3.3).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain numpy, one term
at a time, written from the definitions:

* smoothing: s = G(s_hat), a normalised 5^3 Gaussian (separable, 5 taps per
  axis, sigma = 1 node spacing) with replicated edge nodes (Sec. 3.3: "the raw
  SDF is convolved by a 5^3 gaussian kernel");
* L_sdf = sum_voxel |s - s_hat|^2 (Eq. 11);
* L_Eik = sum_voxel (||grad s|| - 1)^2 (Eq. 12);
* L_normal = sum_voxel ||grad n||^2, n = grad s / ||grad s|| (Eq. 13);
* L_features = sum_texel ||grad F_x||^2 + ||grad F_y||^2 + ||grad F_z||^2 (Eq. 14);
* L_probes = sum_i sum_j sum_{k in V_i} ||b_ij - b_kj||^2 (Eq. 15);
* the gradients of the per-voxel terms scaled by (1 + 5 |s|)^-1 (Sec. 3.3).

Readings where the paper is silent (each listed in the design notes):
grad s at a node is the central difference over the two neighbours (node
spacing h_a per axis), defined at interior nodes only; the Eikonal and normal
terms are summed over interior nodes; ||grad n||^2 at node i is
sum_a ||n(i + e_a) - n(i)||^2 over the axes whose neighbour is interior too;
n = g / sqrt(|g|^2 + eps^2) with eps = 1e-12; the texel gradient of a plane
is the forward difference to the next texel in each in-plane direction,
inside a tile; V_i is the 6-neighbourhood of probe i (both orders of a pair
count); the (1 + 5|s|)^-1 factor uses the smoothed s at the term's voxel and
is not differentiated.  The value of each loss is returned unweighted.
"""
from __future__ import annotations

import numpy as np

EPS_NORMAL = 1e-12
SIGMA = 1.0
TAPS = 2  # 5 taps: -2..2


def gauss_taps(sigma=SIGMA):
    k = np.arange(-TAPS, TAPS + 1, dtype=np.float64)
    w = np.exp(-0.5 * (k / sigma) ** 2)
    return w / w.sum()


def _conv_axis(a, w, axis):
    """1D convolution along `axis` with edge replication."""
    n = a.shape[axis]
    out = np.zeros_like(a)
    for j, wj in enumerate(w):
        off = j - TAPS
        idx = np.clip(np.arange(n) + off, 0, n - 1)
        out += wj * np.take(a, idx, axis=axis)
    return out


def _conv_axis_t(a, w, axis):
    """Transpose of _conv_axis (edge contributions gathered onto the edges)."""
    n = a.shape[axis]
    out = np.zeros_like(a)
    for j, wj in enumerate(w):
        off = j - TAPS
        idx = np.clip(np.arange(n) + off, 0, n - 1)
        # out[idx[i]] += w_j a[i]
        moved = np.moveaxis(out, axis, 0)
        src = np.moveaxis(a, axis, 0)
        np.add.at(moved, idx, wj * src)
    return out


def smooth(s_hat, sigma=SIGMA):
    """s = G(s_hat) for s_hat [Rz][Ry][Rx]."""
    w = gauss_taps(sigma)
    s = np.asarray(s_hat, np.float64)
    for ax in (2, 1, 0):
        s = _conv_axis(s, w, ax)
    return s


def smooth_adjoint(ds, sigma=SIGMA):
    """G^T ds."""
    w = gauss_taps(sigma)
    g = np.asarray(ds, np.float64)
    for ax in (0, 1, 2):
        g = _conv_axis_t(g, w, ax)
    return g


def voxel_weight(s):
    return 1.0 / (1.0 + 5.0 * np.abs(s))


def _interior(shape):
    m = np.zeros(shape, bool)
    m[1:-1, 1:-1, 1:-1] = True
    return m


def _central_grad(s, h):
    """Central differences [3][Rz][Ry][Rx] (x, y, z components), zero at
    boundary nodes."""
    g = np.zeros((3,) + s.shape)
    g[0][:, :, 1:-1] = (s[:, :, 2:] - s[:, :, :-2]) / (2 * h[0])
    g[1][:, 1:-1, :] = (s[:, 2:, :] - s[:, :-2, :]) / (2 * h[1])
    g[2][1:-1, :, :] = (s[2:, :, :] - s[:-2, :, :]) / (2 * h[2])
    return g


def _grad_adjoint(dg, h):
    """Adjoint of _central_grad restricted to the interior: dg [3][..] -> ds."""
    ds = np.zeros(dg.shape[1:])
    ds[:, :, 2:] += dg[0][:, :, 1:-1] / (2 * h[0])
    ds[:, :, :-2] -= dg[0][:, :, 1:-1] / (2 * h[0])
    ds[:, 2:, :] += dg[1][:, 1:-1, :] / (2 * h[1])
    ds[:, :-2, :] -= dg[1][:, 1:-1, :] / (2 * h[1])
    ds[2:, :, :] += dg[2][1:-1, :, :] / (2 * h[2])
    ds[:-2, :, :] -= dg[2][1:-1, :, :] / (2 * h[2])
    return ds


def spacing(dims, box_min, box_max):
    return np.array([(float(box_max[a]) - float(box_min[a])) / (int(dims[a]) - 1)
                     for a in range(3)])


def sdf_terms(s_hat, s, h, lam_sdf, lam_eik, lam_normal, weights=None, owner=None):
    """Per-voxel terms on the smoothed s.  Returns the three loss values, the
    weighted objective sum_i w_i (lam_sdf sdf_i + lam_eik eik_i + lam_normal
    normal_i) whose gradient the two arrays are (w.r.t. s, and w.r.t. s_hat
    directly), with w_i = (1 + 5 |s_i|)^-1 (or the given weights, held fixed).
    owner (bool, the grid's shape, default all): only the voxels it marks
    contribute their terms (their sdf_i, eik_i and the normal pairs they own);
    the others still enter those terms as neighbours (a sparse grid's absent
    nodes, whose s is fixed)."""
    s_hat = np.asarray(s_hat, np.float64)
    s = np.asarray(s, np.float64)
    wv = voxel_weight(s) if weights is None else np.asarray(weights, np.float64)
    own = np.ones(s.shape, bool) if owner is None else np.asarray(owner, bool)
    inner = _interior(s.shape)
    # L_sdf
    r = (s - s_hat) * own
    l_sdf = float(np.sum(r * r))
    objective = lam_sdf * float(np.sum(wv * r * r))
    ds = lam_sdf * wv * 2 * r
    ds_hat = -lam_sdf * wv * 2 * r
    # L_Eik on interior nodes
    g = _central_grad(s, h)
    gn = np.sqrt(np.sum(g * g, axis=0))
    e = np.where(inner & own, gn - 1.0, 0.0)
    l_eik = float(np.sum(e * e))
    objective += lam_eik * float(np.sum(wv * e * e))
    unit = g / np.maximum(gn, 1e-300)
    dg = lam_eik * (wv * 2 * e)[None] * unit * inner[None]
    # L_normal: n at interior nodes, forward pairs between interior nodes
    rho = np.sqrt(np.sum(g * g, axis=0) + EPS_NORMAL ** 2)
    n = g / rho[None]
    l_norm = 0.0
    dn = np.zeros_like(n)
    for a, sl in ((0, (slice(None), slice(None), slice(1, None))),
                  (1, (slice(None), slice(1, None), slice(None))),
                  (2, (slice(1, None), slice(None), slice(None)))):
        # pair (i, i + e_a) owned by voxel i
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[2 - a] = slice(0, -1)
        hi[2 - a] = slice(1, None)
        lo, hi = tuple(lo), tuple(hi)
        both = inner[lo] & inner[hi] & own[lo]
        diff = (n[(slice(None),) + hi] - n[(slice(None),) + lo]) * both[None]
        l_norm += float(np.sum(diff * diff))
        objective += lam_normal * float(np.sum(wv[lo] * np.sum(diff * diff, axis=0)))
        wpair = (lam_normal * wv[lo] * 2)[None] * diff
        dn[(slice(None),) + hi] += wpair
        dn[(slice(None),) + lo] -= wpair
    # through n = g / rho: dg += (dn - n (n . dn)) / rho
    ndn = np.sum(n * dn, axis=0)
    dg += (dn - n * ndn[None]) / rho[None] * inner[None]
    ds += _grad_adjoint(dg, h)
    return {"sdf": l_sdf, "eik": l_eik, "normal": l_norm, "objective": objective}, ds, ds_hat


def plane_terms(planes, lam):
    """L_features over tile planes [tz][ty][tx][3][16][16][n_s]: forward
    differences inside each plane.  Returns (value, gradient)."""
    P = np.asarray(planes, np.float64)
    g = np.zeros_like(P)
    val = 0.0
    dr = P[..., 1:, :, :] - P[..., :-1, :, :]   # along rows
    dc = P[..., :, 1:, :] - P[..., :, :-1, :]   # along columns
    val = float(np.sum(dr * dr) + np.sum(dc * dc))
    g[..., 1:, :, :] += 2 * lam * dr
    g[..., :-1, :, :] -= 2 * lam * dr
    g[..., :, 1:, :] += 2 * lam * dc
    g[..., :, :-1, :] -= 2 * lam * dc
    return val, g


def probe_terms(probes, lam):
    """L_probes over [Pz][Py][Px][l^2][n_a]: every ordered pair of
    6-neighbours.  Returns (value, gradient)."""
    b = np.asarray(probes, np.float64)
    g = np.zeros_like(b)
    val = 0.0
    for ax in (0, 1, 2):
        d = np.diff(b, axis=ax)
        val += 2.0 * float(np.sum(d * d))  # (i, k) and (k, i)
        lo = [slice(None)] * b.ndim
        hi = [slice(None)] * b.ndim
        lo[ax] = slice(0, -1)
        hi[ax] = slice(1, None)
        g[tuple(hi)] += 4 * lam * d
        g[tuple(lo)] -= 4 * lam * d
    return val, g
