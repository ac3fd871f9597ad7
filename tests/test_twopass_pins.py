"""Pins of the oracle's two-pass inference (per-view node shading, then a march
over the SDF and the interpolated node colours; the paper's viewer, Tab. 8)
to the pinned per-sample oracle and to closed forms (CPU only)."""
import numpy as np
import pytest

import oracle
import synth
from test_oracle_pins import effective_points, planar_scene, rays_into_box, tiny_scene

CAM = np.array([2.1, -1.3, 1.7])


def node_index_grid(sc):
    Rx, Ry, Rz = sc.dims
    iz, iy, ix = np.meshgrid(np.arange(Rz), np.arange(Ry), np.arange(Rx), indexing="ij")
    return ix, iy, iz


def node_world(sc, ix, iy, iz):
    lo, hi = sc.box_min.astype(np.float64), sc.box_max.astype(np.float64)
    h = (hi - lo) / (np.array(sc.dims) - 1)
    return lo + np.stack([ix, iy, iz], -1) * h


def point_colour(m, x, mode):
    """Colour of the per-sample oracle at world point x, seen from CAM (the
    ray from the camera through x, evaluated at x)."""
    d = x - CAM
    t = np.linalg.norm(d)
    return oracle.point_eval(m, CAM.astype(np.float32), (d / t).astype(np.float32),
                             np.float32(t), dir_mode=mode)["C"]


@pytest.mark.parametrize("mode", [oracle.DIR_REFLECT, oracle.DIR_VIEW])
def test_node_colour_is_the_point_colour_on_a_planar_sdf(mode):
    """A linear SDF makes the node's central (and one-sided) differences the
    exact gradient, which is also the trilinear gradient at the point: so the
    node's colour is the per-sample colour at the node, faces included."""
    sc, _ = planar_scene([0.3, -0.5, 0.8], offset=-0.2)
    m = oracle.Model.from_scene(sc)
    col = oracle.shade_nodes(m, CAM, band=1e9, dir_mode=mode)
    ix, iy, iz = node_index_grid(sc)
    X = node_world(sc, ix, iy, iz)
    for idx in np.ndindex(ix.shape):
        want = point_colour(m, X[idx], mode)
        np.testing.assert_allclose(col[idx], want, rtol=0, atol=2e-6)


def test_band_leaves_far_nodes_black():
    sc = tiny_scene(R=(9, 8, 10))
    m = oracle.Model.from_scene(sc)
    band = 0.12
    col = oracle.shade_nodes(m, CAM, band)
    inside = np.abs(sc.sdf.astype(np.float64)) < band
    assert inside.any() and (~inside).any()
    assert np.all(col[~inside] == 0.0)
    assert np.all(col[inside] > 0.0) and np.all(col[inside] < 1.0)


def test_triplane_node_features_are_the_point_features():
    """Tri-plane features at a node equal the per-sample lookup at the node
    (nodes on an inner tile face are left out: F_s is discontinuous there and
    the FP32 position of the per-sample path may fall in either tile)."""
    sc, _ = planar_scene([0.2, 0.9, -0.3], offset=0.1, R=(20, 18, 35), P=(4, 4, 4))
    sc = synth.with_triplanes(sc, 12)
    m = oracle.Model.from_scene(sc)
    col = oracle.shade_nodes(m, CAM, band=1e9)
    ix, iy, iz = node_index_grid(sc)
    X = node_world(sc, ix, iy, iz)
    checked = 0
    for idx in np.ndindex(ix.shape):
        i = (ix[idx], iy[idx], iz[idx])
        if any(i[a] % 16 == 0 and 0 < i[a] < sc.dims[a] - 1 for a in range(3)):
            continue
        if checked % 7 == 0:
            np.testing.assert_allclose(col[idx], point_colour(m, X[idx], oracle.DIR_REFLECT),
                                       rtol=0, atol=2e-6)
        checked += 1
    assert checked > 1000


def test_constant_colour_field_gives_the_weight_sum():
    sc = tiny_scene(R=(12, 10, 11))
    m = oracle.Model.from_scene(sc)
    o, d = rays_into_box(64, 3)
    c = np.array([0.2, 0.55, 0.9])
    bg = (0.3, 0.1, 0.7)
    col = np.broadcast_to(c, sc.sdf.shape + (3,))
    two = oracle.render_colour_field(m, col, o, d, 64.0, 40, bg=bg)
    ref = oracle.render_forward(m, o, d, 64.0, 40, bg=bg)
    np.testing.assert_allclose(two["wsum"], ref["wsum"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(two["depth"], ref["depth"], rtol=0, atol=1e-13)
    T = 1.0 - ref["wsum"]
    np.testing.assert_allclose(two["rgb"], ref["wsum"][:, None] * c + T[:, None] * np.array(bg),
                               rtol=0, atol=1e-12)


def test_affine_colour_field_is_interpolated_exactly():
    """Node colours affine in the position: the trilinear blend gives the
    affine function at the evaluated point, so rgb = sum_k w_k (A x_k + b)."""
    sc = tiny_scene(R=(9, 12, 10))
    m = oracle.Model.from_scene(sc)
    ix, iy, iz = node_index_grid(sc)
    X = node_world(sc, ix, iy, iz)
    A = np.array([[0.3, -0.2, 0.5], [0.1, 0.4, -0.3], [-0.25, 0.15, 0.2]])
    b = np.array([0.2, 0.4, 0.6])
    col = X @ A.T + b
    o, d = rays_into_box(24, 5)
    N = 33
    two = oracle.render_colour_field(m, col, o, d, 64.0, N)
    for r in range(o.shape[0]):
        tr = oracle.render_trace(m, o[r], d[r], 64.0, N)
        if not tr["hit"]:
            assert np.all(two["rgb"][r] == 0.0)
            continue
        xk = effective_points(sc, o[r], d[r], tr["t"][:N])
        want = (tr["w"][:, None] * (xk @ A.T + b)).sum(0)
        np.testing.assert_allclose(two["rgb"][r], want, rtol=0, atol=1e-12)


def test_two_pass_equals_per_sample_render_for_a_constant_mlp():
    """Zero weights make every colour sigmoid(b3); with every node shaded the
    two passes reproduce the per-sample render."""
    sc = tiny_scene(R=(10, 9, 12))
    n_in = sc.n_s + sc.n_a + sc.n_fresnel
    W = sc.width
    sc.mlp = np.zeros_like(sc.mlp)
    sc.mlp[-3:] = (0.4, -1.1, 2.0)
    m = oracle.Model.from_scene(sc)
    assert sc.mlp.size == W * n_in + W + W * W + W + 3 * W + 3
    o, d = rays_into_box(48, 9)
    col = oracle.shade_nodes(m, CAM, band=np.inf)
    two = oracle.render_colour_field(m, col, o, d, 64.0, 50)
    ref = oracle.render_forward(m, o, d, 64.0, 50)
    for k in ("rgb", "depth", "wsum"):
        np.testing.assert_allclose(two[k], ref[k], rtol=0, atol=1e-12)


def test_node_list_matches_the_full_pass():
    sc = tiny_scene(R=(9, 8, 10))
    m = oracle.Model.from_scene(sc)
    full = oracle.shade_nodes(m, CAM, 0.2).reshape(-1, 3)
    idx = synth.rng(4).choice(full.shape[0], 60, replace=False)
    np.testing.assert_array_equal(oracle.shade_node_list(m, CAM, 0.2, idx), full[idx])
