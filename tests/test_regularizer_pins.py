"""Pins of the oracle's grid-level training terms (Sec. 3.3, Eqs. 11-15):
closed forms, invariants, the adjoint identity and central differences."""
import numpy as np
import pytest

import synth
from oracle import regularizers as R


def _field(shape, seed):
    return synth.rng(seed).normal(size=shape)


def test_gaussian_taps_normalised_and_symmetric():
    w = R.gauss_taps()
    assert w.shape == (5,) and abs(w.sum() - 1) < 1e-15
    np.testing.assert_allclose(w, w[::-1], rtol=0, atol=0)
    np.testing.assert_allclose(w[1] / w[2], np.exp(-0.5), rtol=1e-15)


def test_smoothing_keeps_constants_and_interior_linear_fields():
    s = np.full((9, 10, 11), 2.5)
    np.testing.assert_allclose(R.smooth(s), 2.5, rtol=1e-15)
    z, y, x = np.meshgrid(np.arange(9.0), np.arange(10.0), np.arange(11.0), indexing="ij")
    lin = 0.3 * x - 1.2 * y + 0.7 * z + 4.0
    out = R.smooth(lin)
    inner = (slice(2, -2),) * 3  # two nodes from every face: no edge replication involved
    np.testing.assert_allclose(out[inner], lin[inner], atol=1e-12)


def test_smoothing_adjoint_identity():
    x = _field((7, 9, 8), 1)
    y = _field((7, 9, 8), 2)
    lhs = np.sum(R.smooth(x) * y)
    rhs = np.sum(x * R.smooth_adjoint(y))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_eikonal_and_normal_terms_vanish_on_a_plane_sdf():
    dims, bmin, bmax = (12, 10, 9), (0.0, 0.0, 0.0), (1.1, 0.9, 0.8)
    h = R.spacing(dims, bmin, bmax)
    z, y, x = np.meshgrid(*(np.arange(dims[a]) * h[a] for a in (2, 1, 0)), indexing="ij")
    nvec = np.array([0.48, -0.6, 0.64])  # unit
    s = nvec[0] * x + nvec[1] * y + nvec[2] * z - 0.3
    vals, ds, _ = R.sdf_terms(s, s, h, 0.0, 1.0, 1.0)
    assert vals["eik"] < 1e-24 and vals["normal"] < 1e-24
    assert np.abs(ds).max() < 1e-10


def test_eikonal_of_a_scaled_plane():
    dims = (8, 8, 8)
    h = R.spacing(dims, (0, 0, 0), (1, 1, 1))
    x = np.broadcast_to(np.arange(8) * h[0], (8, 8, 8))
    vals, _, _ = R.sdf_terms(2.0 * x, 2.0 * x, h, 0.0, 1.0, 0.0)
    # |grad s| = 2 at the 6^3 interior nodes
    assert abs(vals["eik"] - 6 ** 3 * 1.0) < 1e-9


def test_normal_term_positive_on_a_sphere():
    dims = (16, 16, 16)
    h = R.spacing(dims, (0, 0, 0), (1, 1, 1))
    s = synth.sphere_sdf(dims, np.zeros(3), np.ones(3), (0.5, 0.5, 0.5), 0.3)
    vals, _, _ = R.sdf_terms(s, s, h, 0.0, 0.0, 1.0)
    assert vals["normal"] > 1e-3


def test_probe_term_hand_example_and_constants():
    b = np.zeros((1, 1, 2, 9, 4))
    b[0, 0, 1] = 1.0
    val, g = R.probe_terms(b, 1.0)
    assert val == 2 * 36  # two ordered pairs, 36 coefficients differing by 1
    np.testing.assert_allclose(g[0, 0, 0], -4.0)
    np.testing.assert_allclose(g[0, 0, 1], 4.0)
    val, g = R.probe_terms(np.full((3, 4, 5, 9, 4), 0.7), 1.0)
    assert val == 0 and np.abs(g).max() == 0


def test_plane_term_linear_texels():
    P = np.zeros((1, 1, 2, 3, 16, 16, 3))
    P[...] = 0.25 * np.arange(16)[None, :, None]  # slope along columns only
    val, _ = R.plane_terms(P, 1.0)
    # 2 tiles x 3 planes x 16 rows x 15 column pairs x 3 channels, each (0.25)^2
    assert abs(val - 2 * 3 * 16 * 15 * 3 * 0.0625) < 1e-12


@pytest.mark.parametrize("which", ["sdf", "eik", "normal"])
def test_sdf_terms_gradient_central_differences(which):
    dims = (9, 8, 10)
    h = R.spacing(dims, (0, 0, 0), (1.0, 0.9, 1.2))
    s_hat = synth.sphere_sdf(dims, np.zeros(3), np.array([1.0, 0.9, 1.2]), (0.5, 0.45, 0.6), 0.3)
    s_hat = s_hat + 0.02 * _field(s_hat.shape, 3)
    s = R.smooth(s_hat)
    lam = {"sdf": (1.0, 0, 0), "eik": (0, 1.0, 0), "normal": (0, 0, 1.0)}[which]
    w = R.voxel_weight(s)  # held fixed, as the method scales the gradients
    _, ds, ds_hat = R.sdf_terms(s_hat, s, h, *lam, weights=w)
    g = synth.rng(4)
    eps = 1e-6
    for arr, grad in ((s, ds), (s_hat, ds_hat)):
        flat, gflat = arr.reshape(-1), grad.reshape(-1)
        for i in g.choice(flat.size, 60, replace=False):
            old = flat[i]
            flat[i] = old + eps
            lp = R.sdf_terms(s_hat, s, h, *lam, weights=w)[0]["objective"]
            flat[i] = old - eps
            lm = R.sdf_terms(s_hat, s, h, *lam, weights=w)[0]["objective"]
            flat[i] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - gflat[i]) <= 1e-6 * max(1.0, abs(gflat).max()), (which, i, fd, gflat[i])


@pytest.mark.parametrize("which", ["sdf", "eik", "normal"])
def test_owned_sdf_terms_gradient_central_differences(which):
    """The terms of a subset of owner voxels (a sparse grid's stored nodes):
    gradients against central differences of the owned objective, everywhere
    (unowned voxels enter as neighbours); with every voxel an owner the result
    is the unrestricted one; owned and unowned terms add up to the whole."""
    dims = (9, 8, 10)
    h = R.spacing(dims, (0, 0, 0), (1.0, 0.9, 1.2))
    s_hat = synth.sphere_sdf(dims, np.zeros(3), np.array([1.0, 0.9, 1.2]), (0.5, 0.45, 0.6), 0.3)
    s_hat = s_hat + 0.02 * _field(s_hat.shape, 5)
    s = R.smooth(s_hat)
    lam = {"sdf": (1.0, 0, 0), "eik": (0, 1.0, 0), "normal": (0, 0, 1.0)}[which]
    w = R.voxel_weight(s)
    own = synth.rng(6).uniform(size=s.shape) < 0.5
    vals, ds, ds_hat = R.sdf_terms(s_hat, s, h, *lam, weights=w, owner=own)
    full = R.sdf_terms(s_hat, s, h, *lam, weights=w)
    every = R.sdf_terms(s_hat, s, h, *lam, weights=w, owner=np.ones(s.shape, bool))
    assert every[0] == full[0]
    assert np.array_equal(every[1], full[1]) and np.array_equal(every[2], full[2])
    rest = R.sdf_terms(s_hat, s, h, *lam, weights=w, owner=~own)
    for k in ("sdf", "eik", "normal", "objective"):
        assert abs(vals[k] + rest[0][k] - full[0][k]) <= 1e-12 * max(1.0, abs(full[0][k]))
    assert np.allclose(ds + rest[1], full[1], rtol=0, atol=1e-12)
    g = synth.rng(7)
    eps = 1e-6
    for arr, grad in ((s, ds), (s_hat, ds_hat)):
        flat, gflat = arr.reshape(-1), grad.reshape(-1)
        for i in g.choice(flat.size, 60, replace=False):
            old = flat[i]
            flat[i] = old + eps
            lp = R.sdf_terms(s_hat, s, h, *lam, weights=w, owner=own)[0]["objective"]
            flat[i] = old - eps
            lm = R.sdf_terms(s_hat, s, h, *lam, weights=w, owner=own)[0]["objective"]
            flat[i] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - gflat[i]) <= 1e-6 * max(1.0, abs(gflat).max()), (which, i, fd, gflat[i])


def test_probe_and_plane_gradients_central_differences():
    # both losses are quadratic: central differences are exact for any step
    b = _field((3, 4, 3, 9, 4), 5)
    P = _field((1, 2, 1, 3, 16, 16, 3), 6)
    h = 1e-2
    for arr, fn in ((b, R.probe_terms), (P, R.plane_terms)):
        _, grad = fn(arr, 0.7)
        flat, gflat = arr.reshape(-1), grad.reshape(-1)
        for i in synth.rng(7).choice(flat.size, 50, replace=False):
            old = flat[i]
            flat[i] = old + h
            lp = 0.7 * fn(arr, 0.7)[0]
            flat[i] = old - h
            lm = 0.7 * fn(arr, 0.7)[0]
            flat[i] = old
            assert abs((lp - lm) / (2 * h) - gflat[i]) <= 1e-9 * max(1, abs(gflat[i]))
