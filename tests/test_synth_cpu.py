"""The seeded input generators that only the bench and the sparse tests use
(CPU): the sparse object scene stores exactly the dense scene's values in its
bricks and keeps every brick near the surface; smooth features vary over a
few voxels."""
import numpy as np

import synth


def test_sparse_object_bricks_hold_the_dense_scene():
    R, band = 64, 0.05
    keep, bsdf, bfeat, probes, mlp = synth.sparse_object(R, band)
    shapes = synth.object_shapes(synth.rng(1240), 32)
    dense = synth.object_sdf((R, R, R), (0, 0, 0), (1, 1, 1), shapes)
    idx = np.argwhere(keep)
    assert idx.shape[0] == bsdf.shape[0] == bfeat.shape[0]
    for k in range(0, idx.shape[0], max(1, idx.shape[0] // 16)):
        bz, by, bx = idx[k]
        np.testing.assert_array_equal(
            bsdf[k], dense[bz * 16:bz * 16 + 16, by * 16:by * 16 + 16, bx * 16:bx * 16 + 16])
    # every brick holding a node within the band is stored
    near = (np.abs(dense) < band).reshape(R // 16, 16, R // 16, 16, R // 16, 16).any(axis=(1, 3, 5))
    assert not np.any(near & ~keep)
    assert probes.shape == ((R - 1) // 16 + 1,) * 3 + (9, 4)
    assert mlp.size == synth.mlp_param_count(10, 32)


def test_smooth_features_scale_and_smoothness():
    g = synth.rng(3)
    f = synth.smooth_features((40, 36, 32), 3, g, sigma_vox=3.0, std=0.1)
    assert f.shape == (32, 36, 40, 3)
    np.testing.assert_allclose(f.std(axis=(0, 1, 2)), 0.1, rtol=1e-4)
    # neighbouring nodes differ far less than independent draws would
    step = np.abs(np.diff(f, axis=2)).mean()
    assert step < 0.25 * np.sqrt(2) * 0.1 * np.sqrt(2 / np.pi)
