"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test ties one step of the oracle to a closed form, an invariant, a
library routine or finite differences, so that a dropped term, a wrong sign,
a wrong index or a transposed operand anywhere in the oracle fails here.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------
# helpers: tiny scenes built directly
# ----------------------------------------------------------------------------

def tiny_scene(R=(5, 6, 7), P=(3, 3, 4), n_s=3, n_a=4, sh_l=3, width=8, K=3, seed=3,
               box=((0.0, 0.0, 0.0), (1.0, 1.0, 1.0)), sdf=None):
    g = synth.rng(seed)
    Rx, Ry, Rz = R
    Px, Py, Pz = P
    bmin = np.array(box[0], np.float32)
    bmax = np.array(box[1], np.float32)
    if sdf is None:
        sdf = synth.sphere_sdf(R, bmin.astype(float), bmax.astype(float), (0.5, 0.5, 0.5), 0.3)
        sdf = sdf + g.normal(0, 0.02, size=sdf.shape)
    feat = g.normal(0, 0.3, size=(Rz, Ry, Rx, n_s))
    probes = g.normal(0, 0.3, size=(Pz, Py, Px, sh_l * sh_l, n_a))
    mlp = synth.mlp_params(n_s + n_a + K, width, g).astype(np.float64)
    mlp += g.normal(0, 0.05, size=mlp.shape)  # non-zero biases too
    sc = synth.Scene(sdf=np.asarray(sdf, np.float32), feat=feat.astype(np.float32),
                     probes=probes.astype(np.float32), mlp=mlp.astype(np.float32),
                     box_min=bmin, box_max=bmax, sh_l=sh_l, width=width, n_fresnel=K)
    return sc


def node_positions(sc):
    Rx, Ry, Rz = sc.dims
    lo, hi = sc.box_min.astype(np.float64), sc.box_max.astype(np.float64)
    xs = np.linspace(lo[0], hi[0], Rx)
    ys = np.linspace(lo[1], hi[1], Ry)
    zs = np.linspace(lo[2], hi[2], Rz)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    return X, Y, Z


def rays_into_box(n, seed, center=(0.5, 0.5, 0.5), dist=1.8, spread=0.3):
    g = synth.rng(seed)
    dirs = synth.random_unit_vectors(n, g)
    o = np.asarray(center) - dist * dirs
    aim = np.asarray(center) + g.uniform(-spread, spread, size=(n, 3))
    d = aim - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return o.astype(np.float32), d.astype(np.float32)


def effective_points(sc, o, d, t):
    """Points at which the oracle evaluates the grid: x = fma(t, d, o) and
    u = (x - bmin) * (R-1)/extent, both rounded to FP32 (the stated sample
    position rule), mapped back to world units in FP64."""
    o64, d64 = o.astype(np.float64), d.astype(np.float64)
    t64 = np.asarray(t, np.float32).astype(np.float64)
    x32 = (t64[:, None] * d64[None] + o64[None]).astype(np.float32)   # exact product, one rounding
    bmin = sc.box_min.astype(np.float32)
    scale = (np.array(sc.dims, np.float32) - np.float32(1)) / (sc.box_max - sc.box_min)
    u32 = (x32 - bmin) * scale.astype(np.float32)
    return bmin.astype(np.float64) + u32.astype(np.float64) / scale.astype(np.float64)


def phi(tau, s):
    return 1.0 / (1.0 + np.exp(-tau * s))


# ----------------------------------------------------------------------------
# Spherical harmonics (Eq. 5): library routine + quadrature
# ----------------------------------------------------------------------------

def real_sh_scipy(l, r):
    from scipy.special import sph_harm_y
    x, y, z = r
    theta = math.acos(max(-1.0, min(1.0, z)))
    ph = math.atan2(y, x) % (2 * math.pi)
    out = []
    for deg in range(l):
        for m in range(-deg, deg + 1):
            Yc = complex(sph_harm_y(deg, abs(m), theta, ph))
            if m == 0:
                out.append(Yc.real)
            elif m > 0:  # remove scipy's Condon-Shortley phase
                out.append(math.sqrt(2) * (-1) ** m * Yc.real)
            else:
                out.append(math.sqrt(2) * (-1) ** m * Yc.imag)
    return np.array(out)


@pytest.mark.parametrize("l", [1, 2, 3, 4])
def test_sh_matches_scipy(l):
    g = synth.rng(11)
    for r in synth.random_unit_vectors(50, g):
        np.testing.assert_allclose(oracle.sh_eval(l, r), real_sh_scipy(l, r), atol=1e-13)


def test_sh_orthonormal_by_quadrature():
    # Gauss-Legendre in cos(theta) x uniform phi integrates products of degree <= 6 exactly.
    ct, wt = np.polynomial.legendre.leggauss(8)
    nphi = 16
    Ys, ws = [], []
    for c, w in zip(ct, wt):
        s = math.sqrt(1 - c * c)
        for k in range(nphi):
            p = 2 * math.pi * k / nphi
            Ys.append(oracle.sh_eval(4, [s * math.cos(p), s * math.sin(p), c]))
            ws.append(w * 2 * math.pi / nphi)
    Ys, ws = np.array(Ys), np.array(ws)
    gram = (Ys * ws[:, None]).T @ Ys
    np.testing.assert_allclose(gram, np.eye(16), atol=1e-13)


def test_sh_gradient_central_differences():
    g = synth.rng(12)
    h = 1e-6
    for r in synth.random_unit_vectors(10, g):
        dY = oracle.sh_grad(4, r)
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            fd = (oracle.sh_eval(4, r + e) - oracle.sh_eval(4, r - e)) / (2 * h)
            np.testing.assert_allclose(dY[:, a], fd, atol=1e-8)


# ----------------------------------------------------------------------------
# Trilinear interpolation (Sec. 3.1, Eq. 13 normal): affine fields are exact
# ----------------------------------------------------------------------------

def test_trilinear_reproduces_affine_field_and_gradient():
    sc = tiny_scene(R=(6, 5, 7), box=((-0.5, 0.25, 0.0), (1.5, 1.25, 2.0)))
    X, Y, Z = node_positions(sc)
    a = np.array([0.7, -1.3, 0.4])
    sc.sdf = (a[0] * X + a[1] * Y + a[2] * Z + 0.1).astype(np.float64)
    fa = [(X - 2 * Y + 0.5 * Z), (3 * X + Y), (-Z + 0.2)]
    sc.feat = np.stack(fa, -1)
    m = oracle.Model.from_scene(sc)
    g = synth.rng(5)
    for _ in range(40):
        # dyadic points: the FP32 grid coordinate (x - bmin) * (R-1)/extent is exact
        ext = (sc.box_max - sc.box_min).astype(np.float64)
        p = sc.box_min + g.integers(0, 1024, size=3) / 1024.0 * ext
        o = p.astype(np.float32)
        d = np.array([0.0, 0.0, 1.0], np.float32)
        out = oracle.point_eval(m, o, d, 0.0)
        x = o.astype(np.float64)
        assert abs(out["s"] - (a @ x + 0.1)) < 1e-12
        np.testing.assert_allclose(out["g"], a, atol=1e-12)
        expect = [x[0] - 2 * x[1] + 0.5 * x[2], 3 * x[0] + x[1], -x[2] + 0.2]
        np.testing.assert_allclose(out["x"][:3], expect, atol=1e-12)


def test_trilinear_gradient_is_central_difference_inside_a_cell():
    sc = tiny_scene(R=(5, 5, 5))
    m = oracle.Model.from_scene(sc)
    d = np.array([1.0, 0.0, 0.0], np.float32)
    # point well inside cell (1,2,1); cell size 0.25, a 1e-3 step stays inside
    base = np.array([0.3125, 0.5625, 0.3125], np.float32)
    out = oracle.point_eval(m, base, d, 0.0)
    h = np.float32(2 ** -12)
    for a in range(3):
        e = np.zeros(3, np.float32)
        e[a] = h
        sp = oracle.point_eval(m, base + e, d, 0.0)["s"]
        sm = oracle.point_eval(m, base - e, d, 0.0)["s"]
        assert abs((sp - sm) / (2 * float(h)) - out["g"][a]) < 1e-9


# ----------------------------------------------------------------------------
# Angular features, reflection, Fresnel (Eqs. 4-7)
# ----------------------------------------------------------------------------

def planar_scene(normal, offset=0.0, **kw):
    sc = tiny_scene(**kw)
    X, Y, Z = node_positions(sc)
    n = np.asarray(normal, float) / np.linalg.norm(normal)
    sc.sdf = (n[0] * X + n[1] * Y + n[2] * Z + offset).astype(np.float64)
    return sc, n


def test_l1_angular_feature_is_trilinear_blend_of_dc_coefficient():
    sc, _ = planar_scene([0.3, 0.2, 1.0], sh_l=1, n_a=2)
    X, Y, Z = [v for v in np.meshgrid(*(np.linspace(0, 1, k) for k in sc.probe_dims[::-1]),
                                      indexing="ij")][::-1]
    b0 = np.stack([2 * X - Y + Z, 0.5 * Z - X], -1)  # affine -> trilinear exact
    sc.probes = b0[:, :, :, None, :]
    m = oracle.Model.from_scene(sc)
    g = synth.rng(8)
    Y0 = 0.5 / math.sqrt(math.pi)
    for _ in range(20):
        p = (g.integers(51, 973, size=3) / 1024.0).astype(np.float32)  # exact FP32 grid coords
        d = synth.random_unit_vectors(1, g)[0].astype(np.float32)
        out = oracle.point_eval(m, p, d, 0.0)
        x = p.astype(np.float64)
        expect = np.array([2 * x[0] - x[1] + x[2], 0.5 * x[2] - x[0]]) * Y0
        np.testing.assert_allclose(out["x"][3:5], expect, atol=1e-12)


def _linear_probe_scene(normal, dir_mode):
    """Probes whose SH coefficients make F_a equal to the lookup direction:
    channel c holds 1/c1 on the degree-1 coefficient of axis c."""
    sc, n = planar_scene(normal, sh_l=2, n_a=3)
    c1 = math.sqrt(3.0 / (4.0 * math.pi))
    Pz, Py, Px = sc.probes.shape[:3]
    pr = np.zeros((Pz, Py, Px, 4, 3))
    pr[..., 3, 0] = 1 / c1  # Y_3 ~ x
    pr[..., 1, 1] = 1 / c1  # Y_1 ~ y
    pr[..., 2, 2] = 1 / c1  # Y_2 ~ z
    sc.probes = pr
    return sc, n


def test_reflected_direction_is_mirror_of_view_about_normal():
    sc, n = _linear_probe_scene([0.2, -0.5, 1.0], oracle.DIR_REFLECT)
    m = oracle.Model.from_scene(sc)
    g = synth.rng(9)
    for _ in range(20):
        p = g.uniform(0.1, 0.9, size=3).astype(np.float32)
        d = synth.random_unit_vectors(1, g)[0].astype(np.float32)
        v = -d.astype(np.float64)
        r = oracle.point_eval(m, p, d, 0.0)["x"][3:6]
        assert abs(np.linalg.norm(r) - 1.0) < 1e-6          # |r| = |v| (d is FP32-unit)
        assert abs(r @ n - v @ n) < 1e-6                     # same angle to the normal
        np.testing.assert_allclose(np.cross(r + v, n), 0, atol=1e-6)   # r + v along n
        assert abs((r - v) @ n) < 1e-6                       # r - v tangent
    # normal incidence (v = n): r = v
    d = (-n).astype(np.float32)
    r = oracle.point_eval(m, np.array([0.5, 0.5, 0.5], np.float32), d, 0.0)["x"][3:6]
    np.testing.assert_allclose(r, -d.astype(np.float64), atol=1e-7)


def test_view_mode_uses_view_direction():
    sc, n = _linear_probe_scene([0.2, -0.5, 1.0], oracle.DIR_VIEW)
    m = oracle.Model.from_scene(sc)
    d = synth.random_unit_vectors(1, synth.rng(4))[0].astype(np.float32)
    r = oracle.point_eval(m, np.array([0.4, 0.5, 0.6], np.float32), d, 0.0,
                          dir_mode=oracle.DIR_VIEW)["x"][3:6]
    np.testing.assert_allclose(r, -d.astype(np.float64), atol=1e-12)


def test_fresnel_inputs():
    # normal incidence: n.v = 1 disables the Fresnel inputs (the paper's ablation switch)
    sc, n = planar_scene([0.0, 0.0, 1.0])
    m = oracle.Model.from_scene(sc)
    x = oracle.point_eval(m, np.array([0.5, 0.5, 0.5], np.float32),
                          np.array([0.0, 0.0, -1.0], np.float32), 0.0)["x"]
    np.testing.assert_array_equal(x[7:10], 0.0)
    sc, n = planar_scene([0.0, 0.6, 0.8])
    m = oracle.Model.from_scene(sc)
    # oblique: (1 - cos(theta))^k with cos(theta) = n.v known from the plane
    g = synth.rng(10)
    for _ in range(10):
        d = synth.random_unit_vectors(1, g)[0].astype(np.float32)
        c = float(n @ -d.astype(np.float64))
        x = oracle.point_eval(m, np.array([0.5, 0.5, 0.5], np.float32), d, 0.0)["x"]
        np.testing.assert_allclose(x[7:10], [(1 - c), (1 - c) ** 2, (1 - c) ** 3], atol=1e-12)


# ----------------------------------------------------------------------------
# MLP (Sec. 4): zero weights and an identity construction
# ----------------------------------------------------------------------------

def test_mlp_zero_weights_gives_sigmoid_of_output_bias():
    sc = tiny_scene(width=8)
    W, n_in = 8, 10
    mlp = np.zeros(synth.mlp_param_count(n_in, W))
    b3 = np.array([0.3, -1.2, 2.0])
    mlp[-3:] = b3
    mlp[W * n_in:W * n_in + W] = 0.7  # b1 irrelevant once W3 = 0
    sc.mlp = mlp
    m = oracle.Model.from_scene(sc)
    out = oracle.point_eval(m, np.array([0.4, 0.5, 0.6], np.float32),
                            np.array([0, 0, 1], np.float32), 0.0)
    np.testing.assert_allclose(out["C"], 1 / (1 + np.exp(-b3)), atol=1e-15)


def test_mlp_layer_wiring_identity_construction():
    """W1 = [I; -I], W2 = I, W3 rows = [+1 .. +1, -1 .. -1] weighted per
    channel: z3_c = sum_i q_c(i) x_i, so C_c = sigmoid(sum_i q_c(i) x_i)."""
    n_in = 10
    W = 2 * n_in
    sc = tiny_scene(width=W)
    q = np.array([[1.0] * n_in, [(-1.0) ** i for i in range(n_in)], [0.1 * i for i in range(n_in)]])
    W1 = np.concatenate([np.eye(n_in), -np.eye(n_in)])
    W2 = np.eye(W)
    W3 = np.concatenate([q, -q], axis=1)
    sc.mlp = np.concatenate([W1.ravel(), np.zeros(W), W2.ravel(), np.zeros(W), W3.ravel(),
                             np.zeros(3)])
    m = oracle.Model.from_scene(sc)
    out = oracle.point_eval(m, np.array([0.35, 0.55, 0.6], np.float32),
                            synth.random_unit_vectors(1, synth.rng(2))[0].astype(np.float32), 0.0)
    z3 = q @ out["x"]
    np.testing.assert_allclose(out["C"], 1 / (1 + np.exp(-z3)), atol=1e-14)


# ----------------------------------------------------------------------------
# Compositing (Eqs. 8-10): closed forms and invariants
# ----------------------------------------------------------------------------

def test_fp32_sdf_option_is_the_same_trilinear_value_rounded():
    """The oracle's FP32-rounded SDF option (used only to isolate the FP32
    rounding of s in a GPU comparison) returns a FP32 number within a few FP32
    units of the FP64 trilinear value at every point, equals it exactly where
    the corner values and weights are exact in FP32, and does change some
    values (it is not a no-op)."""
    sc = tiny_scene(R=(9, 8, 7))
    m = oracle.Model.from_scene(sc)
    g = synth.rng(41)
    scale = float(np.max(np.abs(sc.sdf)))
    differ = 0
    for _ in range(300):
        o = g.uniform(0.05, 0.95, 3).astype(np.float32)
        d = g.normal(size=3)
        d = (d / np.linalg.norm(d)).astype(np.float32)
        t = float(g.uniform(0.0, 0.05))
        s64 = oracle.point_eval(m, o, d, t)["s"]
        s32 = oracle.point_eval(m, o, d, t, sdf_fp32=True)["s"]
        assert float(np.float32(s32)) == s32
        assert abs(s32 - s64) <= 8 * np.finfo(np.float32).eps * scale, (s32, s64)
        differ += s32 != s64
    assert differ > 10
    # dyadic corner values at points with dyadic fractions (node spacing 1/8):
    # every FP32 weight, product and sum is exact, so the two agree exactly
    sc2 = tiny_scene(R=(9, 9, 9))
    sc2.sdf = (np.round(sc2.sdf * 64) / 64).astype(np.float32)
    m2 = oracle.Model.from_scene(sc2)
    d = np.array([0.0, 0.0, 1.0], np.float32)
    for cell, frac in (((3, 2, 4), (0.5, 0.5, 0.5)), ((0, 6, 1), (0.25, 0.75, 0.125))):
        x = (np.array(cell) + np.array(frac)) / 8.0
        o = np.array([x[0], x[1], 0.0], np.float32)
        a = oracle.point_eval(m2, o, d, float(x[2]))["s"]
        b = oracle.point_eval(m2, o, d, float(x[2]), sdf_fp32=True)["s"]
        assert a == b, (cell, a, b)


def test_round_f16_is_ieee_binary16_rounding():
    """The oracle's binary16 rounding equals numpy's IEEE half-precision
    conversion (nearest, ties to even) on normal, subnormal, tie, overflow and
    signed-zero inputs."""
    g = synth.rng(43)
    v = g.normal(size=4000) * np.exp(g.uniform(-25.0, 12.0, size=4000))
    u = 2.0 ** -24
    special = np.array([1 + 2.0 ** -11, 1 + 3 * 2.0 ** -11, -(1 + 2.0 ** -11), 0.5 * u, 1.5 * u,
                        2.5 * u, 2.0 ** -14, 65504.0, 65519.99, 65520.0, -65520.0, 0.0, -0.0])
    v = np.concatenate([v, special])
    with np.errstate(over="ignore"):
        ref = v.astype(np.float16).astype(np.float64)
    got = oracle.round_f16(v)
    np.testing.assert_array_equal(got, ref)
    assert np.array_equal(np.signbit(got), np.signbit(ref))


def _mlp_blocks(sc, nin):
    p = np.asarray(sc.mlp, np.float64)
    W = sc.width
    o = 0
    out = []
    for shape in ((W, nin), (W,), (W, W), (W,), (3, W), (3,)):
        k = int(np.prod(shape))
        out.append((o, p[o:o + k].reshape(shape)))
        o += k
    return out


def _f16(a):
    return np.asarray(a, np.float64).astype(np.float16).astype(np.float64)


def test_mlp_f16_option_rounds_the_inputs_of_layers_one_and_two():
    """With the binary16 option the MLP input vector is the plain one rounded
    by numpy's IEEE binary16 conversion, and the colour is the sigmoid output
    layer over ReLU layers fed that rounded input and the rounded first hidden
    activations (evaluated here with numpy matrix products); the option does
    change colours."""
    sc = tiny_scene(R=(9, 8, 7), width=8)
    m = oracle.Model.from_scene(sc)
    nin = 3 + 4 + 3
    (_, W1), (_, b1), (_, W2), (_, b2), (_, W3), (_, b3) = _mlp_blocks(sc, nin)
    g = synth.rng(44)
    differ = 0
    for _ in range(100):
        o = g.uniform(0.05, 0.95, 3).astype(np.float32)
        d = g.normal(size=3)
        d = (d / np.linalg.norm(d)).astype(np.float32)
        t = float(g.uniform(0.0, 0.05))
        a = oracle.point_eval(m, o, d, t)
        b = oracle.point_eval(m, o, d, t, mlp_f16=True)
        assert a["s"] == b["s"]
        np.testing.assert_array_equal(b["x"], _f16(a["x"]))
        h1 = _f16(np.maximum(W1 @ b["x"] + b1, 0.0))
        h2 = np.maximum(W2 @ h1 + b2, 0.0)
        C = 1.0 / (1.0 + np.exp(-(W3 @ h2 + b3)))
        np.testing.assert_allclose(b["C"], C, rtol=0.0, atol=1e-14)
        differ += bool(np.any(b["C"] != a["C"]))
    assert differ > 50


def test_mlp_f16_adjoint_takes_the_rounding_as_identity():
    """Adjoint of the binary16 option: (a) the output layer and the second
    layer are smooth in W3, b3, W2 and b2 (the rounded values feeding them do
    not depend on those), so their gradients equal central differences of the
    rounded forward; (b) with one colour sample per ray the first layer's
    weight gradient is the outer product of its bias gradient with the rounded
    input vector."""
    sc = tiny_scene(R=(8, 8, 8), P=(3, 3, 3), width=8)
    m = oracle.Model.from_scene(sc)
    nin = 3 + 4 + 3
    tau, N = 8.0, 16
    o, d = rays_into_box(48, 45)
    fw = oracle.render_forward(m, o, d, tau, N, margin=True, mlp_f16=True)
    keep = (fw["margin"] > 2e-3) & (fw["wsum"] > 0)
    o, d = o[keep][:12], d[keep][:12]
    assert o.shape[0] >= 6
    g = synth.rng(46)
    drgb = g.normal(size=(o.shape[0], 3))
    grads = oracle.render_backward(m, o, d, drgb, tau, N, mlp_f16=True)["mlp"]
    blocks = _mlp_blocks(sc, nin)
    first = blocks[2][0]  # W2, b2, W3, b3 follow contiguously
    flat = m.mlp.reshape(-1)
    scale = np.abs(grads[first:]).max()
    h = 1e-6
    for i in range(first, flat.size):
        old = flat[i]
        flat[i] = old + h
        lp = np.sum(oracle.render_forward(m, o, d, tau, N, mlp_f16=True)["rgb"] * drgb)
        flat[i] = old - h
        lm = np.sum(oracle.render_forward(m, o, d, tau, N, mlp_f16=True)["rgb"] * drgb)
        flat[i] = old
        assert abs((lp - lm) / (2 * h) - grads[i]) <= 1e-6 * scale + 1e-10, i
    # (b) one colour sample per ray at given distances
    W = sc.width
    n_checked = 0
    for r in range(o.shape[0]):
        ts = np.array([[1.45, 1.9]], np.float32)  # both inside the box
        gr = oracle.render_backward(m, o[r:r + 1], d[r:r + 1], drgb[r:r + 1], tau, 1,
                                    t_samples=ts, mlp_f16=True)["mlp"]
        gW1 = gr[:W * nin].reshape(W, nin)
        gb1 = gr[W * nin:W * nin + W]
        if not np.any(gb1):
            continue
        xr = oracle.point_eval(m, o[r], d[r], float(ts[0, 0]), mlp_f16=True)["x"]
        x = oracle.point_eval(m, o[r], d[r], float(ts[0, 0]))["x"]
        np.testing.assert_array_equal(gW1, np.outer(gb1, xr))
        assert not np.array_equal(gW1, np.outer(gb1, x))
        n_checked += 1
    assert n_checked >= 3


def test_weights_plus_final_transmittance_is_one():
    sc = tiny_scene(R=(12, 12, 12))
    m = oracle.Model.from_scene(sc)
    o, d = rays_into_box(200, 21)
    out = oracle.render_forward(m, o, d, 64.0, 40)
    hit = out["wsum"] > 0
    assert hit.sum() > 150
    np.testing.assert_allclose(out["wsum"] + np.exp(out["logT"]), 1.0, atol=1e-13)
    assert np.all(out["wsum"] >= 0) and np.all(out["wsum"] <= 1 + 1e-15)


def test_planar_sdf_closed_form():
    """A plane is exact on the grid; with W3 = 0 every colour is sigmoid(b3), so
    rgb = sigmoid(b3) (1 - Phi(s_N)/Phi(s_0)) and w_k = (Phi(s_k)-Phi(s_k+1))/Phi(s_0)
    when s decreases along the ray."""
    sc, n = planar_scene([0.1, 0.2, -1.0], offset=0.5, R=(9, 9, 9))
    W, n_in = sc.width, 10
    mlp = sc.mlp.astype(np.float64).copy()
    o3 = W * n_in + W + W * W + W
    mlp[o3:o3 + 3 * W] = 0.0
    b3 = mlp[-3:] = np.array([0.4, -0.3, 1.1])
    sc.mlp = mlp
    m = oracle.Model.from_scene(sc)
    tau, N = 20.0, 50
    g = synth.rng(30)
    for _ in range(10):
        o = np.array([g.uniform(0.3, 0.7), g.uniform(0.3, 0.7), -1.0], np.float32)
        d = np.array([g.uniform(-0.2, 0.2), g.uniform(-0.2, 0.2), 1.0])
        d = (d / np.linalg.norm(d)).astype(np.float32)
        tr = oracle.render_trace(m, o, d, tau, N)
        s = effective_points(sc, o, d, tr["t"]) @ n + 0.5
        assert np.all(np.diff(s) < 0)
        np.testing.assert_allclose(tr["s"], s, atol=1e-12)
        ph = phi(tau, s)
        np.testing.assert_allclose(tr["w"], (ph[:-1] - ph[1:]) / ph[0], rtol=1e-10, atol=1e-15)
        out = oracle.render_forward(m, o[None], d[None], tau, N)
        np.testing.assert_allclose(out["rgb"][0], (1 - ph[-1] / ph[0]) / (1 + np.exp(-b3)),
                                   rtol=1e-12)
        np.testing.assert_allclose(out["depth"][0],
                                   np.sum(tr["t"][:-1] * (ph[:-1] - ph[1:]) / ph[0]), rtol=1e-12)


def test_unimodal_ray_transmittance_telescopes():
    """For an SDF that falls then rises along a ray, the clipped log-steps
    telescope: wsum = 1 - Phi(min_k s_k) / Phi(s_0)."""
    R = (40, 40, 40)
    X, Y, Z = np.meshgrid(*(np.linspace(0, 1, k) for k in R), indexing="ij")
    sdf = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2) - 0.3
    sc = tiny_scene(R=R, sdf=sdf.transpose(2, 1, 0))
    m = oracle.Model.from_scene(sc)
    o, d = rays_into_box(60, 31, spread=0.35)
    tau, N = 30.0, 80
    checked = 0
    for i in range(60):
        tr = oracle.render_trace(m, o[i], d[i], tau, N)
        if not tr["hit"]:
            continue
        s = tr["s"]
        k = int(np.argmin(s))
        if not (np.all(np.diff(s[:k + 1]) < 0) and np.all(np.diff(s[k:]) >= 0)):
            continue
        checked += 1
        out = oracle.render_forward(m, o[i:i + 1], d[i:i + 1], tau, N)
        np.testing.assert_allclose(out["wsum"][0], 1 - phi(tau, s[k]) / phi(tau, s[0]),
                                   rtol=1e-12, atol=1e-14)
    assert checked > 30


def test_sphere_depth_at_true_surface():
    R = (128, 128, 128)
    X, Y, Z = np.meshgrid(*(np.linspace(0, 1, k) for k in R), indexing="ij")
    sdf = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2) - 0.3
    sc = tiny_scene(R=R, sdf=sdf.transpose(2, 1, 0))
    m = oracle.Model.from_scene(sc)
    o, d = rays_into_box(80, 41, spread=0.06)
    tau, N = 64.0, 256
    out = oracle.render_forward(m, o, d, tau, N)
    c = np.array([0.5, 0.5, 0.5])
    checked = 0
    for i in range(80):
        oo, dd = o[i].astype(float), d[i].astype(float)
        b = dd @ (oo - c)
        disc = b * b - ((oo - c) @ (oo - c) - 0.3 ** 2)
        closest = np.linalg.norm((oo - c) - ((oo - c) @ dd) * dd)
        if disc < 0 or closest > 0.07:  # keep rays passing deep inside: Phi(s_min) < 1e-6
            continue
        t_hit = -b - math.sqrt(disc)
        # box segment length / N bounds the sample spacing
        delta = math.sqrt(3) / N
        assert out["wsum"][i] > 1 - 1e-6
        assert abs(out["depth"][i] / out["wsum"][i] - t_hit) <= delta + 4.0 / tau
        checked += 1
    assert checked > 20


def test_missing_rays_give_background():
    sc = tiny_scene()
    m = oracle.Model.from_scene(sc)
    o = np.array([[2.0, 2.0, 2.0], [-1.0, 0.5, 0.5]], np.float32)
    d = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]], np.float32)
    out = oracle.render_forward(m, o, d, 64.0, 16, bg=(0.1, 0.2, 0.3))
    np.testing.assert_allclose(out["rgb"], [[0.1, 0.2, 0.3]] * 2)
    assert np.all(out["wsum"] == 0) and np.all(out["depth"] == 0)


# ----------------------------------------------------------------------------
# Adjoint (Sec. 3.3-3.4): central finite differences in FP64
# ----------------------------------------------------------------------------

def _loss(m, o, d, drgb, ddepth, dwsum, tau, N, dir_mode, bg):
    out = oracle.render_forward(m, o, d, tau, N, dir_mode=dir_mode, bg=bg)
    return (np.sum(out["rgb"] * drgb) + np.sum(out["depth"] * ddepth) +
            np.sum(out["wsum"] * dwsum))


@pytest.mark.parametrize("dir_mode", [oracle.DIR_REFLECT, oracle.DIR_VIEW])
def test_adjoint_matches_central_differences(dir_mode):
    sc = tiny_scene(R=(8, 8, 8), P=(3, 3, 3), width=4, sh_l=3, n_a=4)
    m = oracle.Model.from_scene(sc)
    tau, N, bg = 8.0, 16, (0.2, 0.1, 0.3)
    o, d = rays_into_box(48, 51)
    fw = oracle.render_forward(m, o, d, tau, N, dir_mode=dir_mode, bg=bg, margin=True)
    keep = (fw["margin"] > 2e-3) & (fw["wsum"] > 0)
    o, d = o[keep][:16], d[keep][:16]
    assert o.shape[0] >= 8
    g = synth.rng(52)
    n = o.shape[0]
    drgb, ddepth, dwsum = g.normal(size=(n, 3)), g.normal(size=n), g.normal(size=n)
    grads = oracle.render_backward(m, o, d, drgb, tau, N, d_depth=ddepth, d_wsum=dwsum,
                                   dir_mode=dir_mode, bg=bg)
    h = 1e-6
    for name, arr in (("sdf", m.sdf), ("feat", m.feat), ("probes", m.probes), ("mlp", m.mlp)):
        flat = arr.reshape(-1)
        gflat = grads[name].reshape(-1)
        scale = max(np.abs(gflat).max(), 1e-12)
        idx = np.arange(flat.size) if flat.size <= 700 else g.choice(flat.size, 700, replace=False)
        # include every parameter with a non-zero gradient for the small tensors
        for i in idx:
            old = flat[i]
            flat[i] = old + h
            lp = _loss(m, o, d, drgb, ddepth, dwsum, tau, N, dir_mode, bg)
            flat[i] = old - h
            lm = _loss(m, o, d, drgb, ddepth, dwsum, tau, N, dir_mode, bg)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - gflat[i]) <= 1e-6 * scale + 1e-9, (name, i, fd, gflat[i])


def test_adjoint_directional_derivative():
    """<grad, delta> equals the central difference along a random direction of
    every parameter at once."""
    sc = tiny_scene(R=(10, 9, 8), P=(4, 3, 3), width=8)
    m = oracle.Model.from_scene(sc)
    tau, N = 16.0, 24
    o, d = rays_into_box(64, 61)
    fw = oracle.render_forward(m, o, d, tau, N, margin=True)
    keep = fw["margin"] > 1e-3
    o, d = o[keep], d[keep]
    g = synth.rng(62)
    n = o.shape[0]
    drgb = g.normal(size=(n, 3))
    grads = oracle.render_backward(m, o, d, drgb, tau, N)
    arrs = [m.sdf, m.feat, m.probes, m.mlp]
    deltas = [g.normal(size=a.shape) for a in arrs]
    base = [a.copy() for a in arrs]
    h = 1e-6
    vals = []
    for sgn in (1, -1):
        for a, b0, dl in zip(arrs, base, deltas):
            a[...] = b0 + sgn * h * dl
        vals.append(_loss(m, o, d, drgb, 0, 0, tau, N, oracle.DIR_REFLECT, (0, 0, 0)))
    for a, b0 in zip(arrs, base):
        a[...] = b0
    fd = (vals[0] - vals[1]) / (2 * h)
    ana = sum(np.sum(grads[k] * dl) for k, dl in zip(("sdf", "feat", "probes", "mlp"), deltas))
    assert abs(fd - ana) <= 1e-7 * abs(ana) + 1e-10


def test_threaded_backward_equals_single_thread():
    sc = tiny_scene(R=(16, 16, 16), P=(5, 5, 5))
    m = oracle.Model.from_scene(sc)
    o, d = rays_into_box(300, 71)
    drgb = synth.rng(72).normal(size=(300, 3))
    g1 = oracle.render_backward(m, o, d, drgb, 32.0, 32, n_threads=1)
    g4 = oracle.render_backward(m, o, d, drgb, 32.0, 32, n_threads=4)
    for k in g1:
        np.testing.assert_allclose(g4[k], g1[k], atol=1e-12 * max(1.0, np.abs(g1[k]).max()))
    f1 = oracle.render_forward(m, o, d, 32.0, 32, n_threads=1)
    f4 = oracle.render_forward(m, o, d, 32.0, 32, n_threads=4)
    for k in f1:
        np.testing.assert_array_equal(f1[k], f4[k])


def test_oracle_reproduces_committed_fixture():
    """The oracle built on this machine gives the committed values (written by
    tests/golden/make_oracle_fixture.py, which calls only the oracle)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "make_oracle_fixture", os.path.join(GOLDEN, "make_oracle_fixture.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    with open(os.path.join(GOLDEN, "oracle_fixture_small.json")) as f:
        gold = json.load(f)
    now = mod.compute()
    for k in ("rgb", "depth", "wsum", "logT"):
        np.testing.assert_allclose(now[k], gold[k], rtol=1e-11, atol=1e-14)
    for k in ("sdf", "feat", "probes", "mlp"):
        g = gold["grad_" + k]
        np.testing.assert_allclose(now["grad_" + k][g["index"]], g["value"], rtol=1e-10,
                                   atol=1e-15)


# ----------------------------------------------------------------------------
# Learned sample proposal (not in the paper): pins of its oracle
# ----------------------------------------------------------------------------

def _proposal_fixture(seed=81, logit_scale=1.0):
    sc = tiny_scene(R=(16, 16, 16), P=(4, 4, 4))
    m = oracle.Model.from_scene(sc)
    occ = oracle.occupancy(m, (6, 6, 6), 2.0 / 15)
    g = synth.rng(seed)
    params = synth.proposal_params(g).astype(np.float64)
    params[-8 - 8 * 32:] *= logit_scale
    return sc, m, occ, params


@pytest.mark.parametrize("occ_fill", [0.0, 1.0])
def test_proposal_uniform_density_gives_uniform_quantiles(occ_fill):
    sc, m, occ, params = _proposal_fixture()
    params[-8 - 8 * 32:] = 0.0  # W3 = 0, b3 = 0: every logit 0
    # no bin occupied, or every bin: the mix share is uniform as well
    prop = oracle.Proposal(np.full_like(occ, occ_fill), params, mix=0.1, theta=0.0)
    o, d = rays_into_box(40, 82)
    out = oracle.proposal_forward(m, prop, o, d, 24)
    np.testing.assert_allclose(out["probs"], 1.0 / 8, atol=1e-15)
    for i in range(40):
        tr = oracle.render_trace(m, o[i], d[i], 10.0, 24)  # uniform sample positions
        if not tr["hit"]:
            assert np.all(out["t"][i] == 0)
            continue
        tn, tf = float(tr["t"][0]), float(tr["t"][-1])
        np.testing.assert_allclose(out["t"][i], tn + (tf - tn) * np.arange(25) / 24, atol=1e-12)


def test_proposal_quantile_placement_follows_density():
    sc, m, occ, params = _proposal_fixture(logit_scale=8.0)
    prop = oracle.Proposal(occ, params, mix=0.1, theta=0.0)
    o, d = rays_into_box(30, 83)
    n_out = 400
    out = oracle.proposal_forward(m, prop, o, d, n_out)
    for i in range(30):
        t = out["t"][i]
        if t[-1] <= t[0]:
            continue
        assert np.all(np.diff(t) >= 0)
        edges = t[0] + (t[-1] - t[0]) * np.arange(9) / 8
        # fraction of the n_out sample intervals falling in each bin = the density
        counts = np.histogram(0.5 * (t[1:] + t[:-1]), bins=edges)[0] / n_out
        np.testing.assert_allclose(counts, out["probs"][i], atol=2.0 / n_out)
        # the piecewise-linear CDF of the bin density reaches k / n_out at t_k
        cdf = np.interp(t, edges, np.concatenate([[0.0], np.cumsum(out["probs"][i])]))
        np.testing.assert_allclose(cdf, np.arange(n_out + 1) / n_out, atol=1e-6)
        assert abs(out["probs"][i].sum() - 1) < 1e-12 and out["probs"][i].min() >= 0.1 / 32 - 1e-15


def test_weight_histogram_sums_to_wsum():
    sc = tiny_scene(R=(12, 12, 12))
    m = oracle.Model.from_scene(sc)
    o, d = rays_into_box(50, 84)
    h = oracle.weight_histogram(m, o, d, 32.0, 48, 8)
    fw = oracle.render_forward(m, o, d, 32.0, 48)
    np.testing.assert_allclose(h.sum(1), fw["wsum"], atol=1e-13)
    tr = oracle.render_trace(m, o[0], d[0], 32.0, 48)
    np.testing.assert_allclose(h[0], tr["w"].reshape(8, 6).sum(1), atol=1e-15)


def test_occupancy_of_a_sphere_shell():
    R = (24, 24, 24)
    X, Y, Z = np.meshgrid(*(np.linspace(0, 1, k) for k in R), indexing="ij")
    dist = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2)
    sc = tiny_scene(R=R, sdf=(dist - 0.3).transpose(2, 1, 0))
    m = oracle.Model.from_scene(sc)
    thr = 2.0 / 23
    occ = oracle.occupancy(m, (8, 8, 8), thr)
    cs = (np.arange(8) + 0.5) / 8
    CZ, CY, CX = np.meshgrid(cs, cs, cs, indexing="ij")
    shell = np.abs(np.sqrt((CX - 0.5) ** 2 + (CY - 0.5) ** 2 + (CZ - 0.5) ** 2) - 0.3)
    half_diag = np.sqrt(3) * (0.5 / 8 + 1.0 / 23)
    assert np.all(occ[shell < thr - half_diag] == 1)       # cells straddling the shell
    assert np.all(occ[shell > thr + half_diag] == 0)       # cells far from it
    assert 0 < occ.mean() < 0.8


def test_proposal_gradient_central_differences():
    sc, m, occ, params = _proposal_fixture(seed=85)
    o, d = rays_into_box(24, 86)
    hist = oracle.weight_histogram(m, o, d, 16.0, 32, 8)
    keep = hist.sum(1) > 1e-3
    o, d, hist = o[keep], d[keep], hist[keep]
    prop = oracle.Proposal(occ, params)
    g, loss = oracle.proposal_backward(m, prop, o, d, hist, 1e-3, 0.5)
    flat = prop.params
    h = 1e-6
    idx = synth.rng(87).choice(flat.size, 300, replace=False)
    for i in idx:
        old = flat[i]
        flat[i] = old + h
        lp = oracle.proposal_backward(m, prop, o, d, hist, 1e-3, 0.5)[1].sum()
        flat[i] = old - h
        lm = oracle.proposal_backward(m, prop, o, d, hist, 1e-3, 0.5)[1].sum()
        flat[i] = old
        fd = 0.5 * (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * np.abs(g).max() + 1e-9, (i, fd, g[i])


def _passthrough_params(B, pick):
    """Proposal weights whose logits equal its occupancy inputs (all >= 0, so
    the ReLUs pass them): the bin fractions (pick "frac"), the step inputs
    ("step"), or the first-position input in logit 0 ("first")."""
    W, nin = 32, 7 + 2 * B
    W1 = np.zeros((W, nin))
    first_col = {"frac": 7, "step": 7 + B, "first": 6}[pick]
    for u in range(B if pick != "first" else 1):
        W1[u, first_col + u] = 1.0
    W2 = np.eye(W)
    W3 = np.zeros((B, W))
    for b in range(B if pick != "first" else 1):
        W3[b, b] = 1.0
    return np.concatenate([W1.ravel(), np.zeros(W), W2.ravel(), np.zeros(W), W3.ravel(),
                           np.zeros(B)])


@pytest.mark.parametrize("B,n_sub,res", [(8, 3, (4, 5, 3)), (16, 2, (7, 7, 7))])
def test_proposal_occupancy_inputs_brute_force(B, n_sub, res):
    sc = tiny_scene(R=(16, 16, 16), P=(4, 4, 4))
    m = oracle.Model.from_scene(sc)
    g = synth.rng(88 + B)
    occ = (g.uniform(size=res[::-1]) < 0.3).astype(np.float64)
    o, d = rays_into_box(60, 89 + B)
    fr, fi, fs = (oracle.proposal_forward(m, oracle.Proposal(occ, _passthrough_params(B, k),
                                                             n_bins=B, n_sub=n_sub), o, d, 4)
                  for k in ("frac", "first", "step"))
    bmin = np.asarray(sc.box_min, np.float64)
    ext = np.asarray(sc.box_max, np.float64) - bmin
    checked = 0
    for i in range(60):
        tn, tf = fr["t"][i, 0], fr["t"][i, -1]
        if not tf > tn:
            continue
        k = np.arange(B * n_sub)
        t = tn + (k + 0.5) * (tf - tn) / (B * n_sub)
        u = (o[i].astype(np.float64) + t[:, None] * d[i].astype(np.float64) - bmin) / ext * res
        r = np.round(u)
        inner = (r >= 1) & (r <= np.array(res) - 1)  # the faces between two cells
        if np.any(inner & (np.abs(u - r) < 1e-4)):
            continue  # a point on a cell face: its cell is decided by FP32 rounding
        c = np.floor(np.clip(u, 0, np.array(res) - 1)).astype(int)
        hit = occ[c[:, 2], c[:, 1], c[:, 0]] > 0.5
        frac = hit.reshape(B, n_sub).mean(1)
        first = (np.argmax(hit) + 0.5) / (B * n_sub) if hit.any() else 1.0
        np.testing.assert_allclose(fr["logits"][i], frac, atol=1e-12)
        assert abs(fi["logits"][i, 0] - first) < 1e-12
        # share of each bin before the first occupied point
        before = np.array([np.clip(first * B - b, 0.0, 1.0) for b in range(B)])
        np.testing.assert_allclose(fs["logits"][i], before, atol=1e-12)
        checked += 1
    assert checked > 20


# ----------------------------------------------------------------------------
# Tile tri-plane spatial features (Sec. 3.1, Sec. 4)
# ----------------------------------------------------------------------------

def _triplane_scene(R=(20, 35, 18), seed=5, planes=None):
    sc = tiny_scene(R=R, P=(4, 4, 4), seed=seed)
    sc = synth.with_triplanes(sc, seed + 1)
    if planes is not None:
        sc.planes[...] = planes
    return sc


def _fs_at(m, sc, pts):
    """F_s (the first n_s MLP inputs) at world points, looked up along +x rays."""
    out = []
    for x in pts:
        o = np.asarray(x, np.float32) - np.float32([1.0, 0.0, 0.0])
        d = np.float32([1.0, 0.0, 0.0])
        r = oracle.point_eval(m, o, d, 1.0)
        out.append(r["x"][:sc.n_s])
    return np.array(out)


def test_triplane_constant_planes_give_the_product():
    sc = _triplane_scene()
    c = np.array([1.5, -0.7, 2.0])  # plane p holds c[p] in every texel and channel
    sc.planes[...] = c[None, None, None, :, None, None, None]
    m = oracle.Model.from_scene(sc)
    pts = synth.rng(7).uniform(0.02, 0.98, size=(40, 3))
    want = np.prod(c.astype(np.float32).astype(np.float64))  # the planes are stored in FP32
    np.testing.assert_allclose(_fs_at(m, sc, pts), want, rtol=1e-14)


def test_triplane_affine_planes_are_reproduced_inside_a_tile():
    """Texels affine in their in-plane coordinates: the bilinear lookups are
    exact, so F_s is the product of the affine functions of the point's local
    coordinates (texel i sits at local coordinate i + 1/2)."""
    R = (33, 33, 33)  # two tiles per axis, spacing 1/32
    sc = _triplane_scene(R=R)
    i = np.arange(16) + 0.5
    a = [(0.3, 1.0), (-0.2, 4.0), (0.05, 0.5)]  # per plane: slope in its column coordinate
    b = [(0.1,), (0.0,), (0.2,)]                 # and in its row coordinate
    for p in range(3):
        for ch in range(sc.n_s):
            val = a[p][0] * i[None, :] + a[p][1] + b[p][0] * i[:, None] + 0.1 * ch
            sc.planes[:, :, :, p, :, :, ch] = val
    m = oracle.Model.from_scene(sc)
    g = synth.rng(8)
    tile = g.integers(0, 2, size=(60, 3))
    local = g.uniform(0.6, 15.4, size=(60, 3))  # away from the clamped edge texels
    u = tile * 16 + local
    pts = u / 32.0
    fs = _fs_at(m, sc, pts)
    lx, ly, lz = local[:, 0], local[:, 1], local[:, 2]
    for ch in range(sc.n_s):
        f0 = a[0][0] * ly + a[0][1] + b[0][0] * lz + 0.1 * ch   # plane [z][y]
        f1 = a[1][0] * lx + a[1][1] + b[1][0] * lz + 0.1 * ch   # plane [z][x]
        f2 = a[2][0] * lx + a[2][1] + b[2][0] * ly + 0.1 * ch   # plane [y][x]
        np.testing.assert_allclose(fs[:, ch], f0 * f1 * f2, rtol=2e-6)


def test_triplane_tile_of_a_point():
    """A point reads the planes of the tile holding its cell; the far face of
    the last tile belongs to the last tile."""
    R = (40, 17, 17)  # x: 39 cells -> tiles of 16, 16, 7
    sc = _triplane_scene(R=R)
    sc.planes[...] = 1.0
    sc.planes[:, :, 1, 0] = 2.0   # tile x = 1: plane 0 doubled
    sc.planes[:, :, 2, 1] = 3.0   # tile x = 2: plane 1 tripled
    m = oracle.Model.from_scene(sc)
    h = 1.0 / 39
    for ux, want in ((15.5, 1.0), (16.5, 2.0), (31.9, 2.0), (32.1, 3.0), (38.999, 3.0)):
        fs = _fs_at(m, sc, [(ux * h, 0.5, 0.5)])[0]
        np.testing.assert_allclose(fs, want, rtol=1e-12)


@pytest.mark.parametrize("dir_mode", [oracle.DIR_REFLECT])
def test_triplane_adjoint_matches_central_differences(dir_mode):
    sc = _triplane_scene(R=(20, 18, 19), seed=9)
    sc.planes[...] = synth.rng(10).normal(1.0, 0.3, size=sc.planes.shape)
    m = oracle.Model.from_scene(sc)
    tau, N = 8.0, 16
    o, d = rays_into_box(48, 53)
    fw = oracle.render_forward(m, o, d, tau, N, margin=True)
    keep = (fw["margin"] > 2e-3) & (fw["wsum"] > 0)
    o, d = o[keep][:16], d[keep][:16]
    assert o.shape[0] >= 8
    g = synth.rng(54)
    drgb = g.normal(size=(o.shape[0], 3))
    grads = oracle.render_backward(m, o, d, drgb, tau, N)
    gp = grads["feat"]
    assert gp.shape == m.planes.shape and np.abs(gp).max() > 0
    flat, gflat = m.planes.reshape(-1), gp.reshape(-1)
    nz = np.nonzero(gflat)[0]
    idx = np.concatenate([g.choice(nz, min(300, nz.size), replace=False),
                          g.choice(flat.size, 100, replace=False)])
    scale = np.abs(gflat).max()
    h = 1e-6
    for i in idx:
        old = flat[i]
        flat[i] = old + h
        lp = _loss(m, o, d, drgb, 0, 0, tau, N, dir_mode, (0, 0, 0))
        flat[i] = old - h
        lm = _loss(m, o, d, drgb, 0, 0, tau, N, dir_mode, (0, 0, 0))
        flat[i] = old
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gflat[i]) <= 1e-6 * scale + 1e-9, (i, fd, gflat[i])
