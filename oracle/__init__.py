"""FP64 CPU oracle of the ProbeSDF per-ray render and its adjoint.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product path (``paper_2412_10084_gb300``) never imports it, and this package
never imports the product: the two share only the seeded input generators of
``synth``.

The arithmetic lives in ``probesdf_oracle.c`` (plain C, FP64, one ray at a
time); this module compiles it with gcc and marshals numpy arrays through
ctypes.  Every function's paper passage is cited in the C source.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "probesdf_oracle.c")
_HDR = os.path.join(_HERE, "probesdf_oracle.h")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

DIR_REFLECT = 0
DIR_VIEW = 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off: the FP32 sample
    positions must be computed with exactly the stated roundings)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-shared", "-fPIC",
           "-ffp-contract=off", "-fno-fast-math", "-pthread", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Model(ctypes.Structure):
    _fields_ = [
        ("R", ctypes.c_int32 * 3),
        ("bmin", ctypes.c_float * 3),
        ("bmax", ctypes.c_float * 3),
        ("n_s", ctypes.c_int32),
        ("sdf", ctypes.c_void_p),
        ("feat", ctypes.c_void_p),
        ("P", ctypes.c_int32 * 3),
        ("sh_l", ctypes.c_int32),
        ("n_a", ctypes.c_int32),
        ("probes", ctypes.c_void_p),
        ("width", ctypes.c_int32),
        ("n_fresnel", ctypes.c_int32),
        ("mlp", ctypes.c_void_p),
        ("feat_layout", ctypes.c_int32),
        ("planes", ctypes.c_void_p),
    ]


FEAT_NODES = 0
FEAT_TRIPLANE = 1
TILE = 16


def n_tiles(R):
    return (int(R) - 1 + TILE - 1) // TILE


class _Params(ctypes.Structure):
    _fields_ = [
        ("tau", ctypes.c_double),
        ("n_samples", ctypes.c_int32),
        ("dir_mode", ctypes.c_int32),
        ("bg", ctypes.c_double * 3),
        ("sdf_fp32", ctypes.c_int32),
        ("mlp_f16", ctypes.c_int32),
    ]


class _Proposal(ctypes.Structure):
    _fields_ = [
        ("occ_res", ctypes.c_int32 * 3),
        ("occ", ctypes.c_void_p),
        ("width", ctypes.c_int32),
        ("n_bins", ctypes.c_int32),
        ("n_sub", ctypes.c_int32),
        ("params", ctypes.c_void_p),
        ("mix", ctypes.c_double),
        ("theta", ctypes.c_double),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.orc_round_f16.argtypes = [ctypes.c_double]
            lib.orc_round_f16.restype = ctypes.c_double
            lib.orc_sh_eval.argtypes = [ctypes.c_int32, P, P]
            lib.orc_sh_grad.argtypes = [ctypes.c_int32, P, P]
            lib.orc_render_forward.argtypes = [P, P, ctypes.c_int64, P, P, P, P, P, P, P, P,
                                               ctypes.c_int32]
            lib.orc_render_forward.restype = ctypes.c_int32
            lib.orc_render_backward.argtypes = [P, P, ctypes.c_int64, P, P, P, P, P, P, P, P, P,
                                                P, ctypes.c_int32]
            lib.orc_render_backward.restype = ctypes.c_int32
            lib.orc_render_trace.argtypes = [P, P, P, P, P, P, P, P, P, P]
            lib.orc_render_trace.restype = ctypes.c_int32
            lib.orc_point_eval.argtypes = [P, P, P, P, ctypes.c_float, P, P, P, P]
            lib.orc_point_eval.restype = ctypes.c_int32
            lib.orc_occupancy.argtypes = [P, P, ctypes.c_double, P]
            lib.orc_occupancy.restype = ctypes.c_int32
            lib.orc_proposal_forward.argtypes = [P, P, ctypes.c_int64, P, P, ctypes.c_int32, P,
                                                 P, P, P]
            lib.orc_proposal_forward.restype = ctypes.c_int32
            lib.orc_place_samples.argtypes = [P, ctypes.c_int64, P, P, P, ctypes.c_int32,
                                              ctypes.c_int32, P]
            lib.orc_place_samples.restype = ctypes.c_int32
            lib.orc_weight_histogram.argtypes = [P, P, ctypes.c_int64, P, P, ctypes.c_int32, P,
                                                 ctypes.c_int32]
            lib.orc_weight_histogram.restype = ctypes.c_int32
            lib.orc_proposal_backward.argtypes = [P, P, ctypes.c_int64, P, P, P, ctypes.c_double,
                                                  ctypes.c_double, P, P]
            lib.orc_proposal_backward.restype = ctypes.c_int32
            lib.orc_shade_nodes.argtypes = [P, P, P, ctypes.c_double, P]
            lib.orc_shade_nodes.restype = ctypes.c_int32
            lib.orc_shade_node_list.argtypes = [P, P, P, ctypes.c_double, ctypes.c_int64, P, P]
            lib.orc_shade_node_list.restype = ctypes.c_int32
            lib.orc_render_colour_field.argtypes = [P, P, P, ctypes.c_int64, P, P, P, P, P, P]
            lib.orc_render_colour_field.restype = ctypes.c_int32
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


class Model:
    """Oracle copy of a scene: every parameter promoted to FP64.

    sdf [Rz,Ry,Rx], feat [Rz,Ry,Rx,n_s], probes [Pz,Py,Px,l*l,n_a], mlp flat
    (W1[W][n_in] b1 W2[W][W] b2 W3[3][W] b3), box in FP32.
    """

    def __init__(self, sdf, feat, probes, mlp, box_min, box_max, sh_l, width, n_fresnel,
                 planes=None):
        self.sdf = _f64(sdf)
        self.feat = _f64(feat)
        self.planes = None if planes is None else _f64(planes)
        self.probes = _f64(probes)
        self.mlp = _f64(mlp).ravel()
        self.box_min = _f32(box_min)
        self.box_max = _f32(box_max)
        self.sh_l = int(sh_l)
        self.width = int(width)
        self.n_fresnel = int(n_fresnel)
        Rz, Ry, Rx = self.sdf.shape
        self.n_s = self.feat.shape[-1] if self.planes is None else self.planes.shape[-1]
        if self.planes is not None:
            assert self.planes.shape == (n_tiles(Rz), n_tiles(Ry), n_tiles(Rx), 3, TILE, TILE,
                                         self.n_s), "planes [tz][ty][tx][3][16][16][n_s]"
        Pz, Py, Px, L2, na = self.probes.shape
        assert L2 == self.sh_l ** 2
        self.n_a = na
        n_in = self.n_s + self.n_a + self.n_fresnel
        W = self.width
        assert self.mlp.size == W * n_in + W + W * W + W + 3 * W + 3, "mlp size"
        s = _Model()
        s.R[:] = (Rx, Ry, Rz)
        s.bmin[:] = tuple(float(v) for v in self.box_min)
        s.bmax[:] = tuple(float(v) for v in self.box_max)
        s.n_s = self.n_s
        s.sdf = self.sdf.ctypes.data
        s.feat = self.feat.ctypes.data
        s.P[:] = (Px, Py, Pz)
        s.sh_l = self.sh_l
        s.n_a = self.n_a
        s.probes = self.probes.ctypes.data
        s.width = W
        s.n_fresnel = self.n_fresnel
        s.mlp = self.mlp.ctypes.data
        s.feat_layout = FEAT_NODES if self.planes is None else FEAT_TRIPLANE
        s.planes = None if self.planes is None else self.planes.ctypes.data
        self._s = s

    @classmethod
    def from_scene(cls, sc):
        return cls(sc.sdf, sc.feat, sc.probes, sc.mlp, sc.box_min, sc.box_max, sc.sh_l,
                   sc.width, sc.n_fresnel, planes=getattr(sc, "planes", None))


def _params(tau, n_samples, dir_mode=DIR_REFLECT, bg=(0.0, 0.0, 0.0), sdf_fp32=False,
            mlp_f16=False):
    p = _Params()
    p.tau = float(tau)
    p.n_samples = int(n_samples)
    p.dir_mode = int(dir_mode)
    p.bg[:] = tuple(float(v) for v in bg)
    p.sdf_fp32 = int(bool(sdf_fp32))
    p.mlp_f16 = int(bool(mlp_f16))
    return p


def render_forward(model: Model, rays_o, rays_d, tau, n_samples, dir_mode=DIR_REFLECT,
                   bg=(0.0, 0.0, 0.0), t_samples=None, n_threads=1, margin=False,
                   sdf_fp32=False, mlp_f16=False):
    """rgb [n,3], depth [n], wsum [n], logT_final [n] (and the per-ray
    smallest relative distance to a ReLU or alpha-clip kink if asked).
    sdf_fp32: the SDF at each point rounded as the FP32 evaluation rounds it
    (everything else in FP64), to isolate that rounding in a comparison.
    mlp_f16: the MLP's layer-1 and layer-2 inputs rounded to binary16 as a
    reduced-precision evaluation stores them, so that both sides take the ReLU
    decisions on the same values (everything else in FP64)."""
    lib = _load()
    o, d = _f32(rays_o).reshape(-1, 3), _f32(rays_d).reshape(-1, 3)
    n = o.shape[0]
    ts = None if t_samples is None else _f32(t_samples).reshape(n, n_samples + 1)
    rgb = np.zeros((n, 3))
    depth, wsum, logT = np.zeros(n), np.zeros(n), np.zeros(n)
    mg = np.full(n, np.inf) if margin else None
    p = _params(tau, n_samples, dir_mode, bg, sdf_fp32, mlp_f16)
    st = lib.orc_render_forward(ctypes.byref(model._s), ctypes.byref(p), n, _ptr(o), _ptr(d),
                                _ptr(ts), _ptr(rgb), _ptr(depth), _ptr(wsum), _ptr(logT),
                                _ptr(mg), int(n_threads))
    if st != 0:
        raise ValueError(f"oracle forward rejected its arguments ({st})")
    out = {"rgb": rgb, "depth": depth, "wsum": wsum, "logT": logT}
    if margin:
        out["margin"] = mg
    return out


def render_backward(model: Model, rays_o, rays_d, d_rgb, tau, n_samples, d_depth=None,
                    d_wsum=None, dir_mode=DIR_REFLECT, bg=(0.0, 0.0, 0.0), t_samples=None,
                    n_threads=1, mlp_f16=False):
    """Gradients of sum(d_rgb*rgb + d_depth*depth + d_wsum*wsum) w.r.t. the
    SDF nodes, node features (or tile planes), probe coefficients and MLP
    parameters (mlp_f16 as in render_forward; the rounding is taken as the
    identity in the adjoint)."""
    lib = _load()
    o, d = _f32(rays_o).reshape(-1, 3), _f32(rays_d).reshape(-1, 3)
    n = o.shape[0]
    ts = None if t_samples is None else _f32(t_samples).reshape(n, n_samples + 1)
    drgb = _f64(d_rgb).reshape(n, 3)
    dd = None if d_depth is None else _f64(d_depth).reshape(n)
    dw = None if d_wsum is None else _f64(d_wsum).reshape(n)
    g_sdf = np.zeros_like(model.sdf)
    g_feat = np.zeros_like(model.feat if model.planes is None else model.planes)
    g_probe = np.zeros_like(model.probes)
    g_mlp = np.zeros_like(model.mlp)
    p = _params(tau, n_samples, dir_mode, bg, mlp_f16=mlp_f16)
    st = lib.orc_render_backward(ctypes.byref(model._s), ctypes.byref(p), n, _ptr(o), _ptr(d),
                                 _ptr(ts), _ptr(drgb), _ptr(dd), _ptr(dw), _ptr(g_sdf),
                                 _ptr(g_feat), _ptr(g_probe), _ptr(g_mlp), int(n_threads))
    if st != 0:
        raise ValueError(f"oracle backward rejected its arguments ({st})")
    return {"sdf": g_sdf, "feat": g_feat, "probes": g_probe, "mlp": g_mlp}


def shade_nodes(model: Model, camera, band, dir_mode=DIR_REFLECT):
    """Two-pass inference, first pass: the colour of every node seen from a
    camera at `camera` ([Rz,Ry,Rx,3]; nodes with |s| >= band are 0)."""
    lib = _load()
    out = np.zeros(model.sdf.shape + (3,))
    cam = _f64(camera).reshape(3)
    p = _params(1.0, 1, dir_mode)
    st = lib.orc_shade_nodes(ctypes.byref(model._s), ctypes.byref(p), _ptr(cam), float(band),
                             _ptr(out))
    if st != 0:
        raise ValueError(f"oracle shade_nodes rejected its arguments ({st})")
    return out


def shade_node_list(model: Model, camera, band, nodes, dir_mode=DIR_REFLECT):
    """shade_nodes for the listed linear node indices only -> [n, 3]."""
    lib = _load()
    idx = np.ascontiguousarray(nodes, dtype=np.int64).ravel()
    out = np.zeros((idx.size, 3))
    cam = _f64(camera).reshape(3)
    p = _params(1.0, 1, dir_mode)
    st = lib.orc_shade_node_list(ctypes.byref(model._s), ctypes.byref(p), _ptr(cam),
                                 float(band), idx.size, _ptr(idx), _ptr(out))
    if st != 0:
        raise ValueError(f"oracle shade_node_list rejected its arguments ({st})")
    return out


def render_colour_field(model: Model, colours, rays_o, rays_d, tau, n_samples,
                        bg=(0.0, 0.0, 0.0), t_samples=None):
    """Two-pass inference, second pass: the NeuS march with every sample's
    colour the trilinear blend of the node colours [Rz,Ry,Rx,3]."""
    lib = _load()
    o, d = _f32(rays_o).reshape(-1, 3), _f32(rays_d).reshape(-1, 3)
    n = o.shape[0]
    col = _f64(colours)
    assert col.shape == model.sdf.shape + (3,), "colours [Rz,Ry,Rx,3]"
    ts = None if t_samples is None else _f32(t_samples).reshape(n, n_samples + 1)
    rgb = np.zeros((n, 3))
    depth, wsum = np.zeros(n), np.zeros(n)
    p = _params(tau, n_samples, DIR_REFLECT, bg)
    st = lib.orc_render_colour_field(ctypes.byref(model._s), ctypes.byref(p), _ptr(col), n,
                                     _ptr(o), _ptr(d), _ptr(ts), _ptr(rgb), _ptr(depth),
                                     _ptr(wsum))
    if st != 0:
        raise ValueError(f"oracle render_colour_field rejected its arguments ({st})")
    return {"rgb": rgb, "depth": depth, "wsum": wsum}


def render_trace(model: Model, o, d, tau, n_samples, dir_mode=DIR_REFLECT, t_samples=None):
    """Per-sample detail of one ray: t[N+1], s[N+1], w[N], C[N,3], normal[N,3]."""
    lib = _load()
    o, d = _f32(o).reshape(3), _f32(d).reshape(3)
    ts = None if t_samples is None else _f32(t_samples).reshape(n_samples + 1)
    t = np.zeros(n_samples + 1, np.float32)
    s = np.zeros(n_samples + 1)
    w = np.zeros(n_samples)
    C = np.zeros((n_samples, 3))
    nrm = np.zeros((n_samples, 3))
    p = _params(tau, n_samples, dir_mode)
    hit = lib.orc_render_trace(ctypes.byref(model._s), ctypes.byref(p), _ptr(o), _ptr(d),
                               _ptr(ts), _ptr(t), _ptr(s), _ptr(w), _ptr(C), _ptr(nrm))
    if hit < 0:
        raise ValueError("oracle trace rejected its arguments")
    return {"hit": bool(hit), "t": t, "s": s, "w": w, "C": C, "normal": nrm}


def point_eval(model: Model, o, d, t, dir_mode=DIR_REFLECT, sdf_fp32=False, mlp_f16=False):
    """SDF value, gradient, MLP input vector and colour at the point o + t d
    (sdf_fp32: the SDF value rounded as the FP32 evaluation rounds it;
    mlp_f16: the MLP's layer inputs rounded to binary16, x returned rounded)."""
    lib = _load()
    o, d = _f32(o).reshape(3), _f32(d).reshape(3)
    s = np.zeros(1)
    g = np.zeros(3)
    x = np.zeros(model.n_s + model.n_a + model.n_fresnel)
    C = np.zeros(3)
    p = _params(1.0, 1, dir_mode, sdf_fp32=sdf_fp32, mlp_f16=mlp_f16)
    st = lib.orc_point_eval(ctypes.byref(model._s), ctypes.byref(p), _ptr(o), _ptr(d),
                            ctypes.c_float(t), _ptr(s), _ptr(g), _ptr(x), _ptr(C))
    if st != 0:
        raise ValueError("oracle point_eval rejected its arguments")
    return {"s": s[0], "g": g, "x": x, "C": C}


def round_f16(v):
    """Nearest binary16 value of each element (ties to even), as FP64."""
    lib = _load()
    v = np.asarray(v, np.float64)
    return np.array([lib.orc_round_f16(float(x)) for x in v.ravel()]).reshape(v.shape)


def sh_eval(l, r):
    lib = _load()
    r = _f64(r).reshape(3)
    Y = np.zeros(l * l)
    lib.orc_sh_eval(int(l), _ptr(r), _ptr(Y))
    return Y


def sh_grad(l, r):
    lib = _load()
    r = _f64(r).reshape(3)
    dY = np.zeros((l * l, 3))
    lib.orc_sh_grad(int(l), _ptr(r), _ptr(dY))
    return dY


# ----------------------------------------------------------------------------
# Learned sample proposal (not part of the paper)
# ----------------------------------------------------------------------------

class Proposal:
    """Oracle copy of a proposal network: occupancy [rz, ry, rx] and packed
    parameters W1[W][7+2B] b1 W2[W][W] b2 W3[B][W] b3, promoted to FP64."""

    def __init__(self, occ, params, width=32, n_bins=8, mix=0.1, theta=0.2, n_sub=8):
        self.occ = _f64(occ)
        self.params = _f64(params).ravel()
        rz, ry, rx = self.occ.shape
        nin = 7 + 2 * n_bins
        assert self.params.size == width * nin + width + width * width + width + n_bins * width + n_bins
        s = _Proposal()
        s.occ_res[:] = (rx, ry, rz)
        s.occ = self.occ.ctypes.data
        s.width = int(width)
        s.n_bins = int(n_bins)
        s.n_sub = int(n_sub)
        s.params = self.params.ctypes.data
        s.mix = float(mix)
        s.theta = float(theta)
        self._s = s
        self.n_bins = int(n_bins)


def occupancy(model: Model, res, threshold):
    """[rz, ry, rx] in {0, 1}: cells whose covered nodes reach |sdf| < threshold."""
    lib = _load()
    rx, ry, rz = (int(v) for v in res)
    out = np.zeros((rz, ry, rx))
    r = (ctypes.c_int32 * 3)(rx, ry, rz)
    st = lib.orc_occupancy(ctypes.byref(model._s), r, float(threshold), _ptr(out))
    if st != 0:
        raise ValueError("oracle occupancy rejected its arguments")
    return out


def proposal_forward(model: Model, prop: Proposal, rays_o, rays_d, n_out):
    """logits [n, B], mixed density p' [n, B], t_samples [n, n_out + 1] and
    margin [n]: the smallest |pre-activation| of a hidden unit per ray."""
    lib = _load()
    o, d = _f32(rays_o).reshape(-1, 3), _f32(rays_d).reshape(-1, 3)
    n = o.shape[0]
    B = prop.n_bins
    logits, probs = np.zeros((n, B)), np.zeros((n, B))
    t = np.zeros((n, n_out + 1))
    mg = np.zeros(n)
    st = lib.orc_proposal_forward(ctypes.byref(model._s), ctypes.byref(prop._s), n, _ptr(o),
                                  _ptr(d), int(n_out), _ptr(logits), _ptr(probs), _ptr(t),
                                  _ptr(mg))
    if st != 0:
        raise ValueError("oracle proposal_forward rejected its arguments")
    return {"logits": logits, "probs": probs, "t": t, "margin": mg}


def place_samples(model: Model, rays_o, rays_d, q, n_out):
    """[n, n_out + 1] distances at the quantiles of the per-bin densities q [n, B]
    over each ray's box segment (zeros for misses)."""
    lib = _load()
    o, d = _f32(rays_o).reshape(-1, 3), _f32(rays_d).reshape(-1, 3)
    n = o.shape[0]
    qq = _f64(q).reshape(n, -1)
    t = np.zeros((n, n_out + 1))
    st = lib.orc_place_samples(ctypes.byref(model._s), n, _ptr(o), _ptr(d), _ptr(qq),
                               qq.shape[1], int(n_out), _ptr(t))
    if st != 0:
        raise ValueError("oracle place_samples rejected its arguments")
    return t


def weight_histogram(model: Model, rays_o, rays_d, tau, n_samples, n_bins):
    """[n, n_bins] per-bin sums of the uniform render's weights."""
    lib = _load()
    o, d = _f32(rays_o).reshape(-1, 3), _f32(rays_d).reshape(-1, 3)
    n = o.shape[0]
    out = np.zeros((n, n_bins))
    p = _params(tau, n_samples)
    st = lib.orc_weight_histogram(ctypes.byref(model._s), ctypes.byref(p), n, _ptr(o), _ptr(d),
                                  int(n_bins), _ptr(out), 1)
    if st != 0:
        raise ValueError("oracle weight_histogram rejected its arguments")
    return out


def proposal_backward(model: Model, prop: Proposal, rays_o, rays_d, hist, min_mass, scale):
    """(gradient of scale * sum loss w.r.t. the parameters, per-ray loss
    -sum_b hist_b log p_b)."""
    lib = _load()
    o, d = _f32(rays_o).reshape(-1, 3), _f32(rays_d).reshape(-1, 3)
    n = o.shape[0]
    h = _f64(hist).reshape(n, prop.n_bins)
    g = np.zeros_like(prop.params)
    loss = np.zeros(n)
    st = lib.orc_proposal_backward(ctypes.byref(model._s), ctypes.byref(prop._s), n, _ptr(o),
                                   _ptr(d), _ptr(h), float(min_mass), float(scale), _ptr(g),
                                   _ptr(loss))
    if st != 0:
        raise ValueError("oracle proposal_backward rejected its arguments")
    return g, loss
