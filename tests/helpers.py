"""Shared test helpers: scene construction and parity metrics."""
import json
import os

import numpy as np

import oracle
import synth

# Parity tolerances of the FP32 path against the FP64 oracle.
RGB_DEPTH_RTOL = 1e-5     # |gpu - ref| <= 1e-5 * max(|ref|, REL_FLOOR), elementwise
REL_FLOOR = 1e-2          # outputs under 1% of the unit colour / weight scale are held
                          # to an absolute 1e-7 against the FP64 oracle ...
REL_FLOOR_S32 = 1e-3      # ... and to 1e-8 against the oracle whose SDF values are rounded
                          # as the FP32 evaluation rounds them (the rest FP64): what the
                          # 1e-2 floor allows beyond 1e-3 is that rounding, amplified by
                          # tau in the opacity of nearly transparent rays
GRAD_RTOL = 1e-4          # per tensor: max|g - g_ref| <= 1e-4 * max|g_ref|
KINK_MARGIN = 3e-5        # rays closer than this (relative) to a ReLU or alpha-clip
                          # kink are left out of gradient comparisons

THREADS = max(1, min(32, os.cpu_count() or 1))


def small_scene(name="sphere64", dims=None, probe_dims=None):
    return synth.make_scene(name, dims=dims, probe_dims=probe_dims)


def rel_err_elementwise(gpu, ref, floor=REL_FLOOR):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.max(np.abs(gpu - ref) / np.maximum(np.abs(ref), floor))) if ref.size else 0.0


def rel_err_tensor(gpu, ref):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = np.max(np.abs(ref)) if ref.size else 0.0
    if scale == 0.0:
        return float(np.max(np.abs(gpu))) if gpu.size else 0.0
    return float(np.max(np.abs(gpu - ref)) / scale)


def oracle_forward(sc, o, d, tau, n_samples, **kw):
    m = oracle.Model.from_scene(sc)
    return oracle.render_forward(m, o, d, tau, n_samples, n_threads=THREADS, **kw)


def oracle_backward(sc, o, d, drgb, tau, n_samples, **kw):
    m = oracle.Model.from_scene(sc)
    return oracle.render_backward(m, o, d, drgb, tau, n_samples, n_threads=THREADS, **kw)


def clean_rays(sc, o, d, tau, n_samples, margin=KINK_MARGIN, **kw):
    """Indices of rays whose every ReLU / alpha-clip decision is at least
    `margin` (relative) away from its kink: there both precisions take the same
    branch, so their gradients are comparable."""
    out = oracle_forward(sc, o, d, tau, n_samples, margin=True, **kw)
    return np.nonzero(out["margin"] > margin)[0]


def packed_to_dense_grad(g_packed, dims):
    """[R^3, 4] packed gradient -> (sdf [Rz,Ry,Rx], feat [Rz,Ry,Rx,3])."""
    Rx, Ry, Rz = dims
    g = np.asarray(g_packed).reshape(Rz, Ry, Rx, 4)
    return g[..., 0], g[..., 1:]


def worst(gpu, ref, floor=REL_FLOOR):
    """(index, gpu value, reference value) of the largest elementwise error."""
    gpu = np.asarray(gpu, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    i = int(np.argmax(np.abs(gpu - ref) / np.maximum(np.abs(ref), floor)))
    return i, float(gpu[i]), float(ref[i])


def log_errors(test, errs):
    """Appends measured errors to $PSDF_PARITY_LOG (JSON lines) if it is set."""
    path = os.environ.get("PSDF_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"test": test, **errs}) + "\n")


def box_interval(o, d, bmin, bmax):
    """FP64 slab test: (t_near, t_far, hit) per ray."""
    o = np.asarray(o, np.float64)
    d = np.asarray(d, np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        t0 = (np.asarray(bmin, np.float64) - o) / d
        t1 = (np.asarray(bmax, np.float64) - o) / d
    tn = np.max(np.minimum(t0, t1), axis=1)
    tf = np.min(np.maximum(t0, t1), axis=1)
    tn = np.maximum(tn, 0.0)
    return tn, tf, tf > tn
