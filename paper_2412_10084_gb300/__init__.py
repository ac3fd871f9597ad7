"""GB300 (sm_103a) ProbeSDF per-ray render and adjoint.

A thin ctypes binding over ``libprobesdf.so`` (C ABI in include/probesdf.h):
argument marshalling only, every step of the render and its adjoint runs in
the library's CUDA kernels.  PyTorch provides device memory and streams.

There is no CPU fallback: if the library cannot be built or loaded, or no
CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading

import torch

from . import build as _build

__all__ = [
    "GridDesc", "ProbeDesc", "MlpDesc", "RenderParams", "Scene", "LibraryError",
    "library", "grid_bytes", "mlp_param_count", "pack_grid", "unpack_grid", "BF16", "F16", "F32",
    "FEAT_NODES", "FEAT_TRIPLANE", "tri_tiles",
    "render_forward", "render_backward", "render", "device_status", "set_wait_polls",
    "wait_polls", "DIR_REFLECT", "DIR_VIEW",
    "ProposalDesc", "proposal_desc", "proposal_param_count", "occupancy_build",
    "weight_histogram", "proposal_forward", "proposal_backward", "adam_step", "Adam",
    "occupancy_words", "occupancy_unpack", "sdf_smooth", "sdf_smooth_adjoint",
    "grid_regularizers", "probe_smoothness", "shade_nodes", "render_colour_field",
    "colour_field_bytes", "brick_table", "pack_sparse", "table_words", "sparse_scene",
]

DIR_REFLECT = 0
DIR_VIEW = 1
F32 = 0
BF16 = 1
F16 = 2
GRID_VALUES = 0
GRID_GRAD = 1
FEAT_NODES = 0
FEAT_TRIPLANE = 1
TILE = 16


def tri_tiles(dims):
    """Tiles of 16 cells along x, y, z of a grid with `dims` nodes."""
    return tuple((int(r) - 1 + TILE - 1) // TILE for r in dims)


class LibraryError(RuntimeError):
    pass


class GridDesc(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32 * 3), ("box_min", ctypes.c_float * 3),
                ("box_max", ctypes.c_float * 3), ("n_feat", ctypes.c_int32),
                ("feat_dtype", ctypes.c_int32), ("feat_layout", ctypes.c_int32),
                ("n_bricks", ctypes.c_int32), ("empty_sdf", ctypes.c_float)]


class ProbeDesc(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32 * 3), ("sh_l", ctypes.c_int32),
                ("n_ang", ctypes.c_int32), ("dtype", ctypes.c_int32)]


class MlpDesc(ctypes.Structure):
    _fields_ = [("n_in", ctypes.c_int32), ("width", ctypes.c_int32), ("dtype", ctypes.c_int32)]


class RenderParams(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_float), ("n_samples", ctypes.c_int32),
                ("dir_mode", ctypes.c_int32), ("n_fresnel", ctypes.c_int32),
                ("bg", ctypes.c_float * 3), ("n_bins", ctypes.c_int32)]


class ProposalDesc(ctypes.Structure):
    _fields_ = [("occ_res", ctypes.c_int32 * 3), ("n_bins", ctypes.c_int32),
                ("width", ctypes.c_int32), ("n_sub", ctypes.c_int32), ("mix", ctypes.c_float),
                ("theta", ctypes.c_float)]


_lock = threading.Lock()
_lib = None
_P = ctypes.c_void_p


def library() -> ctypes.CDLL:
    """Load (building first if needed) libprobesdf.so and declare its ABI."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build()
        lib = ctypes.CDLL(path)
        lib.psdf_status_string.restype = ctypes.c_char_p
        lib.psdf_status_string.argtypes = [ctypes.c_int32]
        lib.psdf_last_cuda_error.restype = ctypes.c_int32
        lib.psdf_version.restype = ctypes.c_int32
        lib.psdf_device_status.argtypes = [_P, ctypes.POINTER(ctypes.c_int32)]
        lib.psdf_device_status.restype = ctypes.c_int32
        lib.psdf_set_wait_polls.argtypes = [ctypes.c_uint32]
        lib.psdf_set_wait_polls.restype = ctypes.c_int32
        lib.psdf_wait_polls.restype = ctypes.c_uint32
        lib.psdf_grid_bytes.argtypes = [_P, ctypes.POINTER(ctypes.c_size_t),
                                         ctypes.POINTER(ctypes.c_size_t)]
        lib.psdf_grid_create.argtypes = [_P, _P, ctypes.POINTER(_P)]
        lib.psdf_grid_destroy.argtypes = [_P]
        lib.psdf_grid_destroy.restype = None
        lib.psdf_grid_pack.argtypes = [_P, _P, _P, _P, _P]
        lib.psdf_grid_unpack.argtypes = [_P, ctypes.c_int32, _P, _P, _P, _P]
        lib.psdf_probes_create.argtypes = [_P, _P, ctypes.POINTER(_P)]
        lib.psdf_probes_destroy.argtypes = [_P]
        lib.psdf_probes_destroy.restype = None
        lib.psdf_mlp_param_count.argtypes = [_P, ctypes.POINTER(ctypes.c_int64)]
        lib.psdf_mlp_create.argtypes = [_P, _P, ctypes.POINTER(_P)]
        lib.psdf_mlp_destroy.argtypes = [_P]
        lib.psdf_mlp_destroy.restype = None
        lib.psdf_render_forward.argtypes = [_P, _P, _P, _P, _P, _P, _P, ctypes.c_int64,
                                            _P, _P, _P, _P, _P, _P]
        lib.psdf_render_backward.argtypes = [_P, _P, _P, _P, _P, _P, _P, ctypes.c_int64,
                                             _P, _P, _P, _P, _P, _P, _P, _P, _P]
        lib.psdf_render_occupancy.argtypes = [_P, _P, _P, _P, ctypes.POINTER(ctypes.c_int32),
                                              ctypes.POINTER(ctypes.c_int32)]
        lib.psdf_adam_step.argtypes = [_P, _P, _P, _P, ctypes.c_int64, ctypes.c_float,
                                       ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                       ctypes.c_int32, ctypes.c_int32, _P]
        lib.psdf_proposal_param_count.argtypes = [_P, ctypes.POINTER(ctypes.c_int64)]
        lib.psdf_occupancy_words.argtypes = [_P, ctypes.POINTER(ctypes.c_int64)]
        lib.psdf_occupancy_build.argtypes = [_P, _P, ctypes.c_float, _P, _P]
        lib.psdf_weight_histogram.argtypes = [_P, _P, _P, _P, ctypes.c_int64, ctypes.c_int32,
                                              _P, _P]
        lib.psdf_proposal_forward.argtypes = [_P, _P, _P, _P, _P, _P, ctypes.c_int64,
                                              ctypes.c_int32, _P, _P, _P]
        lib.psdf_proposal_backward.argtypes = [_P, _P, _P, _P, _P, _P, ctypes.c_int64, _P,
                                               ctypes.c_float, ctypes.c_float, _P, _P, _P]
        lib.psdf_sdf_smooth.argtypes = [_P, _P, _P, _P]
        lib.psdf_sdf_smooth_adjoint.argtypes = [_P, _P, _P, ctypes.c_int32, _P]
        lib.psdf_grid_regularizers.argtypes = [_P, _P, _P, ctypes.c_float, ctypes.c_float,
                                               ctypes.c_float, ctypes.c_float, _P, _P, _P, _P]
        lib.psdf_probe_smoothness.argtypes = [_P, _P, ctypes.c_float, _P, _P, _P]
        lib.psdf_colour_field_bytes.argtypes = [_P, ctypes.POINTER(ctypes.c_size_t)]
        lib.psdf_shade_nodes.argtypes = [_P, _P, _P, _P, _P, ctypes.c_float, _P, _P]
        lib.psdf_render_colour_field.argtypes = [_P, _P, _P, _P, _P, _P, ctypes.c_int64, _P, _P,
                                                 _P, _P]
        for name in ("psdf_colour_field_bytes", "psdf_shade_nodes", "psdf_render_colour_field",
                     "psdf_sdf_smooth", "psdf_sdf_smooth_adjoint", "psdf_grid_regularizers",
                     "psdf_probe_smoothness", "psdf_grid_bytes", "psdf_grid_create", "psdf_grid_pack", "psdf_grid_unpack",
                     "psdf_probes_create", "psdf_mlp_param_count", "psdf_mlp_create",
                     "psdf_render_forward", "psdf_render_backward", "psdf_render_occupancy",
                     "psdf_adam_step", "psdf_proposal_param_count", "psdf_occupancy_words",
                     "psdf_occupancy_build", "psdf_weight_histogram",
                     "psdf_proposal_forward", "psdf_proposal_backward"):
            getattr(lib, name).restype = ctypes.c_int32
        _lib = lib
        return lib


def _check(status: int, what: str):
    if status != 0:
        lib = library()
        msg = lib.psdf_status_string(status).decode()
        extra = ""
        if status == -5:
            extra = f" (cudaError {lib.psdf_last_cuda_error()})"
        raise LibraryError(f"{what}: {msg}{extra}")


def device_status(stream=None) -> int:
    """Synchronises the stream, then reads and clears the device status word
    (0 = no kernel gave up waiting on its tensor-core work)."""
    flags = ctypes.c_int32()
    _check(library().psdf_device_status(_stream(stream), ctypes.byref(flags)),
           "psdf_device_status")
    return flags.value


def set_wait_polls(polls=None):
    """Polls of each tensor-core completion wait in the kernels this thread
    launches next (None: the default).  A small value makes the waits run out
    on purpose: the kernels then stop early, set bit 0 of the device status
    word and free their tensor memory; their outputs are invalid."""
    _check(library().psdf_set_wait_polls(0xFFFFFFFF if polls is None else int(polls)),
           "psdf_set_wait_polls")


def wait_polls() -> int:
    return int(library().psdf_wait_polls())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _require_cuda(*tensors, dtypes=(torch.float32,)):
    for t in tensors:
        if t is not None:
            if not t.is_cuda:
                raise LibraryError("tensors must be on a CUDA device (there is no CPU path)")
            if t.dtype not in dtypes:
                raise LibraryError(f"expected {dtypes}, got {t.dtype}")
            if not t.is_contiguous():
                raise LibraryError("tensors must be contiguous")


def grid_desc(dims, box_min, box_max, n_feat=3, feat_dtype=F32,
              feat_layout=FEAT_NODES, n_bricks=0, empty_sdf=1.0) -> GridDesc:
    """n_bricks > 0: a sparse grid of 16^3-node bricks of which n_bricks are
    stored (the others read as SDF empty_sdf, features 0)."""
    d = GridDesc()
    d.n_bricks = int(n_bricks)
    d.empty_sdf = float(empty_sdf)
    d.feat_layout = int(feat_layout)
    d.dims[:] = tuple(int(v) for v in dims)
    d.box_min[:] = tuple(float(v) for v in box_min)
    d.box_max[:] = tuple(float(v) for v in box_max)
    d.n_feat = int(n_feat)
    d.feat_dtype = int(feat_dtype)
    return d


def grid_bytes(desc: GridDesc):
    """(packed value bytes, gradient bytes) of a grid."""
    n, g = ctypes.c_size_t(), ctypes.c_size_t()
    _check(library().psdf_grid_bytes(ctypes.byref(desc), ctypes.byref(n), ctypes.byref(g)),
           "psdf_grid_bytes")
    return n.value, g.value


def mlp_param_count(n_in: int, width: int) -> int:
    d = MlpDesc(n_in, width, F32)
    n = ctypes.c_int64()
    _check(library().psdf_mlp_param_count(ctypes.byref(d), ctypes.byref(n)),
           "psdf_mlp_param_count")
    return n.value


def brick_table(keep) -> torch.Tensor:
    """int32 [Bz, By, Bx] brick table from a boolean brick mask: the kept
    bricks get slots 0, 1, ... in x-fastest order, the others -1."""
    keep = torch.as_tensor(keep, dtype=torch.bool)
    flat = keep.reshape(-1)
    table = torch.full(flat.shape, -1, dtype=torch.int32)
    table[flat] = torch.arange(int(flat.sum()), dtype=torch.int32)
    return table.reshape(keep.shape)


def table_words(desc: GridDesc) -> int:
    """float32 words in front of a sparse grid's brick records (the table)."""
    nb = (desc.dims[0] // TILE) * (desc.dims[1] // TILE) * (desc.dims[2] // TILE)
    return ((4 * nb + 15) // 16) * 4


def pack_sparse(desc: GridDesc, table, sdf: torch.Tensor, feat: torch.Tensor) -> torch.Tensor:
    """Sparse grid from dense sdf [Rz,Ry,Rx] + feat [Rz,Ry,Rx,3] and a brick
    table [Bz,By,Bx] (slots 0..n_bricks-1 or -1): packed float32 [bytes/16, 4]."""
    nbytes, _ = grid_bytes(desc)
    shape = tuple(int(desc.dims[a]) // TILE for a in (2, 1, 0))
    tab = torch.as_tensor(table, dtype=torch.int32)
    if tuple(tab.shape) != shape:
        raise LibraryError(f"pack_sparse: the brick table must be {shape} (Bz, By, Bx), "
                           f"got {tuple(tab.shape)}")
    slots = tab[tab >= 0]
    if slots.numel() > desc.n_bricks or slots.unique().numel() != slots.numel():
        # a slot named twice would alias one record block (racing pack writes,
        # two bricks' gradients added into one)
        raise LibraryError(f"pack_sparse: the brick table names {slots.numel()} slots "
                           f"({slots.unique().numel()} distinct) for {desc.n_bricks} stored "
                           f"bricks; each slot may appear at most once")
    _require_cuda(sdf, feat)
    out = torch.zeros(nbytes // 4, dtype=torch.float32, device=sdf.device)
    tab = tab.reshape(-1).to(sdf.device)
    out[:tab.numel()] = tab.view(torch.float32)
    out = out.view(-1, 4)
    _check(library().psdf_grid_pack(ctypes.byref(desc), _ptr(sdf), _ptr(feat), _ptr(out),
                                    _stream()), "psdf_grid_pack")
    return out


def pack_grid(desc: GridDesc, sdf: torch.Tensor, feat: torch.Tensor) -> torch.Tensor:
    """Dense sdf [Rz,Ry,Rx] + feat [Rz,Ry,Rx,3] (or tile planes
    [tz,ty,tx,3,16,16,3]) (device FP32) -> packed values: float32 [R^3, 4] for
    FP32 node features, [bytes/16, 4] for tri-planes, a uint8 buffer for BF16."""
    _require_cuda(sdf, feat)
    if desc.n_bricks > 0:
        raise LibraryError("pack_grid: a sparse grid needs its brick table (pack_sparse)")
    nbytes, _ = grid_bytes(desc)
    if desc.feat_layout == FEAT_TRIPLANE:
        out = torch.empty(nbytes // 4, dtype=torch.float32, device=sdf.device).view(-1, 4)
    elif desc.feat_dtype == F32:
        out = torch.empty(nbytes // 4, dtype=torch.float32, device=sdf.device).view(-1, 4)
    else:
        out = torch.empty(nbytes, dtype=torch.uint8, device=sdf.device)
    _check(library().psdf_grid_pack(ctypes.byref(desc), _ptr(sdf), _ptr(feat), _ptr(out),
                                    _stream()), "psdf_grid_pack")
    return out


def unpack_grid(desc: GridDesc, packed: torch.Tensor, which: int = None):
    """Packed values or a gradient buffer -> (sdf [Rz,Ry,Rx], feat [Rz,Ry,Rx,3]).
    `which` defaults to values for a uint8 buffer or when the layout is FP32,
    and must be GRID_GRAD for a float32 gradient of a BF16-feature grid."""
    _require_cuda(packed, dtypes=(torch.float32, torch.uint8))
    if which is None:
        which = GRID_VALUES if (packed.dtype == torch.uint8 or desc.feat_dtype == F32) \
            else GRID_GRAD
    Rx, Ry, Rz = desc.dims
    sdf = torch.empty((Rz, Ry, Rx), dtype=torch.float32, device=packed.device)
    if desc.feat_layout == FEAT_TRIPLANE:
        tx, ty, tz = tri_tiles(desc.dims)
        feat = torch.empty((tz, ty, tx, 3, TILE, TILE, desc.n_feat), dtype=torch.float32,
                           device=packed.device)
    else:
        feat = torch.empty((Rz, Ry, Rx, desc.n_feat), dtype=torch.float32, device=packed.device)
    _check(library().psdf_grid_unpack(ctypes.byref(desc), int(which), _ptr(packed), _ptr(sdf),
                                      _ptr(feat), _stream()), "psdf_grid_unpack")
    return sdf, feat


@dataclasses.dataclass
class Scene:
    """Device-resident parameters: packed grid [R^3,4], probes
    [Pz,Py,Px,l*l,n_a] and the packed MLP vector, with their descriptors."""
    grid: torch.Tensor
    probes: torch.Tensor
    mlp: torch.Tensor
    dims: tuple
    box_min: tuple
    box_max: tuple
    sh_l: int
    width: int
    n_feat: int = 3
    feat_dtype: int = F32    # storage of the spatial features (F32 or BF16)
    feat_layout: int = FEAT_NODES  # node features or tile tri-planes
    probe_dtype: int = F32   # storage of the probe coefficients (F32 or F16)
    mlp_dtype: int = F32     # MLP arithmetic (F32-equivalent or F16)
    n_bricks: int = 0        # sparse grid: stored 16^3-node bricks (0: dense)
    empty_sdf: float = 1.0   # sparse grid: SDF of the bricks not stored

    @property
    def probe_dims(self):
        Pz, Py, Px = self.probes.shape[:3]
        return (Px, Py, Pz)

    @property
    def n_ang(self):
        return self.probes.shape[-1]

    def descs(self, n_fresnel):
        gd = grid_desc(self.dims, self.box_min, self.box_max, self.n_feat, self.feat_dtype,
                       self.feat_layout, self.n_bricks, self.empty_sdf)
        pd = ProbeDesc()
        pd.dims[:] = self.probe_dims
        pd.sh_l = self.sh_l
        pd.n_ang = self.n_ang
        pd.dtype = self.probe_dtype
        md = MlpDesc(self.n_feat + self.n_ang + n_fresnel, self.width, self.mlp_dtype)
        return gd, pd, md

    def grad_buffers(self):
        """Zeroed FP32 gradient buffers: the grid's in its packed gradient
        layout ([R^3, 4] node records; a sparse grid's starts with a copy of
        the brick table), probes, MLP."""
        gd, _, _ = self.descs(3)
        _, gbytes = grid_bytes(gd)
        dev = self.mlp.device
        gg = torch.zeros(gbytes // 16, 4, dtype=torch.float32, device=dev)
        if self.n_bricks > 0:  # the gradient buffer carries the table too (for unpacking)
            w = table_words(gd)
            gg.view(-1)[:w] = self.grid.view(-1)[:w]
        return (gg,
                torch.zeros(self.probes.shape, dtype=torch.float32, device=dev),
                torch.zeros_like(self.mlp))

    @classmethod
    def from_host(cls, sc, device="cuda", feat_dtype=F32, probe_dtype=F32, mlp_dtype=F32,
                  bricks=None, empty_sdf=1.0):
        """Upload a synth.Scene-like object (numpy arrays) and pack its grid in
        the requested storage precision; `bricks` (a boolean [Bz,By,Bx] mask of
        16^3-node bricks to keep) makes it a sparse grid."""
        dev = torch.device(device)
        sdf = torch.as_tensor(sc.sdf, dtype=torch.float32, device=dev).contiguous()
        planes = getattr(sc, "planes", None)
        layout = FEAT_NODES if planes is None else FEAT_TRIPLANE
        feat = torch.as_tensor(sc.feat if planes is None else planes, dtype=torch.float32,
                               device=dev).contiguous()
        n_feat = int(feat.shape[-1])
        n_bricks = 0
        if bricks is not None:
            table = brick_table(bricks)
            n_bricks = int((table >= 0).sum())
            gd = grid_desc(sc.dims, sc.box_min, sc.box_max, n_feat, feat_dtype, layout,
                           n_bricks, empty_sdf)
            grid = pack_sparse(gd, table, sdf, feat)
        else:
            gd = grid_desc(sc.dims, sc.box_min, sc.box_max, n_feat, feat_dtype, layout)
            grid = pack_grid(gd, sdf, feat)
        probes = torch.as_tensor(sc.probes, dtype=torch.float32, device=dev)
        if probe_dtype == F16:
            probes = probes.half()
        mlp = torch.as_tensor(sc.mlp, dtype=torch.float32, device=dev).contiguous()
        return cls(grid=grid, probes=probes.contiguous(), mlp=mlp, dims=tuple(sc.dims),
                   box_min=tuple(float(v) for v in sc.box_min),
                   box_max=tuple(float(v) for v in sc.box_max), sh_l=int(sc.sh_l),
                   width=int(sc.width), n_feat=n_feat, feat_dtype=feat_dtype,
                   probe_dtype=probe_dtype, mlp_dtype=mlp_dtype, feat_layout=layout,
                   n_bricks=n_bricks, empty_sdf=float(empty_sdf))


def sparse_scene(keep, brick_sdf, brick_feat, probes, mlp, dims, box_min, box_max, sh_l,
                 width, empty_sdf=1.0, device="cuda") -> Scene:
    """Scene over a sparse grid given brick by brick: keep [Bz,By,Bx] (bool),
    brick_sdf [n,16,16,16] and brick_feat [n,16,16,16,3] (FP32, bricks in the
    x-fastest order of `keep`).  The packed buffer is assembled with tensor
    copies: the table, then one {sdf, f0, f1, f2} record per stored node."""
    dev = torch.device(device)
    table = brick_table(keep)
    shape = tuple(int(dims[a]) // TILE for a in (2, 1, 0))
    if tuple(table.shape) != shape:
        raise LibraryError(f"sparse_scene: keep must be {shape} (Bz, By, Bx), "
                           f"got {tuple(table.shape)}")
    n = int((table >= 0).sum())
    gd = grid_desc(dims, box_min, box_max, 3, F32, FEAT_NODES, n, empty_sdf)
    nbytes, _ = grid_bytes(gd)
    out = torch.empty(nbytes // 4, dtype=torch.float32, device=dev)
    w = table_words(gd)
    out[:w] = 0.0
    out[:table.numel()] = table.reshape(-1).to(dev).view(torch.float32)
    rec = out[w:].view(n * 4096, 4)
    rec[:, 0] = torch.as_tensor(brick_sdf, device=dev).reshape(-1)
    rec[:, 1:] = torch.as_tensor(brick_feat, device=dev).reshape(-1, 3)
    return Scene(grid=out.view(-1, 4),
                 probes=torch.as_tensor(probes, dtype=torch.float32, device=dev).contiguous(),
                 mlp=torch.as_tensor(mlp, dtype=torch.float32, device=dev).contiguous(),
                 dims=tuple(int(v) for v in dims), box_min=tuple(float(v) for v in box_min),
                 box_max=tuple(float(v) for v in box_max), sh_l=int(sh_l), width=int(width),
                 n_feat=3, n_bricks=n, empty_sdf=float(empty_sdf))


def render_params(tau=64.0, n_samples=128, dir_mode=DIR_REFLECT, n_fresnel=3,
                  bg=(0.0, 0.0, 0.0), n_bins=0) -> RenderParams:
    """n_bins > 0: the render's t_samples argument holds [n, n_bins] bin
    densities (samples at their quantiles) instead of distances."""
    p = RenderParams()
    p.n_bins = int(n_bins)
    p.tau = float(tau)
    p.n_samples = int(n_samples)
    p.dir_mode = int(dir_mode)
    p.n_fresnel = int(n_fresnel)
    p.bg[:] = tuple(float(v) for v in bg)
    return p


class _Handles:
    """Short-lived C handles over the scene's current device pointers."""

    def __init__(self, grid, probes, mlp, gd, pd, md):
        lib = library()
        self.g, self.p, self.m = _P(), _P(), _P()
        _check(lib.psdf_grid_create(ctypes.byref(gd), _ptr(grid), ctypes.byref(self.g)),
               "psdf_grid_create")
        _check(lib.psdf_probes_create(ctypes.byref(pd), _ptr(probes), ctypes.byref(self.p)),
               "psdf_probes_create")
        _check(lib.psdf_mlp_create(ctypes.byref(md), _ptr(mlp), ctypes.byref(self.m)),
               "psdf_mlp_create")

    def close(self):
        lib = library()
        lib.psdf_grid_destroy(self.g)
        lib.psdf_probes_destroy(self.p)
        lib.psdf_mlp_destroy(self.m)


def render_forward(scene: Scene, rays_o, rays_d, params: RenderParams, t_samples=None,
                   grid=None, probes=None, mlp=None, want_live=False):
    """-> rgb [n,3], depth [n], wsum [n], logT_final [n] (device FP32), and
    with want_live n_live [n] (int32: 1 + the last sample with a nonzero
    opacity), which lets render_backward skip the samples after it."""
    grid = scene.grid if grid is None else grid
    probes = scene.probes if probes is None else probes
    mlp = scene.mlp if mlp is None else mlp
    _require_cuda(grid, probes, mlp, dtypes=(torch.float32, torch.float16, torch.uint8))
    _require_cuda(rays_o, rays_d, t_samples)
    n = rays_o.shape[0]
    dev = rays_o.device
    rgb = torch.empty((n, 3), dtype=torch.float32, device=dev)
    depth = torch.empty(n, dtype=torch.float32, device=dev)
    wsum = torch.empty(n, dtype=torch.float32, device=dev)
    logT = torch.empty(n, dtype=torch.float32, device=dev)
    live = torch.empty(n, dtype=torch.int32, device=dev) if want_live else None
    gd, pd, md = scene.descs(params.n_fresnel)
    h = _Handles(grid, probes, mlp, gd, pd, md)
    try:
        _check(library().psdf_render_forward(h.g, h.p, h.m, ctypes.byref(params), _ptr(rays_o),
                                             _ptr(rays_d), _ptr(t_samples), n, _ptr(rgb),
                                             _ptr(depth), _ptr(wsum), _ptr(logT), _ptr(live),
                                             _stream()),
               "psdf_render_forward")
    finally:
        h.close()
    if want_live:
        return rgb, depth, wsum, logT, live
    return rgb, depth, wsum, logT


def render_backward(scene: Scene, rays_o, rays_d, params: RenderParams, d_rgb, logT,
                    d_depth=None, d_wsum=None, t_samples=None, grads=None, grid=None,
                    probes=None, mlp=None, n_live=None):
    """Accumulates into (and returns) grad_grid [R^3,4], grad_probes, grad_mlp.
    n_live: the forward's per-ray live extent (optional)."""
    grid = scene.grid if grid is None else grid
    probes = scene.probes if probes is None else probes
    mlp = scene.mlp if mlp is None else mlp
    _require_cuda(grid, probes, mlp, dtypes=(torch.float32, torch.float16, torch.uint8))
    _require_cuda(rays_o, rays_d, t_samples, d_rgb, d_depth, d_wsum, logT)
    _require_cuda(n_live, dtypes=(torch.int32,))
    if grads is None:
        grads = scene.grad_buffers()
    _require_cuda(*grads)
    gg, gp, gm = grads
    gd, pd, md = scene.descs(params.n_fresnel)
    h = _Handles(grid, probes, mlp, gd, pd, md)
    try:
        _check(library().psdf_render_backward(
            h.g, h.p, h.m, ctypes.byref(params), _ptr(rays_o), _ptr(rays_d), _ptr(t_samples),
            rays_o.shape[0], _ptr(d_rgb), _ptr(d_depth), _ptr(d_wsum), _ptr(logT), _ptr(n_live),
            _ptr(gg), _ptr(gp), _ptr(gm), _stream()), "psdf_render_backward")
    finally:
        h.close()
    return gg, gp, gm


def render_occupancy(scene: Scene, params: RenderParams):
    """(forward, backward) resident CTAs per SM of the render kernels."""
    gd, pd, md = scene.descs(params.n_fresnel)
    h = _Handles(scene.grid, scene.probes, scene.mlp, gd, pd, md)
    f, b = ctypes.c_int32(), ctypes.c_int32()
    try:
        _check(library().psdf_render_occupancy(h.g, h.p, h.m, ctypes.byref(params),
                                               ctypes.byref(f), ctypes.byref(b)),
               "psdf_render_occupancy")
    finally:
        h.close()
    return f.value, b.value


class RenderFunction(torch.autograd.Function):
    """Differentiable render: (grid, probes, mlp) -> (rgb, depth, wsum).

    grid_p / probes_p are the differentiable FP32 parameters: the storage
    tensors themselves for FP32 storage, or FP32 master copies ([R^3, 4]
    records and [Pz,Py,Px,l*l,n_a]) when the scene stores BF16 features or
    FP16 probes; the kernels read the scene's storage either way.  The
    backward recomputes per-sample activations in the library's adjoint
    kernel; only log T_N and the live extent per ray are saved.  With
    check_status (the default) the backward synchronises the stream and
    raises if a render kernel stopped early, instead of handing on partial
    gradients."""

    @staticmethod
    def forward(ctx, grid_p, probes_p, mlp, rays_o, rays_d, t_samples, scene, params,
                check_status=True):
        grid = grid_p if scene.feat_dtype == F32 else scene.grid
        probes = probes_p if scene.probe_dtype == F32 else scene.probes
        rgb, depth, wsum, logT, live = render_forward(scene, rays_o, rays_d, params, t_samples,
                                                      grid=grid, probes=probes, mlp=mlp,
                                                      want_live=True)
        ctx.save_for_backward(mlp, rays_o, rays_d, logT, live,
                              t_samples if t_samples is not None else torch.empty(0))
        ctx.storage = (grid, probes)
        ctx.has_t = t_samples is not None
        ctx.scene = scene
        ctx.params = params
        ctx.check_status = check_status
        ctx.mark_non_differentiable(logT, live)
        return rgb, depth, wsum

    @staticmethod
    def backward(ctx, d_rgb, d_depth, d_wsum):
        mlp, rays_o, rays_d, logT, live, t_samples = ctx.saved_tensors
        grid, probes = ctx.storage
        t_samples = t_samples if ctx.has_t else None
        d_rgb = torch.zeros((rays_o.shape[0], 3), dtype=torch.float32, device=rays_o.device) \
            if d_rgb is None else d_rgb.contiguous()
        d_depth = None if d_depth is None else d_depth.contiguous()
        d_wsum = None if d_wsum is None else d_wsum.contiguous()
        gg, gp, gm = render_backward(ctx.scene, rays_o, rays_d, ctx.params, d_rgb, logT,
                                     d_depth=d_depth, d_wsum=d_wsum, t_samples=t_samples,
                                     grid=grid, probes=probes, mlp=mlp, n_live=live)
        if ctx.scene.n_bricks > 0:
            # a sparse grid's brick table is not a parameter: zero gradient there
            # (the buffer came with a copy of the table bits, which are no gradient)
            gg.view(-1)[:table_words(ctx.scene.descs(ctx.params.n_fresnel)[0])] = 0.0
        if ctx.check_status:
            flags = device_status()
            if flags:
                raise LibraryError(f"render: a render kernel stopped early (device status "
                                   f"{flags:#x}); its outputs and gradients are incomplete")
        return gg, gp, gm, None, None, None, None, None, None


def render(scene: Scene, rays_o, rays_d, params: RenderParams, t_samples=None, masters=None,
           check_status=True):
    """Differentiable w.r.t. the scene's FP32 parameters: scene.grid,
    scene.probes and scene.mlp, or, for reduced-precision storage, the FP32
    masters=(grid [R^3,4], probes) that the storage was packed from.  On a
    sparse grid the brick table at the front of scene.grid gets zero gradient;
    keep it out of any update that changes parameters without a gradient
    (weight decay).  check_status: the backward checks the device status word
    (a stream synchronisation) and raises if a render kernel stopped early."""
    grid_p, probes_p = (scene.grid, scene.probes) if masters is None else masters
    return RenderFunction.apply(grid_p, probes_p, scene.mlp, rays_o, rays_d, t_samples, scene,
                                params, check_status)


# ---------------------------------------------------------------------------
# Optimiser (Adam, Sec. 3.4)
# ---------------------------------------------------------------------------

def adam_step(param, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, clear_grad=True):
    """One in-place Adam update of a FP32 tensor (bias-corrected; `step` from 1)."""
    _require_cuda(param, grad, m, v)
    n = param.numel()
    if grad.numel() != n or m.numel() != n or v.numel() != n:
        raise LibraryError("adam_step: param, grad, m and v must have the same size")
    _check(library().psdf_adam_step(_ptr(param), _ptr(grad), _ptr(m), _ptr(v), n, float(lr),
                                    float(beta1), float(beta2), float(eps), int(step),
                                    int(bool(clear_grad)), _stream()), "psdf_adam_step")


class Adam:
    """Adam over a list of (param, grad, lr) FP32 device tensors; the moments
    live beside them.  step() updates every parameter and clears its grad."""

    def __init__(self, groups, beta1=0.9, beta2=0.999, eps=1e-8):
        self.groups = [(p, g, float(lr), torch.zeros_like(p), torch.zeros_like(p))
                       for p, g, lr in groups]
        self.beta1, self.beta2, self.eps = beta1, beta2, eps
        self.t = 0

    def step(self):
        self.t += 1
        for p, g, lr, m, v in self.groups:
            adam_step(p, g, m, v, self.t, lr, self.beta1, self.beta2, self.eps)


# ---------------------------------------------------------------------------
# Two-pass inference: per-view node colours, then a colour-field march
# ---------------------------------------------------------------------------

def colour_field_bytes(gd) -> int:
    n = ctypes.c_size_t()
    _check(library().psdf_colour_field_bytes(ctypes.byref(gd), ctypes.byref(n)),
           "psdf_colour_field_bytes")
    return n.value


def shade_nodes(scene: Scene, camera, band, params: RenderParams, out=None):
    """Colour of every grid node seen from `camera` (3 floats, world units):
    FP16 [Rz, Ry, Rx, 4] = {r, g, b, 0}; nodes with |s| >= band are 0."""
    _require_cuda(scene.grid, scene.probes, scene.mlp,
                  dtypes=(torch.float32, torch.float16, torch.uint8))
    gd, pd, md = scene.descs(params.n_fresnel)
    Rx, Ry, Rz = (int(v) for v in scene.dims)
    if out is None:
        out = torch.empty((Rz, Ry, Rx, 4), dtype=torch.float16, device=scene.grid.device)
    _require_cuda(out, dtypes=(torch.float16,))
    if out.numel() * 2 != colour_field_bytes(gd) or not out.is_contiguous():
        raise LibraryError("shade_nodes: out must be a contiguous FP16 [Rz, Ry, Rx, 4] tensor")
    cam = (ctypes.c_float * 3)(*(float(v) for v in camera))
    h = _Handles(scene.grid, scene.probes, scene.mlp, gd, pd, md)
    try:
        _check(library().psdf_shade_nodes(h.g, h.p, h.m, ctypes.byref(params), cam, float(band),
                                          _ptr(out), _stream()), "psdf_shade_nodes")
    finally:
        h.close()
    return out


def render_colour_field(scene: Scene, colours, rays_o, rays_d, params: RenderParams,
                        t_samples=None):
    """The NeuS march over the SDF with every sample's colour interpolated from
    the node colours -> rgb [n,3], depth [n], wsum [n]."""
    _require_cuda(scene.grid, dtypes=(torch.float32, torch.float16, torch.uint8))
    _require_cuda(colours, dtypes=(torch.float16,))
    _require_cuda(rays_o, rays_d, t_samples)
    gd, _, _ = scene.descs(params.n_fresnel)
    if colours.numel() * 2 != colour_field_bytes(gd) or not colours.is_contiguous():
        raise LibraryError("render_colour_field: colours must be FP16 [Rz, Ry, Rx, 4]")
    n = rays_o.shape[0]
    dev = rays_o.device
    rgb = torch.empty((n, 3), dtype=torch.float32, device=dev)
    depth = torch.empty(n, dtype=torch.float32, device=dev)
    wsum = torch.empty(n, dtype=torch.float32, device=dev)
    lib = library()
    g = _P()
    _check(lib.psdf_grid_create(ctypes.byref(gd), _ptr(scene.grid), ctypes.byref(g)),
           "psdf_grid_create")
    try:
        _check(lib.psdf_render_colour_field(g, _ptr(colours), ctypes.byref(params), _ptr(rays_o),
                                            _ptr(rays_d), _ptr(t_samples), n, _ptr(rgb),
                                            _ptr(depth), _ptr(wsum), _stream()),
               "psdf_render_colour_field")
    finally:
        lib.psdf_grid_destroy(g)
    return rgb, depth, wsum


# ---------------------------------------------------------------------------
# Grid-level training terms (Sec. 3.3, Eqs. 11-15)
# ---------------------------------------------------------------------------

def _check_dense_sdf(gd, t, what):
    n = int(gd.dims[0]) * int(gd.dims[1]) * int(gd.dims[2])
    if t.numel() != n or not t.is_contiguous():
        raise LibraryError(f"{what}: expected a contiguous FP32 array of {n} nodes")


def _check_sdf_param(gd, t, what):
    """The raw SDF: [Rz,Ry,Rx] for a dense grid, [n_bricks,16,16,16] (slot
    order) for a sparse one."""
    if gd.n_bricks > 0:
        n = int(gd.n_bricks) * TILE ** 3
        if t.numel() != n or not t.is_contiguous():
            raise LibraryError(f"{what}: expected a contiguous FP32 array of {n} stored nodes")
    else:
        _check_dense_sdf(gd, t, what)


def sdf_smooth(gd, sdf_hat, values):
    """Write s = G(sdf_hat) (5^3 Gaussian, sigma = 1 node) into the SDF slot of
    the packed grid `values`; the features are left as they are.  For a sparse
    grid sdf_hat holds the stored bricks, [n_bricks, 16, 16, 16] in slot order,
    and the nodes of absent bricks count as empty_sdf."""
    _require_cuda(sdf_hat, values, dtypes=(torch.float32, torch.uint8, torch.bfloat16))
    _check_sdf_param(gd, sdf_hat, "sdf_smooth")
    _check(library().psdf_sdf_smooth(ctypes.byref(gd), _ptr(sdf_hat), _ptr(values), _stream()),
           "psdf_sdf_smooth")


def sdf_smooth_adjoint(gd, grad_grid, d_sdf_hat, accumulate=True):
    """d_sdf_hat (+)= G^T of the SDF slot of a grid gradient buffer.  For a
    sparse grid d_sdf_hat is [n_bricks, 16, 16, 16] and the brick table is read
    from the gradient buffer's copy (zero only its records)."""
    _require_cuda(grad_grid, d_sdf_hat)
    _check_sdf_param(gd, d_sdf_hat, "sdf_smooth_adjoint")
    _check(library().psdf_sdf_smooth_adjoint(ctypes.byref(gd), _ptr(grad_grid), _ptr(d_sdf_hat),
                                             int(bool(accumulate)), _stream()),
           "psdf_sdf_smooth_adjoint")


def grid_regularizers(gd, sdf_hat, values, grad_grid, d_sdf_hat, lam_sdf, lam_eik, lam_normal,
                      lam_features=0.0, loss=None):
    """Adds the gradients of the weighted L_sdf, L_Eik, L_normal (and, for
    tri-planes, L_features) to grad_grid and d_sdf_hat; adds the unweighted
    values {sdf, eik, normal, features} to `loss` (FP32 [4]) when given.  For
    a sparse grid sdf_hat and d_sdf_hat hold the stored bricks ([n_bricks, 16,
    16, 16], slot order) and the sums run over the stored nodes' terms."""
    _require_cuda(sdf_hat, grad_grid, d_sdf_hat, loss)
    _require_cuda(values, dtypes=(torch.float32, torch.uint8, torch.bfloat16))
    _check_sdf_param(gd, sdf_hat, "grid_regularizers")
    _check_sdf_param(gd, d_sdf_hat, "grid_regularizers")
    if loss is not None and loss.numel() < 4:
        raise LibraryError("grid_regularizers: loss needs 4 entries")
    _check(library().psdf_grid_regularizers(
        ctypes.byref(gd), _ptr(sdf_hat), _ptr(values), float(lam_sdf), float(lam_eik),
        float(lam_normal), float(lam_features), _ptr(grad_grid), _ptr(d_sdf_hat), _ptr(loss),
        _stream()), "psdf_grid_regularizers")


def probe_smoothness(pd, coeffs, grad, lam, loss=None):
    """Adds lam * grad L_probes (6-neighbour pairs) to `grad` and L_probes to loss[0]."""
    _require_cuda(coeffs, grad, loss)
    if grad.numel() != coeffs.numel():
        raise LibraryError("probe_smoothness: coeffs and grad must have the same size")
    _check(library().psdf_probe_smoothness(ctypes.byref(pd), _ptr(coeffs), float(lam), _ptr(grad),
                                           _ptr(loss), _stream()), "psdf_probe_smoothness")


# ---------------------------------------------------------------------------
# Learned sample proposal (the paper marches its sparse grid instead)
# ---------------------------------------------------------------------------

def proposal_desc(occ_res=(32, 32, 32), n_bins=8, width=32, mix=0.1, theta=0.2,
                  n_sub=8) -> ProposalDesc:
    d = ProposalDesc()
    d.occ_res[:] = tuple(int(v) for v in occ_res)
    d.n_bins = int(n_bins)
    d.width = int(width)
    d.n_sub = int(n_sub)
    d.mix = float(mix)
    d.theta = float(theta)
    return d


def proposal_param_count(desc: ProposalDesc) -> int:
    n = ctypes.c_int64()
    _check(library().psdf_proposal_param_count(ctypes.byref(desc), ctypes.byref(n)),
           "psdf_proposal_param_count")
    return n.value


class _GridHandle:
    def __init__(self, scene: Scene):
        gd, _, _ = scene.descs(3)
        self.h = _P()
        _check(library().psdf_grid_create(ctypes.byref(gd), _ptr(scene.grid),
                                          ctypes.byref(self.h)), "psdf_grid_create")

    def __enter__(self):
        return self.h

    def __exit__(self, *exc):
        library().psdf_grid_destroy(self.h)


def occupancy_words(occ_res) -> int:
    res = (ctypes.c_int32 * 3)(*(int(v) for v in occ_res))
    n = ctypes.c_int64()
    _check(library().psdf_occupancy_words(res, ctypes.byref(n)), "psdf_occupancy_words")
    return n.value


def occupancy_build(scene: Scene, occ_res, threshold: float) -> torch.Tensor:
    """Occupancy bitmask (int32 words holding 32 cells each, cell
    (z res_y + y) res_x + x at bit i & 31 of word i >> 5) of the cells near
    the zero level set."""
    occ = torch.empty(occupancy_words(occ_res), dtype=torch.int32, device=scene.grid.device)
    res = (ctypes.c_int32 * 3)(*(int(v) for v in occ_res))
    with _GridHandle(scene) as g:
        _check(library().psdf_occupancy_build(g, res, float(threshold), _ptr(occ), _stream()),
               "psdf_occupancy_build")
    return occ


def occupancy_unpack(occ_bits: torch.Tensor, occ_res) -> torch.Tensor:
    """Bitmask -> [res_z, res_y, res_x] uint8 {0, 1} (host copy, for inspection)."""
    rx, ry, rz = (int(v) for v in occ_res)
    w = occ_bits.cpu().view(-1).to(torch.int64) & 0xFFFFFFFF
    cells = torch.arange(rx * ry * rz)
    return ((w[cells >> 5] >> (cells & 31)) & 1).to(torch.uint8).view(rz, ry, rx)


def weight_histogram(scene: Scene, rays_o, rays_d, params: RenderParams, n_bins=8):
    """[n, n_bins] per-bin sums of the uniform march's weights (SDF only)."""
    _require_cuda(rays_o, rays_d)
    n = rays_o.shape[0]
    hist = torch.empty((n, n_bins), dtype=torch.float32, device=rays_o.device)
    with _GridHandle(scene) as g:
        _check(library().psdf_weight_histogram(g, ctypes.byref(params), _ptr(rays_o),
                                               _ptr(rays_d), n, int(n_bins), _ptr(hist),
                                               _stream()), "psdf_weight_histogram")
    return hist


def proposal_forward(scene: Scene, desc: ProposalDesc, params, occ, rays_o, rays_d, n_out,
                     want_probs=True, want_t=True):
    """(t_samples [n, n_out + 1] or None, mixed density p' [n, B] or None)."""
    _require_cuda(params, rays_o, rays_d)
    _require_cuda(occ, dtypes=(torch.int32,))
    n = rays_o.shape[0]
    t = torch.empty((n, n_out + 1), dtype=torch.float32, device=rays_o.device) \
        if want_t else None
    probs = (torch.empty((n, desc.n_bins), dtype=torch.float32, device=rays_o.device)
             if want_probs else None)
    with _GridHandle(scene) as g:
        _check(library().psdf_proposal_forward(g, ctypes.byref(desc), _ptr(params), _ptr(occ),
                                               _ptr(rays_o), _ptr(rays_d), n, int(n_out),
                                               _ptr(t), _ptr(probs), _stream()),
               "psdf_proposal_forward")
    return t, probs


def proposal_backward(scene: Scene, desc: ProposalDesc, params, occ, rays_o, rays_d, hist,
                      min_mass=1e-3, scale=1.0, grad=None, want_loss=True):
    """(grad [param count] with the gradient of scale * sum(loss) ADDED,
    per-ray cross-entropy loss [n] or None)."""
    _require_cuda(params, rays_o, rays_d, hist, grad)
    _require_cuda(occ, dtypes=(torch.int32,))
    n = rays_o.shape[0]
    if grad is None:
        grad = torch.zeros_like(params)
    loss = torch.empty(n, dtype=torch.float32, device=rays_o.device) if want_loss else None
    with _GridHandle(scene) as g:
        _check(library().psdf_proposal_backward(g, ctypes.byref(desc), _ptr(params), _ptr(occ),
                                                _ptr(rays_o), _ptr(rays_d), n, _ptr(hist),
                                                float(min_mass), float(scale), _ptr(grad),
                                                _ptr(loss), _stream()),
               "psdf_proposal_backward")
    return grad, loss
