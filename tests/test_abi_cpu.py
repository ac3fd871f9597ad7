"""Host-only checks of the C ABI library (no GPU needed, no kernel launched):
it builds for sm_103a, loads, exports every symbol include/*.h declares, and
rejects bad arguments on the host before any CUDA call."""
import ctypes
import glob
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(psdf_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2412_10084_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("psdf_render_forward", "psdf_render_backward", "psdf_grid_create",
                     "psdf_probes_create", "psdf_mlp_create", "psdf_grid_pack",
                     "psdf_grid_unpack"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_version(lib):
    lib.psdf_status_string.restype = ctypes.c_char_p
    assert lib.psdf_status_string(0) == b"ok"
    assert b"aligned" in lib.psdf_status_string(-4)
    assert lib.psdf_version() >= 100


def test_wait_polls_setting_is_thread_local(lib):
    """The tensor-core wait limit: set, read back, restored by 0xFFFFFFFF, and
    private to the host thread that set it (no CUDA call involved)."""
    import threading
    lib.psdf_wait_polls.restype = ctypes.c_uint32
    lib.psdf_set_wait_polls.argtypes = [ctypes.c_uint32]
    default = lib.psdf_wait_polls()
    assert default == 1 << 24
    assert lib.psdf_set_wait_polls(7) == 0 and lib.psdf_wait_polls() == 7
    seen = []
    t = threading.Thread(target=lambda: seen.append(lib.psdf_wait_polls()))
    t.start()
    t.join()
    assert seen == [default]
    assert lib.psdf_set_wait_polls(0xFFFFFFFF) == 0 and lib.psdf_wait_polls() == default


def test_host_validation_without_gpu(lib):
    import paper_2412_10084_gb300 as ps
    gd = ps.grid_desc((64, 64, 64), (0, 0, 0), (1, 1, 1))
    assert ps.grid_bytes(gd) == (64 ** 3 * 16, 64 ** 3 * 16)
    gb = ps.grid_desc((33, 33, 33), (0, 0, 0), (1, 1, 1), feat_dtype=ps.BF16)
    n = 33 ** 3
    assert ps.grid_bytes(gb) == (((4 * n + 15) // 16) * 16 + 8 * n, 16 * n)
    assert ps.mlp_param_count(10, 32) == 32 * 10 + 32 + 32 * 32 + 32 + 96 + 3
    bad = ps.grid_desc((1, 64, 64), (0, 0, 0), (1, 1, 1))
    with pytest.raises(ps.LibraryError, match="shape"):
        ps.grid_bytes(bad)
    flat = ps.grid_desc((8, 8, 8), (0, 0, 0), (1, 0, 1))
    with pytest.raises(ps.LibraryError, match="shape"):
        ps.grid_bytes(flat)
    h = ctypes.c_void_p()
    lib.psdf_grid_create.argtypes = [ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.POINTER(ctypes.c_void_p)]
    assert lib.psdf_grid_create(ctypes.byref(gd), ctypes.c_void_p(0x1008), ctypes.byref(h)) == -4
    assert lib.psdf_grid_create(ctypes.byref(gd), None, ctypes.byref(h)) == -1
    lib.psdf_render_forward.argtypes = [ctypes.c_void_p] * 7 + [ctypes.c_int64] + \
        [ctypes.c_void_p] * 6
    assert lib.psdf_render_forward(None, None, None, None, None, None, None, 0,
                                   None, None, None, None, None, None) == -1


def test_kernel_sh_constants_match_closed_form():
    """The SH constants typed into the kernels equal the Cartesian coefficients
    of the orthonormal real basis of Eq. 5 (normalisation
    sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!), times sqrt 2 for m != 0)."""
    src = open(os.path.join(ROOT, "paper_2412_10084_gb300", "csrc", "render_common.cuh")).read()
    body = src[src.index("sh_basis(const float"):src.index("sh_basis_vjp")]
    consts = sorted({float(v) for v in re.findall(r"(\d\.\d{10,})f", body)})

    # Cartesian coefficients of the real SH, degrees 0..3
    closed = sorted({
        0.5 * math.sqrt(1 / math.pi), math.sqrt(3 / (4 * math.pi)),
        0.5 * math.sqrt(15 / math.pi), 0.25 * math.sqrt(5 / math.pi),
        0.25 * math.sqrt(15 / math.pi), 0.25 * math.sqrt(35 / (2 * math.pi)),
        0.5 * math.sqrt(105 / math.pi), 0.25 * math.sqrt(21 / (2 * math.pi)),
        0.25 * math.sqrt(7 / math.pi), 0.25 * math.sqrt(105 / math.pi)})
    assert len(consts) == len(closed)
    for a, b in zip(consts, closed):
        assert abs(a - b) <= 1e-15 * b


def test_regularizer_entry_points_reject_bad_arguments_on_the_host(lib):
    import paper_2412_10084_gb300 as ps
    P = ctypes.c_void_p
    f = ctypes.c_float
    gd = ps.grid_desc((9, 9, 9), (0, 0, 0), (1, 1, 1))
    lib.psdf_sdf_smooth.argtypes = [P, P, P, P]
    assert lib.psdf_sdf_smooth(ctypes.byref(gd), None, P(0x1000), None) == -1
    assert lib.psdf_sdf_smooth(ctypes.byref(gd), P(0x1004), P(0x1000), None) == -4
    lib.psdf_sdf_smooth_adjoint.argtypes = [P, P, P, ctypes.c_int32, P]
    assert lib.psdf_sdf_smooth_adjoint(ctypes.byref(gd), P(0x1000), None, 1, None) == -1
    lib.psdf_grid_regularizers.argtypes = [P, P, P, f, f, f, f, P, P, P, P]
    args = (P(0x1000), P(0x2000))
    assert lib.psdf_grid_regularizers(ctypes.byref(gd), *args, 1.0, 1.0, 1.0, 0.5, P(0x3000),
                                      P(0x4000), None, None) == -6   # features need tri-planes
    assert lib.psdf_grid_regularizers(ctypes.byref(gd), *args, 1.0, -1.0, 1.0, 0.0, P(0x3000),
                                      P(0x4000), None, None) == -1
    assert lib.psdf_grid_regularizers(ctypes.byref(gd), *args, 1.0, 1.0, 1.0, 0.0, P(0x3000),
                                      P(0x4000), P(0x5002), None) == -4
    pd = ps.ProbeDesc()
    pd.dims[:] = (3, 3, 3)
    pd.sh_l, pd.n_ang, pd.dtype = 3, 4, ps.F16
    lib.psdf_probe_smoothness.argtypes = [P, P, f, P, P, P]
    assert lib.psdf_probe_smoothness(ctypes.byref(pd), P(0x1000), 1.0, P(0x2000), None,
                                     None) == -3
    pd.dtype, pd.n_ang = ps.F32, 3
    assert lib.psdf_probe_smoothness(ctypes.byref(pd), P(0x1000), 1.0, P(0x2000), None,
                                     None) == -6


def test_two_pass_entry_points_on_the_host(lib):
    import paper_2412_10084_gb300 as ps
    P = ctypes.c_void_p
    gd = ps.grid_desc((9, 10, 11), (0, 0, 0), (1, 1, 1))
    assert ps.colour_field_bytes(gd) == 8 * 9 * 10 * 11
    lib.psdf_render_colour_field.argtypes = [P, P, P, P, P, P, ctypes.c_int64, P, P, P, P]
    assert lib.psdf_render_colour_field(None, P(0x1000), None, None, None, None, 0, None, None,
                                        None, None) == -1
    lib.psdf_shade_nodes.argtypes = [P, P, P, P, P, ctypes.c_float, P, P]
    assert lib.psdf_shade_nodes(None, None, None, None, None, 0.1, None, None) == -1


def test_sparse_grid_descriptors_on_the_host(lib):
    """Sparse (brick) descriptors: sizes, and what the host rejects before any
    CUDA call."""
    import paper_2412_10084_gb300 as ps
    P = ctypes.c_void_p
    gd = ps.grid_desc((32, 48, 64), (0, 0, 0), (1, 1, 1), n_bricks=5, empty_sdf=1.0)
    table = ((2 * 3 * 4 * 4 + 15) // 16) * 16
    assert ps.grid_bytes(gd) == (table + 5 * 4096 * 16,) * 2
    assert ps.table_words(gd) * 4 == table
    assert ps.colour_field_bytes(gd) == 8 * 32 * 48 * 64  # one record per node of the full grid
    for kw, what in ((dict(dims=(40, 48, 64)), "shape"),            # not whole bricks
                     (dict(n_bricks=25), "shape"),                   # more than 2 x 3 x 4
                     (dict(feat_dtype=ps.BF16), "compiled"),         # FP32 node records only
                     (dict(empty_sdf=float("nan")), "argument")):
        args = dict(dims=(32, 48, 64), n_bricks=5, empty_sdf=1.0)
        args.update(kw)
        d = ps.grid_desc(args.pop("dims"), (0, 0, 0), (1, 1, 1), **args)
        with pytest.raises(ps.LibraryError, match=what):
            ps.grid_bytes(d)
    f = ctypes.c_float
    lib.psdf_sdf_smooth.argtypes = [P, P, P, P]
    assert lib.psdf_sdf_smooth(ctypes.byref(gd), None, P(0x1000), None) == -1
    assert lib.psdf_sdf_smooth(ctypes.byref(gd), P(0x1000), P(0x2008), None) == -4
    lib.psdf_sdf_smooth_adjoint.argtypes = [P, P, P, ctypes.c_int32, P]
    assert lib.psdf_sdf_smooth_adjoint(ctypes.byref(gd), P(0x1004), P(0x2000), 0, None) == -4
    lib.psdf_grid_regularizers.argtypes = [P, P, P, f, f, f, f, P, P, P, P]
    # the SDF terms take sparse grids; L_features needs tile tri-planes, and the
    # buffers must be 16-byte aligned (both refused before any CUDA call)
    assert lib.psdf_grid_regularizers(ctypes.byref(gd), P(0x1000), P(0x2000), 1.0, 1.0, 1.0,
                                      1.0, P(0x3000), P(0x4000), None, None) == -6
    assert lib.psdf_grid_regularizers(ctypes.byref(gd), P(0x1000), P(0x2004), 1.0, 1.0, 1.0,
                                      0.0, P(0x3000), P(0x4000), None, None) == -4


def test_sparse_scene_checks_the_brick_mask_shape():
    import numpy as np
    import paper_2412_10084_gb300 as ps
    keep = np.ones((2, 3, 4), bool)  # (Bz, By, Bx) of a 64 x 48 x 32 grid, given for 32 x 48 x 64
    with pytest.raises(ps.LibraryError, match=r"\(4, 3, 2\)"):
        ps.sparse_scene(keep, None, None, None, None, (32, 48, 64), (0, 0, 0), (1, 1, 1), 3, 32,
                        device="cpu")
