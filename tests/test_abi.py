"""The C-ABI library builds, loads without a GPU and exports every entry point that
include/cgs.h declares; host-side argument checks work without touching a device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^(?:const\s+)?\w+\s*\*?\s*(cgs_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libcgs():
    from paper_2404_01133_b300 import build
    build.build()
    from paper_2404_01133_b300 import cgs
    return cgs.lib()


def test_every_declared_symbol_is_exported(libcgs):
    names = declared_functions()
    assert len(names) >= 11
    for n in names:
        assert hasattr(libcgs, n), n


def test_workspace_sizing_and_validation(libcgs):
    from paper_2404_01133_b300 import cgs
    b = cgs.cgs_frame_workspace_bytes(1, 1920, 1080, 16, 1, 1_000_000, 8_000_000)
    assert b > 8_000_000 * 16
    assert cgs.cgs_frame_workspace_bytes(1, 1920, 1080, 12, 1, 10, 10) == 0      # tile must be 8 or 16
    assert cgs.cgs_frame_workspace_bytes(0, 1920, 1080, 16, 1, 10, 10) == 0
    assert cgs.cgs_frame_workspace_bytes(1, 1920, 1080, 16, 1, 10, 1 << 30) == 0  # k_cap < 2^30
    # capacity grows the workspace
    assert cgs.cgs_frame_workspace_bytes(1, 64, 64, 16, 1, 2000, 20000) > cgs.cgs_frame_workspace_bytes(
        1, 64, 64, 16, 1, 1000, 10000)


def test_host_argument_checks_need_no_device(libcgs):
    from paper_2404_01133_b300 import cgs
    f = cgs.cgs_frame()
    s = cgs.cgs_scene()
    c = cgs.cgs_config()
    # null workspace and null scene pointers are rejected before any CUDA call
    assert libcgs.cgs_render_forward(C.byref(s), C.byref(f), C.byref(c), None, None, None, None, None, None,
                                     None) == cgs.CGS_ERR_INVALID_ARGUMENT
    assert libcgs.cgs_l1_loss(None, None, 10, None, None, None) == cgs.CGS_ERR_INVALID_ARGUMENT
    # a frame with an unknown flag is rejected before any CUDA call
    f2 = cgs.cgs_frame()
    f2.ws, f2.ws_bytes = 256, 1 << 30
    f2.n_views, f2.width, f2.height, f2.tile, f2.n_blocks, f2.n_cap, f2.k_cap = 1, 64, 64, 16, 1, 100, 1000
    f2.flags = 2
    st, cnt = C.c_int32(0), (C.c_int64 * 8)()
    assert libcgs.cgs_frame_status(C.byref(f2), C.byref(st), cnt, None) == cgs.CGS_ERR_INVALID_ARGUMENT
    assert cgs.cgs_status_string(cgs.CGS_ERR_CAPACITY).startswith("capacity")
    assert cgs.cgs_version() == 1


def test_oracle_is_not_imported_by_the_product_path():
    for dirpath, _, files in os.walk(os.path.join(ROOT, "paper_2404_01133_b300")):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in text and "from oracle" not in text, fn
                assert "liboracle" not in text, fn


def test_partition_host_checks_need_no_device(libcgs):
    from paper_2404_01133_b300 import cgs
    libcgs = cgs.lib()  # with argument types set
    # invalid grids and boxes are rejected before any device work
    assert cgs.cgs_partition_workspace_bytes(1000, (8, 8, 1)) > 0
    assert cgs.cgs_partition_workspace_bytes(1000, (0, 8, 1)) == -1
    assert cgs.cgs_partition_workspace_bytes(1000, (65, 1, 1)) == -1
    assert cgs.cgs_partition_workspace_bytes(1000, (32, 32, 2)) == -1        # 2048 blocks > 1024
    assert cgs.cgs_partition_workspace_bytes(-1, (8, 8, 1)) == -1
    f3 = lambda v: (C.c_float * 3)(*v)
    i3 = lambda v: (C.c_int32 * 3)(*v)
    bad_box = libcgs.cgs_partition(1, 10, 4, f3((0, 0, 0)), f3((1, 0, 1)), i3((2, 2, 1)), 1, 1, None, None, 1,
                                   1 << 20, None)
    assert bad_box == cgs.CGS_ERR_INVALID_ARGUMENT                           # pmax == pmin on y
    assert libcgs.cgs_partition(1, 10, 2, f3((0, 0, 0)), f3((1, 1, 1)), i3((2, 2, 1)), 1, 1, None, None, 1,
                                1 << 20, None) == cgs.CGS_ERR_INVALID_ARGUMENT   # stride < 3
    assert libcgs.cgs_partition(1, 10, 4, f3((0, 0, 0)), f3((1, 1, 1)), i3((2, 2, 1)), 1, 1, None, None, 1, 16,
                                None) == cgs.CGS_ERR_WORKSPACE_TOO_SMALL
    assert libcgs.cgs_scatter_rows(1, 2, 6, 3, 10, None) == cgs.CGS_ERR_INVALID_ARGUMENT
    assert libcgs.cgs_levels_workspace_bytes(100, 0) == -1 and libcgs.cgs_levels_workspace_bytes(100, 1025) == -1
    r2 = (C.c_double * 2)(1.0, 1.5)                                               # a rate above 1
    assert libcgs.cgs_generate_levels(1, 1, 0, 10, 1, 2, None, r2, 2, 1, 1, 1, 1 << 30, None) == \
        cgs.CGS_ERR_INVALID_ARGUMENT
    assert libcgs.cgs_render_forward_hits(C.byref(cgs.cgs_scene()), C.byref(cgs.cgs_frame()),
                                          C.byref(cgs.cgs_config()), None, None, None, None, None, None, None,
                                          None) == cgs.CGS_ERR_INVALID_ARGUMENT
    assert libcgs.cgs_gather_rows(1, 2, 6, 3, 10, None) == cgs.CGS_ERR_INVALID_ARGUMENT   # row bytes % 4
    assert libcgs.cgs_gather_rows(None, None, 16, None, 0, None) == cgs.CGS_OK             # nothing to move
    assert libcgs.cgs_pose_blocks(1, 4, 3, f3((0, 0, 0)), f3((1, 1, 1)), i3((1, 1, 0)), 1, None) == \
        cgs.CGS_ERR_INVALID_ARGUMENT


def test_boundary_entry_points_check_arguments_on_the_host(libcgs):
    """Scene upload, pose assignment and the autotuner reject invalid sizes, pointers and block
    tables before any device work (no GPU here)."""
    import numpy as np
    from paper_2404_01133_b300 import cgs
    n, deg, nb, nl = 1000, 3, 4, 3
    b = cgs.cgs_scene_bytes(n, deg, nb, nl, 0)
    assert b >= n * (16 + 16 + 16 + 192) and b % 256 == 0
    assert cgs.cgs_scene_bytes(n, deg, nb, nl, 1) < b                     # half-precision attributes
    assert cgs.cgs_scene_bytes(n, 4, nb, nl, 0) == -1                     # SH degree above 3
    assert cgs.cgs_scene_bytes(-1, deg, nb, nl, 0) == -1
    mo = np.zeros((n, 4), np.float32)
    sc4 = np.zeros((n, 4), np.float32)
    sh = np.zeros((n, 16, 3), np.float32)
    cell = np.zeros((nb, 4), np.float32)
    cnt = np.full((nb, nl), 100, np.int64)
    good = np.repeat(np.arange(nb, dtype=np.int64)[:, None] * 250, nl, axis=1)
    s = cgs.cgs_scene()
    L = libcgs
    args = lambda off, count, mem=1 << 20, nbytes=b: (C.byref(s), mem, nbytes, mo.ctypes.data, sc4.ctypes.data,
                                                       sc4.ctypes.data, sh.ctypes.data, n, deg, 0, nb, nl,
                                                       off.ctypes.data, count.ctypes.data, cell.ctypes.data, -1.0,
                                                       None)
    overlap = good.copy()
    overlap[2] = 120                                                      # block 2 starts inside block 1
    assert L.cgs_scene_upload(*args(overlap, cnt)) == cgs.CGS_ERR_INVALID_ARGUMENT
    beyond = good.copy()
    beyond[3] = n - 50                                                    # a segment past the last Gaussian
    assert L.cgs_scene_upload(*args(beyond, cnt)) == cgs.CGS_ERR_INVALID_ARGUMENT
    assert L.cgs_scene_upload(*args(good, cnt, mem=None)) == cgs.CGS_ERR_INVALID_ARGUMENT
    assert L.cgs_scene_upload(*args(good, cnt, nbytes=b - 1)) == cgs.CGS_ERR_WORKSPACE_TOO_SMALL
    # pose assignment: sizes and the three outputs
    assert L.cgs_pose_assign(None, None, 2, 4, C.c_float(0.05), None, None, None, None) == cgs.CGS_ERR_INVALID_ARGUMENT
    assert L.cgs_pose_assign(None, None, 0, 4, C.c_float(0.05), 1, None, None, None) == cgs.CGS_OK   # nothing to do
    assert L.cgs_pose_assign(1, 1, 2, 0, C.c_float(0.05), 1, None, None, None) == cgs.CGS_ERR_INVALID_ARGUMENT
    # autotuner workspace and arguments
    wb = cgs.cgs_autotune_workspace_bytes(1, 1920, 1080, 1, 1_000_000, 4_000_000, 3, cgs.CGS_TUNE_FORWARD_BACKWARD)
    wf = cgs.cgs_autotune_workspace_bytes(1, 1920, 1080, 1, 1_000_000, 4_000_000, 3, cgs.CGS_TUNE_FORWARD)
    assert wb > wf > cgs.cgs_frame_workspace_bytes(1, 1920, 1080, 16, 1, 1_000_000, 4_000_000)
    assert cgs.cgs_autotune_workspace_bytes(1, 1920, 1080, 1, 1_000_000, 4_000_000, 3, 7) == -1
    cfg = cgs.cgs_config()
    ms = (C.c_float * cgs.CGS_TUNE_CANDIDATES)()
    assert L.cgs_autotune(None, 1, 1, 64, 64, None, None, 10, 10, 0, 3, 1, 1 << 30, C.byref(cfg), ms, None, None,
                          None) == cgs.CGS_ERR_INVALID_ARGUMENT
