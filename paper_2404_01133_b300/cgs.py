"""ctypes binding of libcgs.so (include/cgs.h): the same entry points, same names.

This module only marshals arguments: device pointers come from torch tensors
(``tensor.data_ptr()``), streams from ``torch.cuda.current_stream().cuda_stream``.  Every
step of the rendering path runs in the CUDA library; if the library is missing this module
raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcgs.so")

CGS_OK = 0
CGS_ERR_INVALID_ARGUMENT = 1
CGS_ERR_WORKSPACE_TOO_SMALL = 2
CGS_ERR_CAPACITY = 3
CGS_ERR_SPIN_TIMEOUT = 4
CGS_ERR_CUDA = 5
CGS_ERR_UNSUPPORTED = 6
CGS_ERR_TOO_LARGE = 7

BUF_TILE_KEYS, BUF_TILE_VALS, BUF_RANGES, BUF_SCENE_INDEX, BUF_RECORDS, BUF_TILES_TOUCHED, BUF_VIEW_BASE, \
    BUF_VISIBLE, BUF_DEPTH_KEYS, BUF_RECTS = range(10)


class cgs_camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("campos", C.c_float * 3),
                ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("width", C.c_int32), ("height", C.c_int32), ("_pad", C.c_float * 3)]


class cgs_scene(C.Structure):
    _fields_ = [("mean_opac", C.c_void_p), ("scale", C.c_void_p), ("quat", C.c_void_p), ("sh", C.c_void_p),
                ("n", C.c_int64), ("sh_degree", C.c_int32), ("n_blocks", C.c_int32), ("n_levels", C.c_int32),
                ("attr_fp16", C.c_int32), ("level_offset", C.c_void_p), ("level_count", C.c_void_p),
                ("block_aabb", C.c_void_p), ("block_cell", C.c_void_p)]


class cgs_config(C.Structure):
    _fields_ = [("tile", C.c_int32), ("batch", C.c_int32), ("near_z", C.c_float), ("bg", C.c_float * 3),
                ("lod_dist", C.c_double * 2), ("lod_mode", C.c_int32), ("exact", C.c_int32)]


CGS_FRAME_NO_PAIR_COUNT = 1
CGS_LOD_BLOCK = 0
CGS_LOD_POINT = 1
CGS_TUNE_CANDIDATES = 6
CGS_TUNE_FORWARD = 0
CGS_TUNE_FORWARD_BACKWARD = 1
TUNE_ORDER = ((16, 256), (16, 128), (16, 64), (16, 32), (8, 64), (8, 32))


class cgs_frame(C.Structure):
    _fields_ = [("ws", C.c_void_p), ("ws_bytes", C.c_int64), ("n_views", C.c_int32), ("width", C.c_int32),
                ("height", C.c_int32), ("tile", C.c_int32), ("n_blocks", C.c_int32), ("flags", C.c_int32),
                ("n_cap", C.c_int64), ("k_cap", C.c_int64)]


assert C.sizeof(cgs_camera) == 96

_lib = None


def lib():
    """Loads libcgs.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libcgs.so not found at {LIB_PATH}; build it with "
                               "`python -m paper_2404_01133_b300.build`")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, P = C.c_void_p, C.c_int32, C.c_int64, C.POINTER
        L.cgs_version.restype = i32
        L.cgs_status_string.restype = C.c_char_p
        L.cgs_status_string.argtypes = [i32]
        L.cgs_frame_workspace_bytes.restype = i64
        L.cgs_frame_workspace_bytes.argtypes = [i32, i32, i32, i32, i32, i64, i64]
        L.cgs_block_bounds_workspace_bytes.restype = i64
        L.cgs_block_bounds_workspace_bytes.argtypes = [i64]
        L.cgs_block_bounds.restype = i32
        L.cgs_block_bounds.argtypes = [P(cgs_scene), C.c_double, vp, vp, i64, vp]
        L.cgs_lod_select.restype = i32
        L.cgs_lod_select.argtypes = [P(cgs_scene), P(cgs_config), vp, i32, vp, vp]
        L.cgs_render_forward.restype = i32
        L.cgs_render_forward.argtypes = [P(cgs_scene), P(cgs_frame), P(cgs_config), vp, vp, vp, vp, vp, vp, vp]
        L.cgs_render_backward.restype = i32
        L.cgs_render_backward.argtypes = [P(cgs_scene), P(cgs_frame), P(cgs_config), vp, vp, vp, vp, vp, vp, vp,
                                          vp, vp]
        L.cgs_render_backward_packed.restype = i32
        L.cgs_render_backward_packed.argtypes = [P(cgs_scene), P(cgs_frame), P(cgs_config), vp, vp, vp, vp, vp, vp,
                                                 vp, vp, vp, vp]
        L.cgs_render_backward_l1.restype = i32
        L.cgs_render_backward_l1.argtypes = [P(cgs_scene), P(cgs_frame), P(cgs_config), vp, vp, vp, i32, vp, vp, vp,
                                             vp, vp, vp, vp, vp, vp]
        L.cgs_l1_loss.restype = i32
        L.cgs_l1_loss.argtypes = [vp, vp, i64, vp, vp, vp]
        L.cgs_l1_loss_u8.restype = i32
        L.cgs_l1_loss_u8.argtypes = [vp, vp, i64, vp, vp, vp]
        L.cgs_frame_status.restype = i32
        L.cgs_frame_status.argtypes = [P(cgs_frame), P(i32), P(i64), vp]
        L.cgs_timing_enable.restype = i32
        L.cgs_timing_enable.argtypes = [i32]
        L.cgs_timing_read.restype = i32
        L.cgs_timing_read.argtypes = [P(C.c_double), P(i64)]
        L.cgs_kernel_launches.restype = i64
        L.cgs_render_forward_static.restype = i32
        L.cgs_render_forward_static.argtypes = [P(cgs_scene), P(cgs_config), vp, i32, i32, vp, vp, vp, vp, vp, vp, vp]
        L.cgs_frame_buffer.restype = i32
        L.cgs_frame_buffer.argtypes = [P(cgs_frame), i32, P(vp), P(i64)]
        L.cgs_render_forward_hits.restype = i32
        L.cgs_render_forward_hits.argtypes = [P(cgs_scene), P(cgs_frame), P(cgs_config), vp, vp, vp, vp, vp, vp, vp,
                                              vp]
        L.cgs_levels_workspace_bytes.restype = i64
        L.cgs_levels_workspace_bytes.argtypes = [i64, i32]
        L.cgs_generate_levels.restype = i32
        L.cgs_generate_levels.argtypes = [vp, vp, i32, i64, vp, i32, vp, vp, i32, vp, vp, vp, i64, vp]
        L.cgs_levels_status.restype = i32
        L.cgs_levels_status.argtypes = [vp, vp]
        L.cgs_ssim.restype = i32
        L.cgs_ssim.argtypes = [vp, i64, vp, i32, i32, i32, i32, vp, vp, vp]
        L.cgs_contract.restype = i32
        L.cgs_contract.argtypes = [vp, i64, i64, vp, vp, vp, vp]
        L.cgs_pose_blocks.restype = i32
        L.cgs_pose_blocks.argtypes = [vp, i64, i64, vp, vp, vp, vp, vp]
        L.cgs_partition_workspace_bytes.restype = i64
        L.cgs_partition_workspace_bytes.argtypes = [i64, vp]
        L.cgs_partition.restype = i32
        L.cgs_partition.argtypes = [vp, i64, i64, vp, vp, vp, vp, vp, vp, vp, vp, i64, vp]
        L.cgs_scatter_rows.restype = i32
        L.cgs_scatter_rows.argtypes = [vp, vp, i64, vp, i64, vp]
        L.cgs_partition_status.restype = i32
        L.cgs_partition_status.argtypes = [vp, vp]
        L.cgs_gather_rows.restype = i32
        L.cgs_gather_rows.argtypes = [vp, vp, i64, vp, i64, vp]
        L.cgs_debug_exp2.restype = i32
        L.cgs_debug_exp2.argtypes = [vp, i64, vp, vp]
        L.cgs_scene_bytes.restype = i64
        L.cgs_scene_bytes.argtypes = [i64, i32, i32, i32, i32]
        L.cgs_scene_upload.restype = i32
        L.cgs_scene_upload.argtypes = [P(cgs_scene), vp, i64, vp, vp, vp, vp, i64, i32, i32, i32, i32, vp, vp, vp,
                                       C.c_double, vp]
        L.cgs_pose_assign.restype = i32
        L.cgs_pose_assign.argtypes = [vp, vp, i32, i32, C.c_float, vp, vp, vp, vp]
        L.cgs_autotune_workspace_bytes.restype = i64
        L.cgs_autotune_workspace_bytes.argtypes = [i32, i32, i32, i32, i64, i64, i32, i32]
        L.cgs_autotune.restype = i32
        L.cgs_autotune.argtypes = [P(cgs_scene), vp, i32, i32, i32, vp, vp, i64, i64, i32, i32, vp, i64,
                                   P(cgs_config), P(C.c_float), C.c_char_p, C.c_char_p, vp]
        L.cgs_measure_peaks.restype = i32
        L.cgs_measure_peaks.argtypes = [P(C.c_double), i32, vp, i64, vp]
        _lib = L
    return _lib


class CgsError(RuntimeError):
    def __init__(self, code, where):
        super().__init__(f"{where}: {lib().cgs_status_string(code).decode()} (code {code})")
        self.code = code


def _check(code, where):
    if code != CGS_OK:
        raise CgsError(code, where)
    return code


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


# ---------------------------------------------------------------------------------------
# the C entry points, one for one
# ---------------------------------------------------------------------------------------
def cgs_version():
    return lib().cgs_version()


def cgs_status_string(code):
    return lib().cgs_status_string(code).decode()


def cgs_frame_workspace_bytes(n_views, width, height, tile, n_blocks, n_cap, k_cap):
    return lib().cgs_frame_workspace_bytes(n_views, width, height, tile, n_blocks, n_cap, k_cap)


def cgs_block_bounds_workspace_bytes(n):
    return lib().cgs_block_bounds_workspace_bytes(n)


def cgs_block_bounds(scene, n_mad, d_aabb, d_ws=None, ws_bytes=0, stream=None):
    return _check(lib().cgs_block_bounds(C.byref(scene), float(n_mad), _ptr(d_aabb), _ptr(d_ws), ws_bytes,
                                         _stream(stream)), "cgs_block_bounds")


def cgs_lod_select(scene, cfg, d_cams, n_views, d_levels, stream=None):
    return _check(lib().cgs_lod_select(C.byref(scene), C.byref(cfg), _ptr(d_cams), n_views, _ptr(d_levels),
                                       _stream(stream)), "cgs_lod_select")


def cgs_render_forward(scene, frame, cfg, d_cams, d_view_block, d_levels, d_image, d_final_T, d_n_contrib,
                       stream=None):
    return _check(lib().cgs_render_forward(C.byref(scene), C.byref(frame), C.byref(cfg), _ptr(d_cams),
                                           _ptr(d_view_block), _ptr(d_levels), _ptr(d_image), _ptr(d_final_T),
                                           _ptr(d_n_contrib), _stream(stream)), "cgs_render_forward")


def cgs_render_forward_static(scene, cfg, d_cam, width, height, d_view_block, d_levels, d_image, d_final_T,
                              d_n_contrib, d_status=None, stream=None):
    """Returns the host status code (no exception), so callers can see CGS_ERR_TOO_LARGE."""
    return lib().cgs_render_forward_static(C.byref(scene), C.byref(cfg), _ptr(d_cam), width, height,
                                           _ptr(d_view_block), _ptr(d_levels), _ptr(d_image), _ptr(d_final_T),
                                           _ptr(d_n_contrib), _ptr(d_status), _stream(stream))


def cgs_render_backward(scene, frame, cfg, d_cams, d_dL_dimage, d_final_T, d_n_contrib, d_g_mean_opac, d_g_scale,
                        d_g_quat, d_g_sh, stream=None):
    return _check(lib().cgs_render_backward(C.byref(scene), C.byref(frame), C.byref(cfg), _ptr(d_cams),
                                            _ptr(d_dL_dimage), _ptr(d_final_T), _ptr(d_n_contrib),
                                            _ptr(d_g_mean_opac), _ptr(d_g_scale), _ptr(d_g_quat), _ptr(d_g_sh),
                                            _stream(stream)), "cgs_render_backward")


def cgs_render_backward_packed(scene, frame, cfg, d_cams, d_dL_dimage, d_final_T, d_n_contrib, d_g_mean_opac,
                               d_g_scale, d_g_quat, d_g_sh, d_g_index, stream=None):
    return _check(lib().cgs_render_backward_packed(C.byref(scene), C.byref(frame), C.byref(cfg), _ptr(d_cams),
                                                   _ptr(d_dL_dimage), _ptr(d_final_T), _ptr(d_n_contrib),
                                                   _ptr(d_g_mean_opac), _ptr(d_g_scale), _ptr(d_g_quat),
                                                   _ptr(d_g_sh), _ptr(d_g_index), _stream(stream)),
                  "cgs_render_backward_packed")


def cgs_render_backward_l1(scene, frame, cfg, d_cams, d_image, d_target, target_u8, d_final_T, d_n_contrib,
                           d_loss, d_g_mean_opac, d_g_scale, d_g_quat, d_g_sh, d_g_index=None, stream=None):
    return _check(lib().cgs_render_backward_l1(C.byref(scene), C.byref(frame), C.byref(cfg), _ptr(d_cams),
                                               _ptr(d_image), _ptr(d_target), int(target_u8), _ptr(d_final_T),
                                               _ptr(d_n_contrib), _ptr(d_loss), _ptr(d_g_mean_opac),
                                               _ptr(d_g_scale), _ptr(d_g_quat), _ptr(d_g_sh), _ptr(d_g_index),
                                               _stream(stream)), "cgs_render_backward_l1")


def cgs_l1_loss(d_img, d_target, count, d_loss, d_grad, stream=None):
    return _check(lib().cgs_l1_loss(_ptr(d_img), _ptr(d_target), count, _ptr(d_loss), _ptr(d_grad),
                                    _stream(stream)), "cgs_l1_loss")


def cgs_l1_loss_u8(d_img, d_target, count, d_loss, d_grad, stream=None):
    return _check(lib().cgs_l1_loss_u8(_ptr(d_img), _ptr(d_target), count, _ptr(d_loss), _ptr(d_grad),
                                       _stream(stream)), "cgs_l1_loss_u8")


def cgs_frame_status(frame, stream=None):
    """Returns (status code, [selected, visible, entries, fwd pairs, bwd pairs, give-ups,
    fwd warp steps, useful fwd warp steps])."""
    st = C.c_int32(0)
    counts = (C.c_int64 * 8)()
    lib().cgs_frame_status(C.byref(frame), C.byref(st), counts, _stream(stream))
    return st.value, list(counts)


STAGES = ("select", "project", "duplicate", "sort", "render", "render_bwd", "project_bwd", "loss")


def cgs_timing_enable(on):
    return _check(lib().cgs_timing_enable(1 if on else 0), "cgs_timing_enable")


def cgs_timing_read():
    """Returns {stage: (milliseconds summed, launches)} since the previous read."""
    ms = (C.c_double * len(STAGES))()
    cnt = (C.c_int64 * len(STAGES))()
    _check(lib().cgs_timing_read(ms, cnt), "cgs_timing_read")
    return {s: (ms[i], cnt[i]) for i, s in enumerate(STAGES)}


def cgs_kernel_launches():
    return lib().cgs_kernel_launches()


def cgs_frame_buffer(frame, which):
    p = C.c_void_p(0)
    n = C.c_int64(0)
    _check(lib().cgs_frame_buffer(C.byref(frame), which, C.byref(p), C.byref(n)), "cgs_frame_buffer")
    return p.value, n.value


# ---------------------------------------------------------------------------------------
# block partition (Sec. 3.2.2, Eqs. 2 and 4); pmin, pmax, grid are host sequences
# ---------------------------------------------------------------------------------------
CGS_PARTITION_MAX_CELLS = 64
CGS_PARTITION_MAX_BLOCKS = 1024


def _host_f3(v):
    return (C.c_float * 3)(*[float(x) for x in v])


def _host_i3(v):
    return (C.c_int32 * 3)(*[int(x) for x in v])


def cgs_contract(d_pos, n, stride, pmin, pmax, d_out, stream=None):
    return _check(lib().cgs_contract(_ptr(d_pos), n, stride, _host_f3(pmin), _host_f3(pmax), _ptr(d_out),
                                     _stream(stream)), "cgs_contract")


def cgs_pose_blocks(d_pos, n, stride, pmin, pmax, grid, d_block, stream=None):
    return _check(lib().cgs_pose_blocks(_ptr(d_pos), n, stride, _host_f3(pmin), _host_f3(pmax), _host_i3(grid),
                                        _ptr(d_block), _stream(stream)), "cgs_pose_blocks")


def cgs_partition_workspace_bytes(n, grid):
    return lib().cgs_partition_workspace_bytes(n, _host_i3(grid))


def cgs_partition(d_pos, n, stride, pmin, pmax, grid, d_block, d_block_offset, d_perm, d_rank, d_ws, ws_bytes,
                  stream=None):
    return _check(lib().cgs_partition(_ptr(d_pos), n, stride, _host_f3(pmin), _host_f3(pmax), _host_i3(grid),
                                      _ptr(d_block), _ptr(d_block_offset), _ptr(d_perm), _ptr(d_rank), _ptr(d_ws),
                                      ws_bytes, _stream(stream)), "cgs_partition")


def cgs_scatter_rows(d_src, d_dst, row_bytes, d_rank, n_rows, stream=None):
    return _check(lib().cgs_scatter_rows(_ptr(d_src), _ptr(d_dst), row_bytes, _ptr(d_rank), n_rows,
                                         _stream(stream)), "cgs_scatter_rows")


def cgs_partition_status(d_ws, stream=None):
    return lib().cgs_partition_status(_ptr(d_ws), _stream(stream))


def cgs_gather_rows(d_src, d_dst, row_bytes, d_perm, n_rows, stream=None):
    return _check(lib().cgs_gather_rows(_ptr(d_src), _ptr(d_dst), row_bytes, _ptr(d_perm), n_rows,
                                        _stream(stream)), "cgs_gather_rows")


# ---------------------------------------------------------------------------------------
# detail levels (Sec. 3.3.1)
# ---------------------------------------------------------------------------------------
CGS_MAX_LEVELS = 16


def cgs_render_forward_hits(scene, frame, cfg, d_cams, d_view_block, d_levels, d_image, d_final_T, d_n_contrib,
                            d_hits, stream=None):
    return _check(lib().cgs_render_forward_hits(C.byref(scene), C.byref(frame), C.byref(cfg), _ptr(d_cams),
                                                _ptr(d_view_block), _ptr(d_levels), _ptr(d_image), _ptr(d_final_T),
                                                _ptr(d_n_contrib), _ptr(d_hits), _stream(stream)),
                  "cgs_render_forward_hits")


def cgs_levels_workspace_bytes(n, n_blocks):
    return lib().cgs_levels_workspace_bytes(n, n_blocks)


def cgs_generate_levels(d_mean_opac, d_scale, attr_fp16, n, d_block_offset, n_blocks, d_hits, rates, d_perm,
                        d_level_count, d_ws, ws_bytes, stream=None):
    r = (C.c_double * len(rates))(*[float(x) for x in rates])
    return _check(lib().cgs_generate_levels(_ptr(d_mean_opac), _ptr(d_scale), attr_fp16, n, _ptr(d_block_offset),
                                            n_blocks, _ptr(d_hits), r, len(rates), _ptr(d_perm),
                                            _ptr(d_level_count), _ptr(d_ws), ws_bytes, _stream(stream)),
                  "cgs_generate_levels")


def cgs_levels_status(d_ws, stream=None):
    return lib().cgs_levels_status(_ptr(d_ws), _stream(stream))


def cgs_ssim(d_a, a_stride, d_b, n_pairs, channels, width, height, d_ssim, d_map=None, stream=None):
    return _check(lib().cgs_ssim(_ptr(d_a), a_stride, _ptr(d_b), n_pairs, channels, width, height, _ptr(d_ssim),
                                 _ptr(d_map), _stream(stream)), "cgs_ssim")


# ---------------------------------------------------------------------------------------
# instrumentation
# ---------------------------------------------------------------------------------------
def cgs_debug_exp2(d_p, n, d_g, stream=None):
    return _check(lib().cgs_debug_exp2(_ptr(d_p), n, _ptr(d_g), _stream(stream)), "cgs_debug_exp2")


def cgs_measure_peaks(d_scratch, stream=None):
    """Measured issue rates of the current device (synchronises): FP32 lane operations per
    second from the scalar and the packed FMA loops, and base-2 exponentials per second."""
    r = (C.c_double * 3)()
    _check(lib().cgs_measure_peaks(r, 3, _ptr(d_scratch), d_scratch.numel(), _stream(stream)), "cgs_measure_peaks")
    return {"fp32_lane_ops_s": r[0], "fp32x2_lane_ops_s": r[1], "ex2_s": r[2]}


# ---------------------------------------------------------------------------------------
# scene upload, pose-to-block decision, autotuner
# ---------------------------------------------------------------------------------------
def _host(a):
    """Host pointer of a contiguous numpy array (kept alive by the caller)."""
    return None if a is None else a.ctypes.data


def cgs_scene_bytes(n, sh_degree, n_blocks, n_levels, attr_fp16=0):
    return lib().cgs_scene_bytes(n, sh_degree, n_blocks, n_levels, attr_fp16)


def cgs_scene_upload(d_mem, mem_bytes, h_mean_opac, h_scale, h_quat, h_sh, n, sh_degree, attr_fp16, h_level_offset,
                     h_level_count, h_block_cell, n_mad=-1.0, stream=None):
    """Host numpy arrays in, a cgs_scene over d_mem out."""
    out = cgs_scene()
    nb, nl = h_level_offset.shape
    _check(lib().cgs_scene_upload(C.byref(out), _ptr(d_mem), mem_bytes, _host(h_mean_opac), _host(h_scale),
                                  _host(h_quat), _host(h_sh), n, sh_degree, attr_fp16, nb, nl, _host(h_level_offset),
                                  _host(h_level_count), _host(h_block_cell), float(n_mad), _stream(stream)),
           "cgs_scene_upload")
    return out


def cgs_pose_assign(d_ssim, d_pose_block, n_poses, n_blocks, eps, d_b1=None, d_b2=None, d_b=None, stream=None):
    return _check(lib().cgs_pose_assign(_ptr(d_ssim), _ptr(d_pose_block), n_poses, n_blocks, float(eps), _ptr(d_b1),
                                        _ptr(d_b2), _ptr(d_b), _stream(stream)), "cgs_pose_assign")


def cgs_autotune_workspace_bytes(n_views, width, height, n_blocks, n_cap, k_cap, sh_degree, mode):
    return lib().cgs_autotune_workspace_bytes(n_views, width, height, n_blocks, n_cap, k_cap, sh_degree, mode)


def cgs_autotune(scene, d_cams, n_views, width, height, d_view_block, d_levels, n_cap, k_cap, mode, reps, d_ws,
                 ws_bytes, cfg, cache_path=None, cache_key=None, stream=None):
    """Returns {(tile, batch): median ms or -1}; writes the choice into cfg."""
    ms = (C.c_float * CGS_TUNE_CANDIDATES)()
    _check(lib().cgs_autotune(C.byref(scene), _ptr(d_cams), n_views, width, height, _ptr(d_view_block),
                              _ptr(d_levels), n_cap, k_cap, mode, reps, _ptr(d_ws), ws_bytes, C.byref(cfg), ms,
                              cache_path.encode() if cache_path else None, cache_key.encode() if cache_key else None,
                              _stream(stream)), "cgs_autotune")
    return {c: ms[i] for i, c in enumerate(TUNE_ORDER)}
