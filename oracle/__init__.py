"""CPU oracle for the CityGaussian hot path -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  It wraps ``oracle.c`` (plain single-threaded C, compiled by
``oracle/build.py``) through ctypes; it shares no code with the CUDA library.

Two builds exist: ``f32`` (the parity build: every value in FP32, operation order as
documented in oracle.c) and ``f64`` (values and decisions in FP64, used for the
finite-difference pins).  In both, the key path that decides integers (culls, radius,
tile rect, depth bits) is FP32.

Paper passages: Eq. 1 and Sec. 3.1 (projection, SH colour, depth-sorted alpha blending,
differentiable rendering); Sec. 3.3.1 (nested detail levels from a significance ranking);
Sec. 3.2.2, Eqs. 2 and 4 (normalisation, contraction, block grid,
pose in block); Eq. 7 and Sec. 3.3.2 (MAD block bounds, block frustum test,
camera block, distance-based level, concatenation).
"""
from __future__ import annotations

import ctypes as C
import numpy as np

from . import build as _build

F_CULL_NEAR, F_CULL_DET, F_CLAMP_X, F_CLAMP_Y = 1, 2, 4, 8
F_CLAMP_RGB = (16, 32, 64)


class OrcCamera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("campos", C.c_float * 3),
                ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("width", C.c_int32), ("height", C.c_int32)]


class OrcConfig(C.Structure):
    _fields_ = [("tile", C.c_int32), ("near_z", C.c_float), ("bg", C.c_float * 3)]


def make_camera(cam):
    c = OrcCamera()
    c.R[:] = [float(v) for v in np.asarray(cam["R"], dtype=np.float32).reshape(9)]
    c.t[:] = [float(v) for v in np.asarray(cam["t"], dtype=np.float32)]
    c.campos[:] = [float(v) for v in np.asarray(cam["campos"], dtype=np.float32)]
    c.fx, c.fy, c.cx, c.cy = cam["fx"], cam["fy"], cam["cx"], cam["cy"]
    c.width, c.height = cam["width"], cam["height"]
    return c


def make_config(tile=16, near_z=0.2, bg=(0.0, 0.0, 0.0)):
    c = OrcConfig()
    c.tile = tile
    c.near_z = near_z
    c.bg[:] = list(bg)
    return c


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


_LIBS = {}


def lib(real="f32"):
    if real not in _LIBS:
        _build.build()
        L = C.CDLL(_build.lib_path(real))
        vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
        L.orc_project.restype = i64
        L.orc_project.argtypes = [i64, vp, vp, vp, vp, i32, vp, vp] + [vp] * 9
        L.orc_emit_keys.restype = i64
        L.orc_emit_keys.argtypes = [i64, vp, vp, vp, i32, vp, vp, i64]
        L.orc_sort_pairs.argtypes = [i64, vp, vp]
        L.orc_tile_ranges.argtypes = [i64, vp, i32, vp]
        L.orc_composite.restype = i64
        L.orc_composite.argtypes = [i64, vp, vp, vp, vp, vp, vp, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp]
        L.orc_composite_brute.argtypes = [i64, vp, vp, vp, vp, vp, vp, i32, i32, vp, vp, vp]
        L.orc_composite_backward.argtypes = [i64, vp, vp, vp, vp, vp, vp, i32, i32, vp, vp, vp, vp, vp, vp, vp]
        L.orc_project_backward.argtypes = [i64, vp, vp, vp, vp, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.orc_l1.argtypes = [i64, vp, vp, vp, vp]
        L.orc_block_bounds.argtypes = [i32, i32, vp, vp, vp, C.c_double, vp]
        L.orc_lod_select.argtypes = [i32, i32, vp, vp, vp, vp, C.c_float, vp, vp]
        L.orc_concat.restype = i64
        L.orc_concat.argtypes = [i32, i32, vp, vp, vp, vp]
        L.orc_sh_basis.argtypes = [i64, vp, i32, vp, vp]
        L.orc_pointwise_select.restype = i64
        L.orc_pointwise_select.argtypes = [i32, i32, vp, vp, vp, vp, vp, vp]
        L.orc_contract.argtypes = [i64, vp, i64, vp, vp, vp]
        L.orc_partition_assign.restype = i64
        L.orc_partition_assign.argtypes = [i64, vp, i64, vp, vp, vp, vp, vp]
        L.orc_partition_order.argtypes = [i64, vp, i32, vp, vp]
        L.orc_hit_counts.argtypes = [i64, vp, vp, vp, vp, vp, vp, i32, i32, vp, vp, vp]
        L.orc_generate_levels.argtypes = [i32, vp, vp, vp, vp, vp, i32, vp, vp, vp]
        L.orc_ssim.restype = C.c_double
        L.orc_ssim.argtypes = [i32, i32, i32, vp, vp, vp]
        L.orc_real_bytes.restype = i32
        _LIBS[real] = L
    return _LIBS[real]


def _dtype(real):
    return np.float32 if real == "f32" else np.float64


def _scene_arrays(scene, real, idx=None):
    dt = _dtype(real)
    mo, sc, q, sh = scene["mean_opac"], scene["scale"], scene["quat"], scene["sh"]
    if idx is not None:
        mo, sc, q, sh = mo[idx], sc[idx], q[idx], sh[idx]
    return (np.ascontiguousarray(mo, dtype=dt), np.ascontiguousarray(sc, dtype=dt),
            np.ascontiguousarray(q, dtype=dt), np.ascontiguousarray(sh, dtype=dt))


def project(scene, cam, cfg=None, real="f32", idx=None, arrays=None):
    """Per-Gaussian projection records (Eq. 1's proj) and tile rects."""
    cfg = cfg or make_config()
    L = lib(real)
    dt = _dtype(real)
    mo, sc, q, sh = arrays if arrays is not None else _scene_arrays(scene, real, idx)
    n = mo.shape[0]
    out = {
        "depth": np.zeros(n, np.float32), "radius": np.zeros(n, np.int32), "rect": np.zeros((n, 4), np.int32),
        "tiles_touched": np.zeros(n, np.int64), "xy": np.zeros((n, 2), dt), "cov2d": np.zeros((n, 3), dt),
        "conic": np.zeros((n, 3), dt), "rgb": np.zeros((n, 3), dt), "flags": np.zeros(n, np.int32),
    }
    c = make_camera(cam)
    k = L.orc_project(n, _p(mo), _p(sc), _p(q), _p(sh), scene["sh_degree"], C.byref(c), C.byref(cfg),
                      _p(out["depth"]), _p(out["radius"]), _p(out["rect"]), _p(out["tiles_touched"]),
                      _p(out["xy"]), _p(out["cov2d"]), _p(out["conic"]), _p(out["rgb"]), _p(out["flags"]))
    out["n_entries"] = int(k)
    out["arrays"] = (mo, sc, q, sh)
    return out


def tiles_xy(cam, tile):
    return (cam["width"] + tile - 1) // tile, (cam["height"] + tile - 1) // tile


def bin_and_sort(pr, cam, cfg=None, real="f32"):
    """(tile | depth bits, index) keys, sorted, and per-tile ranges."""
    cfg = cfg or make_config()
    L = lib(real)
    tx, ty = tiles_xy(cam, cfg.tile)
    k = pr["n_entries"]
    keys = np.zeros(max(k, 1), np.uint64)
    vals = np.zeros(max(k, 1), np.uint32)
    n = pr["depth"].shape[0]
    got = L.orc_emit_keys(n, _p(pr["depth"]), _p(pr["rect"]), _p(pr["tiles_touched"]), tx, _p(keys), _p(vals), k)
    assert got == k
    unsorted = (keys[:k].copy(), vals[:k].copy())
    L.orc_sort_pairs(k, _p(keys), _p(vals))
    ranges = np.zeros((tx * ty, 2), np.int64)
    L.orc_tile_ranges(k, _p(keys), tx * ty, _p(ranges))
    return {"keys": keys[:k], "vals": vals[:k], "ranges": ranges, "unsorted": unsorted}


def composite(pr, srt, cam, cfg=None, real="f32", tile_mask=None):
    cfg = cfg or make_config()
    L = lib(real)
    dt = _dtype(real)
    W, H = cam["width"], cam["height"]
    mo = pr["arrays"][0]
    n = mo.shape[0]
    out = {"image": np.zeros((3, H, W), dt), "final_T": np.zeros((H, W), dt),
           "n_contrib": np.zeros((H, W), np.int32), "n_visited": np.zeros((H, W), np.int32),
           "ambiguous": np.zeros((H, W), np.uint8)}
    h = C.c_uint64(0)
    tm = None if tile_mask is None else np.ascontiguousarray(tile_mask, dtype=np.uint8)
    vals = srt["vals"] if srt["vals"].size else np.zeros(1, np.uint32)
    pairs = L.orc_composite(n, _p(pr["xy"]), _p(pr["conic"]), _p(mo), _p(pr["rgb"]), _p(vals),
                            _p(srt["ranges"]), W, H, C.byref(cfg), _p(tm), _p(out["image"]), _p(out["final_T"]),
                            _p(out["n_contrib"]), _p(out["n_visited"]), _p(out["ambiguous"]), C.byref(h))
    out["pairs"] = int(pairs)
    out["hash"] = int(h.value)
    return out


def render(scene, cam, cfg=None, real="f32", idx=None, tile_mask=None):
    """Full forward: project, bin, sort, range, composite.  ``idx`` selects a subset (LoD)."""
    cfg = cfg or make_config()
    pr = project(scene, cam, cfg, real, idx)
    srt = bin_and_sort(pr, cam, cfg, real)
    out = composite(pr, srt, cam, cfg, real, tile_mask)
    out["proj"] = pr
    out["sort"] = srt
    return out


def composite_brute(pr, cam, cfg=None, real="f32"):
    cfg = cfg or make_config()
    L = lib(real)
    dt = _dtype(real)
    W, H = cam["width"], cam["height"]
    mo = pr["arrays"][0]
    img = np.zeros((3, H, W), dt)
    T = np.zeros((H, W), dt)
    L.orc_composite_brute(mo.shape[0], _p(pr["xy"]), _p(pr["conic"]), _p(mo), _p(pr["rgb"]), _p(pr["depth"]),
                          _p(pr["flags"]), W, H, C.byref(cfg), _p(img), _p(T))
    return img, T


def render_backward(scene, cam, dL_dimage, cfg=None, real="f32", idx=None, fwd=None, tile_mask=None):
    """Analytic gradient of sum(dL_dimage * image) w.r.t. every Gaussian attribute
    (restricted to the pixels of the tiles in ``tile_mask`` when given)."""
    cfg = cfg or make_config()
    L = lib(real)
    dt = _dtype(real)
    if fwd is None:
        fwd = render(scene, cam, cfg, real, idx)
    pr, srt = fwd["proj"], fwd["sort"]
    mo, sc, q, sh = pr["arrays"]
    n = mo.shape[0]
    W, H = cam["width"], cam["height"]
    g2 = {"xy": np.zeros((n, 2), dt), "conic": np.zeros((n, 3), dt), "opac": np.zeros(n, dt),
          "rgb": np.zeros((n, 3), dt)}
    gimg = np.ascontiguousarray(dL_dimage, dtype=dt)
    vals = srt["vals"] if srt["vals"].size else np.zeros(1, np.uint32)
    tm = None if tile_mask is None else np.ascontiguousarray(tile_mask, dtype=np.uint8)
    L.orc_composite_backward(n, _p(pr["xy"]), _p(pr["conic"]), _p(mo), _p(pr["rgb"]), _p(vals), _p(srt["ranges"]),
                             W, H, C.byref(cfg), _p(tm), _p(gimg), _p(g2["xy"]), _p(g2["conic"]), _p(g2["opac"]),
                             _p(g2["rgb"]))
    g = {"mean": np.zeros((n, 3), dt), "scale": np.zeros((n, 3), dt), "quat": np.zeros((n, 4), dt),
         "opac": np.zeros(n, dt), "sh": np.zeros_like(sh)}
    c = make_camera(cam)
    L.orc_project_backward(n, _p(mo), _p(sc), _p(q), _p(sh), scene["sh_degree"], C.byref(c), C.byref(cfg),
                           _p(pr["tiles_touched"]), _p(g2["xy"]), _p(g2["conic"]), _p(g2["opac"]), _p(g2["rgb"]),
                           _p(g["mean"]), _p(g["scale"]), _p(g["quat"]), _p(g["opac"]), _p(g["sh"]))
    g["screen"] = g2
    g["fwd"] = fwd
    return g


def l1(img, target, real="f32"):
    L = lib(real)
    dt = _dtype(real)
    a = np.ascontiguousarray(img, dtype=dt)
    b = np.ascontiguousarray(target, dtype=dt)
    grad = np.zeros_like(a)
    loss = C.c_double(0)
    L.orc_l1(a.size, _p(a), _p(b), _p(grad), C.byref(loss))
    return loss.value, grad


def block_bounds(scene, n_mad=4.0):
    lo = np.ascontiguousarray(scene["level_offset"], np.int64)
    lc = np.ascontiguousarray(scene["level_count"], np.int64)
    nb, nl = lo.shape
    out = np.zeros((nb, 6), np.float32)
    mo = np.ascontiguousarray(scene["mean_opac"], np.float32)
    lib("f64").orc_block_bounds(nb, nl, _p(lo), _p(lc), _p(mo), float(n_mad), _p(out))
    return out


def lod_select(scene, aabb, cam, dist=(200.0, 600.0), near_z=0.2):
    lc = np.ascontiguousarray(scene["level_count"], np.int64)
    nb, nl = lc.shape
    lev = np.zeros(nb, np.int8)
    c = make_camera(cam)
    d = np.asarray(dist, np.float64)
    cell = np.ascontiguousarray(scene["block_cell"], np.float32)
    lib("f64").orc_lod_select(nb, nl, _p(lc), _p(np.ascontiguousarray(aabb, np.float32)), _p(cell), C.byref(c),
                              near_z, _p(d), _p(lev))
    return lev


def concat(scene, level):
    lo = np.ascontiguousarray(scene["level_offset"], np.int64)
    lc = np.ascontiguousarray(scene["level_count"], np.int64)
    nb, nl = lo.shape
    lev = np.ascontiguousarray(level, np.int8)
    total = int(sum(lc[b, lev[b]] for b in range(nb) if lev[b] >= 0))
    out = np.zeros(max(total, 1), np.int64)
    m = lib("f64").orc_concat(nb, nl, _p(lo), _p(lc), _p(lev), _p(out))
    return out[:m]


def pointwise_select(scene, cam, dist=(200.0, 600.0)):
    """Global indices kept by the point-wise level baseline (see oracle.c)."""
    lo = np.ascontiguousarray(scene["level_offset"], np.int64)
    lc = np.ascontiguousarray(scene["level_count"], np.int64)
    nb, nl = lo.shape
    mo = np.ascontiguousarray(scene["mean_opac"], np.float32)
    out = np.zeros(max(int(lc[:, 0].sum()), 1), np.int64)
    c = make_camera(cam)
    d = np.asarray(dist, np.float64)
    m = lib("f64").orc_pointwise_select(nb, nl, _p(lo), _p(lc), _p(mo), C.byref(c), _p(d), _p(out))
    return out[:m]


def sh_basis(dirs, deg=3, real="f64", with_grad=False):
    dt = _dtype(real)
    d = np.ascontiguousarray(dirs, dtype=dt).reshape(-1, 3)
    out = np.zeros((d.shape[0], 16), dt)
    dout = np.zeros((d.shape[0], 16, 3), dt) if with_grad else None
    lib(real).orc_sh_basis(d.shape[0], _p(d), deg, _p(out), _p(dout))
    return (out, dout) if with_grad else out


# ---- block partition (Sec. 3.2.2, Eqs. 2 and 4) -------------------------------------------

def _pos_rows(pos):
    a = np.ascontiguousarray(pos, dtype=np.float32)
    return a, a.shape[1]


def contract(pos, pmin, pmax):
    """Eq. 2 applied to the normalised positions (rows of pos, xyz first), FP32."""
    a, stride = _pos_rows(pos)
    out = np.zeros((a.shape[0], 3), np.float32)
    pl, ph = np.asarray(pmin, np.float32), np.asarray(pmax, np.float32)
    lib().orc_contract(a.shape[0], _p(a), stride, _p(pl), _p(ph), _p(out))
    return out


def partition_assign(pos, pmin, pmax, grid):
    """Block of every point over the uniform grid of the contracted cube, and the per-block
    counts; block -1 for a point whose contraction is not finite."""
    a, stride = _pos_rows(pos)
    g = np.asarray(grid, np.int32)
    nb = int(np.prod(g))
    block = np.zeros(a.shape[0], np.int32)
    count = np.zeros(nb, np.int64)
    pl, ph = np.asarray(pmin, np.float32), np.asarray(pmax, np.float32)
    dropped = lib().orc_partition_assign(a.shape[0], _p(a), stride, _p(pl), _p(ph), _p(g), _p(block), _p(count))
    return {"block": block, "count": count, "dropped": int(dropped)}


def partition_order(block, n_blocks):
    """Stable grouping by block: permutation (grouped position -> scene index) and offsets."""
    b = np.ascontiguousarray(block, np.int32)
    perm = np.zeros(max(1, b.shape[0]), np.int64)
    offset = np.zeros(n_blocks + 1, np.int64)
    lib().orc_partition_order(b.shape[0], _p(b), n_blocks, _p(perm), _p(offset))
    return perm[:offset[-1]], offset


def pose_blocks(campos, pmin, pmax, grid):
    """Eq. 4 (B2): the block that contains each camera centre after normalisation and
    contraction."""
    return partition_assign(np.asarray(campos, np.float32).reshape(-1, 3), pmin, pmax, grid)["block"]


# ---- detail levels (Sec. 3.3.1) ----------------------------------------------------------

def hit_counts(scene, cams, cfg=None, idx=None):
    """Pixels blending each scene Gaussian, summed over the views: (hits, unsure) as int64
    arrays over the scene, unsure counting the pixels where that Gaussian's own decision lies
    within a rounding margin of its threshold (idx selects the rendered subset, as in render)."""
    cfg = cfg or make_config()
    L = lib("f32")
    n_scene = scene["mean_opac"].shape[0]
    hits = np.zeros(n_scene, np.int64)
    amb = np.zeros(n_scene, np.int64)
    for cam in cams:
        pr = project(scene, cam, cfg, idx=idx)
        srt = bin_and_sort(pr, cam, cfg)
        n = pr["depth"].shape[0]
        h = np.zeros(n, np.int64)
        a = np.zeros(n, np.int64)
        vals = srt["vals"] if srt["vals"].size else np.zeros(1, np.uint32)
        L.orc_hit_counts(n, _p(pr["xy"]), _p(pr["conic"]), _p(pr["arrays"][0]), _p(pr["rgb"]), _p(vals),
                         _p(srt["ranges"]), cam["width"], cam["height"], C.byref(cfg), _p(h), _p(a))
        rows = np.arange(n_scene) if idx is None else np.asarray(idx)
        np.add.at(hits, rows, h)
        np.add.at(amb, rows, a)
    return hits, amb


def generate_levels(scene, rates, hits=None):
    """Nested levels of a block-grouped scene (one level per block in level_offset /
    level_count on input): the ranked permutation and level_count [n_blocks][len(rates)]."""
    off = np.ascontiguousarray(scene["level_offset"][:, 0], np.int64)
    cnt = np.ascontiguousarray(scene["level_count"][:, 0], np.int64)
    nb = off.shape[0]
    mo = np.ascontiguousarray(scene["mean_opac"], np.float32)
    sc = np.ascontiguousarray(scene["scale"], np.float32)
    n = mo.shape[0]
    perm = np.arange(n, dtype=np.int64)
    r = np.ascontiguousarray(rates, np.float64)
    lc = np.zeros((nb, len(r)), np.int64)
    h = None if hits is None else np.ascontiguousarray(hits, np.int64)
    lib("f32").orc_generate_levels(nb, _p(off), _p(cnt), _p(mo), _p(sc), _p(h), len(r), _p(r), _p(perm), _p(lc))
    return perm, lc


# ---- SSIM (Eq. 3) --------------------------------------------------------------------------

def ssim(a, b, with_map=False):
    """Mean SSIM of two [C, H, W] images (11x11 Gaussian window, sigma 1.5, zero padding),
    FP64; with_map also returns the per-pixel map averaged over channels."""
    A = np.ascontiguousarray(a, np.float32)
    B = np.ascontiguousarray(b, np.float32)
    c, h, w = A.shape
    m = np.zeros((h, w), np.float64) if with_map else None
    v = lib("f32").orc_ssim(c, w, h, _p(A), _p(B), _p(m))
    return (v, m) if with_map else v


def pose_assign_b1(full, without, eps):
    """Eq. 3: B1 = 1 where the SSIM loss 1 - SSIM(render with all blocks, render without block
    j) exceeds eps; `without` is a sequence of renders, one per block."""
    return np.array([1 - ssim(full, w) > eps for w in without], dtype=bool)
