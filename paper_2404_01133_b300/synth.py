"""Seeded synthetic inputs: Gaussian scenes, block/level tables and pinhole cameras.

This module is shared by the CUDA path, the CPU oracle, the tests and the benchmark.
It only *draws* inputs; it contains none of the rendering method's arithmetic
(no projection, no spherical-harmonics evaluation, no compositing, no LoD rule).

Scene format (all arrays C-contiguous numpy, FP32 unless stated):

* ``mean_opac`` [N, 4]  world position x, y, z (metres, z up) and activated opacity o in (0, 1)
* ``scale``     [N, 4]  linear (activated) scales sx, sy, sz and an unused fourth lane
* ``quat``      [N, 4]  rotation quaternion (w, x, y, z), Hamilton convention
* ``sh``        [N, (deg+1)^2, 3]  SH coefficients, Gaussian-major, channel fastest
* ``sh_degree`` int in 0..3
* block table (optional): ``level_offset`` / ``level_count`` int64 [n_blocks, n_levels],
  ``block_cell`` FP32 [n_blocks, 4] = (x0, x1, y0, y1) of the block's ground cell.

The Gaussian record (position, opacity, scale + rotation, SH features in R^{3x16})
follows the scene representation of Sec. 3.1.  Detail levels are nested prefixes of
each block's Gaussians ranked by opacity x volume (the pruning rule that stands in
for LightGaussian compression, Sec. 3.3.1), level 0 = finest.

Camera format: dict with ``R`` (3x3 world->camera, row major, OpenCV axes: x right,
y down, z forward), ``t`` (3), ``campos`` (3, camera centre in world), ``fx fy cx cy``
and ``width height``.  Pixel (i, j) has its centre at the integer coordinate (i, j).
"""
from __future__ import annotations

import math
import numpy as np

SQRT_4PI = 2.0 * math.sqrt(math.pi)   # base colour c is stored as the DC coefficient (c - 0.5) * 2 sqrt(pi)


# ----------------------------------------------------------------------------------------
# cameras
# ----------------------------------------------------------------------------------------
def camera_from_rt(R, t, fx, fy, cx, cy, width, height):
    """Pinhole camera from a world->camera rotation R and translation t (x_cam = R x + t)."""
    R64 = np.asarray(R, dtype=np.float64).reshape(3, 3)
    t64 = np.asarray(t, dtype=np.float64).reshape(3)
    campos = -R64.T @ t64
    return {
        "R": R64.astype(np.float32), "t": t64.astype(np.float32),
        "campos": campos.astype(np.float32),
        "fx": float(np.float32(fx)), "fy": float(np.float32(fy)),
        "cx": float(np.float32(cx)), "cy": float(np.float32(cy)),
        "width": int(width), "height": int(height),
    }


def look_at(pos, target, up_hint, fx, fy, width, height, cx=None, cy=None):
    """Camera at ``pos`` looking at ``target``; ``up_hint`` fixes the roll (screen up)."""
    pos = np.asarray(pos, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - pos
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up_hint, dtype=np.float64))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f])
    t = -R @ pos
    if cx is None:
        cx = (width - 1) / 2.0
    if cy is None:
        cy = (height - 1) / 2.0
    return camera_from_rt(R, t, fx, fy, cx, cy, width, height)


def pitched_camera(pos, yaw, pitch_down, fx, fy, width, height):
    """Camera at ``pos`` with heading ``yaw`` (0 = +y, counter-clockwise) pitched down."""
    fwd = np.array([-math.sin(yaw) * math.cos(pitch_down), math.cos(yaw) * math.cos(pitch_down),
                    -math.sin(pitch_down)])
    if abs(math.sin(pitch_down)) > 1.0 - 1e-12:
        up = np.array([-math.sin(yaw), math.cos(yaw), 0.0])
    else:
        up = np.array([0.0, 0.0, 1.0])
    return look_at(pos, np.asarray(pos, dtype=np.float64) + fwd, up, fx, fy, width, height)


# ----------------------------------------------------------------------------------------
# attribute draws
# ----------------------------------------------------------------------------------------
def _attributes(rng, n, log_scale_mu, log_scale_sigma):
    """Scales, rotations, opacities and base colours of n Gaussians."""
    scale = np.exp(rng.normal(log_scale_mu, log_scale_sigma, size=(n, 3)))
    q = rng.normal(0.0, 1.0, size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    opac = 1.0 / (1.0 + np.exp(-rng.normal(0.0, 1.0, size=n)))
    base = rng.uniform(0.0, 1.0, size=(n, 3))
    scale4 = np.zeros((n, 4), dtype=np.float32)
    scale4[:, :3] = scale
    return scale4, q.astype(np.float32), opac, base


def sh_from_base(rng, base, sh_degree, hi_sigma=0.05, chunk=1 << 22):
    """SH coefficients [n, (deg+1)^2, 3]: DC from the base colours, higher orders N(0, hi_sigma)
    in FP32, drawn in chunks by torch's CPU generator (multithreaded) seeded from ``rng``."""
    import torch
    n = base.shape[0]
    n_coef = (sh_degree + 1) ** 2
    sh = np.empty((n, n_coef, 3), dtype=np.float32)
    sh[:, 0, :] = ((base - 0.5) * SQRT_4PI).astype(np.float32)
    if n_coef > 1:
        gen = torch.Generator().manual_seed(int(rng.integers(0, 2**62)))
        for c0 in range(0, n, chunk):
            c1 = min(n, c0 + chunk)
            block = torch.randn((c1 - c0, n_coef - 1, 3), generator=gen, dtype=torch.float32)
            sh[c0:c1, 1:, :] = block.numpy() * np.float32(hi_sigma)
    return sh


def _pack(mean, opac, scale4, quat, sh, sh_degree):
    n = mean.shape[0]
    mo = np.empty((n, 4), dtype=np.float32)
    mo[:, :3] = mean
    mo[:, 3] = opac
    return {"mean_opac": mo, "scale": np.ascontiguousarray(scale4), "quat": np.ascontiguousarray(quat),
            "sh": None if sh is None else np.ascontiguousarray(sh), "sh_degree": int(sh_degree)}


def random_cube_scene(n, seed=0, sh_degree=0, extent=1.0, log_scale_mu=-3.0, log_scale_sigma=0.5):
    """Means uniform in [-extent, extent]^3 (the 2,000-Gaussian 128x128 workload with defaults)."""
    rng = np.random.default_rng(seed)
    mean = rng.uniform(-extent, extent, size=(n, 3))
    scale4, quat, opac, base = _attributes(rng, n, log_scale_mu, log_scale_sigma)
    return _pack(mean, opac, scale4, quat, sh_from_base(rng, base, sh_degree), sh_degree)


def small_scene_camera(width=128, height=128, f=150.0, dist=4.0):
    """Camera at (0, 0, -dist) looking down +z with the principal point at the image centre."""
    return camera_from_rt(np.eye(3), [0.0, 0.0, dist], f, f, (width - 1) / 2.0, (height - 1) / 2.0,
                          width, height)


def city_points(rng, n, side, lot=50.0, p_build=0.5, foot=(10.0, 40.0), height=(5.0, 80.0),
                jitter=0.5, origin=(0.0, 0.0)):
    """Points on a synthetic city: ground plane plus random box buildings, jittered."""
    ox, oy = origin
    n_lot = max(1, int(side // lot))
    x0 = ox - side / 2.0
    y0 = oy - side / 2.0
    surf_o, surf_a, surf_b = [], [], []
    # ground
    surf_o.append((x0, y0, 0.0)); surf_a.append((side, 0.0, 0.0)); surf_b.append((0.0, side, 0.0))
    for li in range(n_lot):
        for lj in range(n_lot):
            if rng.uniform() >= p_build:
                continue
            w = rng.uniform(*foot)
            d = rng.uniform(*foot)
            h = rng.uniform(*height)
            cx = x0 + (li + 0.5) * lot
            cy = y0 + (lj + 0.5) * lot
            bx, by = cx - w / 2.0, cy - d / 2.0
            surf_o.append((bx, by, h)); surf_a.append((w, 0, 0)); surf_b.append((0, d, 0))      # roof
            surf_o.append((bx, by, 0)); surf_a.append((w, 0, 0)); surf_b.append((0, 0, h))      # south wall
            surf_o.append((bx, by + d, 0)); surf_a.append((w, 0, 0)); surf_b.append((0, 0, h))  # north wall
            surf_o.append((bx, by, 0)); surf_a.append((0, d, 0)); surf_b.append((0, 0, h))      # west wall
            surf_o.append((bx + w, by, 0)); surf_a.append((0, d, 0)); surf_b.append((0, 0, h))  # east wall
    so = np.asarray(surf_o, dtype=np.float64)
    sa = np.asarray(surf_a, dtype=np.float64)
    sb = np.asarray(surf_b, dtype=np.float64)
    area = np.linalg.norm(np.cross(sa, sb), axis=1)
    idx = rng.choice(len(area), size=n, p=area / area.sum())
    uv = rng.uniform(0.0, 1.0, size=(n, 2))
    pts = so[idx] + uv[:, :1] * sa[idx] + uv[:, 1:] * sb[idx]
    pts += rng.normal(0.0, jitter, size=(n, 3))
    return pts


def city_scene(n, area_km2, seed, sh_degree=3, origin=(0.0, 0.0), defer_sh=False):
    """Seeded aerial-city scene: n Gaussians over a square of area ``area_km2``.

    With defer_sh the SH coefficients are not drawn (``sh`` is None); the base colours are
    kept in ``base_colour`` so a later reordering can draw them in the final order."""
    rng = np.random.default_rng(seed)
    side = math.sqrt(area_km2) * 1000.0
    mean = city_points(rng, n, side, origin=origin)
    scale4, quat, opac, base = _attributes(rng, n, -1.0, 0.7)
    sh = None if defer_sh else sh_from_base(rng, base, sh_degree)
    sc = _pack(mean, opac, scale4, quat, sh, sh_degree)
    if defer_sh:
        sc["base_colour"] = base.astype(np.float32)
        sc["sh_seed"] = seed
    sc["side"] = side
    sc["origin"] = origin
    return sc


def unbounded_city(n, seed, area_km2=6.0, bg_frac=0.1, sh_degree=3, defer_sh=False):
    """An unbounded scene for the block partition: the aerial city of ``city_scene`` with a
    fraction ``bg_frac`` of its Gaussians moved to a far background (directions uniform on
    the upper hemisphere, distances log-uniform from 1 to 30 km), as an optimised global
    prior of a real capture has.  Returns the scene and its foreground box: the city square in
    x and y and, as Table S3 sets it, the minimum and maximum z of all Gaussians."""
    sc = city_scene(n, area_km2, seed, sh_degree=sh_degree, defer_sh=defer_sh)
    rng = np.random.default_rng(seed + 1000)
    nb = int(round(bg_frac * n))
    idx = np.sort(rng.choice(n, size=nb, replace=False))
    d = rng.normal(size=(nb, 3))
    d[:, 2] = np.abs(d[:, 2])
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = np.exp(rng.uniform(math.log(1000.0), math.log(30000.0), size=(nb, 1)))
    sc["mean_opac"][idx, :3] = (d * r).astype(np.float32)
    h = sc["side"] / 2.0
    z = sc["mean_opac"][:, 2]
    box = (np.array([-h, -h, z.min()], np.float32), np.array([h, h, z.max()], np.float32))
    return sc, box


def aerial_poses(side, n_poses, seed, alt=(150.0, 400.0)):
    """Camera centres of an aerial capture: uniform over a square of side ``side`` (1.2 times
    the city) at altitudes in ``alt``."""
    rng = np.random.default_rng(seed)
    xy = rng.uniform(-0.6 * side, 0.6 * side, size=(n_poses, 2))
    z = rng.uniform(alt[0], alt[1], size=(n_poses, 1))
    return np.concatenate([xy, z], axis=1).astype(np.float32)


# ----------------------------------------------------------------------------------------
# blocks and detail levels
# ----------------------------------------------------------------------------------------
def single_block(scene):
    """One block, one level, covering the whole scene (plain rendering without LoD)."""
    n = scene["mean_opac"].shape[0]
    sc = dict(scene)
    sc["level_offset"] = np.zeros((1, 1), dtype=np.int64)
    sc["level_count"] = np.full((1, 1), n, dtype=np.int64)
    big = np.float32(3.0e38)
    sc["block_cell"] = np.array([[-big, big, -big, big]], dtype=np.float32)
    return sc


def build_blocks(scene, grid, fractions=(1.0, 0.5, 0.25), extent=None):
    """Split a scene into a grid x grid xy block table with nested detail levels.

    Gaussians are regrouped block by block (block id = by * grid + bx) and, inside a block,
    ranked by opacity x volume in FP64 (descending, ties to the lower original index);
    level l keeps the top floor(N_j * fractions[l]).  Returns a new scene dict.
    """
    mo = scene["mean_opac"]
    n = mo.shape[0]
    if extent is None:
        side = scene["side"]
        ox, oy = scene.get("origin", (0.0, 0.0))
        extent = (ox - side / 2.0, ox + side / 2.0, oy - side / 2.0, oy + side / 2.0)
    x0, x1, y0, y1 = extent
    cw = (x1 - x0) / grid
    ch = (y1 - y0) / grid
    bx = np.clip(np.floor((mo[:, 0].astype(np.float64) - x0) / cw), 0, grid - 1).astype(np.int64)
    by = np.clip(np.floor((mo[:, 1].astype(np.float64) - y0) / ch), 0, grid - 1).astype(np.int64)
    blk = by * grid + bx
    sc = scene["scale"].astype(np.float64)
    score = mo[:, 3].astype(np.float64) * sc[:, 0] * sc[:, 1] * sc[:, 2]
    # by block, then by descending score, ties to the lower index (two stable sorts)
    order = np.argsort(-score, kind="stable")
    order = order[np.argsort(blk[order], kind="stable")]
    nb = grid * grid
    counts = np.bincount(blk, minlength=nb)
    starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
    L = len(fractions)
    level_offset = np.repeat(starts[:, None], L, axis=1).astype(np.int64)
    level_count = np.stack([np.floor(counts * f).astype(np.int64) for f in fractions], axis=1)
    cells = np.zeros((nb, 4), dtype=np.float32)
    for b in range(nb):
        i, j = b % grid, b // grid
        cells[b] = (x0 + i * cw, x0 + (i + 1) * cw, y0 + j * ch, y0 + (j + 1) * ch)
    if scene["sh"] is not None:
        sh = np.ascontiguousarray(scene["sh"][order])
    else:
        sh = sh_from_base(np.random.default_rng([scene["sh_seed"], 1]), scene["base_colour"][order],
                          scene["sh_degree"])
    out = {
        "mean_opac": np.ascontiguousarray(mo[order]),
        "scale": np.ascontiguousarray(scene["scale"][order]),
        "quat": np.ascontiguousarray(scene["quat"][order]),
        "sh": sh,
        "sh_degree": scene["sh_degree"],
        "level_offset": level_offset, "level_count": level_count, "block_cell": cells,
        "perm": order,
    }
    for k in ("side", "origin"):
        if k in scene:
            out[k] = scene[k]
    return out


# ----------------------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------------------
def workload_small(seed=0):
    """2,000 Gaussians in [-1,1]^3, SH degree 0, one 128x128 view, 16x16 tiles."""
    sc = single_block(random_cube_scene(2000, seed=seed, sh_degree=0))
    return sc, [small_scene_camera()]


def workload_city_1m(seed=2, n=1_000_000, width=1920, height=1080):
    """1M-Gaussian SH-3 city over 1.5 km^2, one 1920x1080 view from 150 m pitched 45 deg."""
    sc = single_block(city_scene(n, 1.5, seed, sh_degree=3))
    cam = pitched_camera((0.0, 0.0, 150.0), 0.0, math.radians(45.0), 1200.0, 1200.0, width, height)
    return sc, [cam]


def target_image(seed, width, height):
    """Seeded U[0,1] target image, planar [3, H, W]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, size=(3, height, width)).astype(np.float32)


def target_image_u8(seed, width, height):
    """Seeded 8-bit target image (uniform channel values 0..255), planar [3, H, W]."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, 256, size=(3, height, width), dtype=np.uint8)


def workload_city_lod(n=20_000_000, grid=8, seed=3, heights=(50.0, 200.0, 500.0, 1000.0, 2000.0),
                      width=1920, height=1080):
    """Block-LoD city (6 km^2, grid x grid blocks, 3 nested levels) and top-down cameras."""
    sc = build_blocks(city_scene(n, 6.0, seed, sh_degree=3, defer_sh=True), grid)
    cams = [pitched_camera((0.0, 0.0, z), 0.0, math.pi / 2.0, 1200.0, 1200.0, width, height)
            for z in heights]
    return sc, cams


def lod_pose_queue(side, n_poses=64, seed=5, width=1920, height=1080):
    """Seeded top-down poses: xy uniform over the extent, height log-uniform in 30-2500 m."""
    rng = np.random.default_rng(seed)
    cams = []
    for _ in range(n_poses):
        x, y = rng.uniform(-side / 2.0, side / 2.0, size=2)
        z = math.exp(rng.uniform(math.log(30.0), math.log(2500.0)))
        yaw = rng.uniform(0.0, 2.0 * math.pi)
        cams.append(pitched_camera((x, y, z), yaw, math.pi / 2.0, 1200.0, 1200.0, width, height))
    return cams


def training_blocks(n_blocks=32, views_per_block=8, seed=4, lo=200_000, hi=3_000_000,
                    width=1600, height=900, density_per_km2=1_000_000 / 1.5, scale_counts=1.0):
    """Blocks with log-uniform Gaussian counts, each a city patch, plus per-block views.

    Returns (scene with one level per block, cameras, view->block map).
    """
    rng = np.random.default_rng(seed)
    counts = np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_blocks))
    counts = np.maximum(1, np.floor(counts * scale_counts)).astype(np.int64)
    parts, cams, vb = [], [], []
    for b in range(n_blocks):
        area = counts[b] / density_per_km2
        origin = (b * 4000.0, 0.0)
        part = city_scene(int(counts[b]), area, seed * 1000 + b, sh_degree=3, origin=origin)
        parts.append(part)
        half = part["side"] / 2.0
        for _ in range(views_per_block):
            px = origin[0] + rng.uniform(-half, half)
            py = origin[1] + rng.uniform(-half, half)
            pz = rng.uniform(100.0, 400.0)
            cams.append(look_at((px, py, pz), (origin[0], origin[1], 0.0), (0.0, 0.0, 1.0),
                                1000.0, 1000.0, width, height))
            vb.append(b)
    sc = {
        "mean_opac": np.concatenate([p["mean_opac"] for p in parts]),
        "scale": np.concatenate([p["scale"] for p in parts]),
        "quat": np.concatenate([p["quat"] for p in parts]),
        "sh": np.concatenate([p["sh"] for p in parts], axis=0),
        "sh_degree": 3,
    }
    starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
    sc["level_offset"] = starts[:, None].astype(np.int64)
    sc["level_count"] = counts[:, None].astype(np.int64)
    cells = np.zeros((n_blocks, 4), dtype=np.float32)
    for b, p in enumerate(parts):
        ox, oy = p["origin"]
        h = p["side"] / 2.0
        cells[b] = (ox - h, ox + h, oy - h, oy + h)
    sc["block_cell"] = cells
    return sc, cams, np.asarray(vb, dtype=np.int32)
