"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI and compare it
with the CPU oracle on the same seeded inputs."""
import numpy as np
import torch

import oracle
from paper_2404_01133_b300 import cgs
from paper_2404_01133_b300 import torch_api as ta

# Pixel tolerance in FP32 (spec bound) for pixels whose skip/stop decisions are not
# within the oracle's ambiguity margins.
PIX_ATOL = 1e-4
# An ambiguous pixel may take the other branch of one near-threshold decision.  A flipped 1/255
# skip changes the pixel by at most alpha T c_max <= c_max / 255 (the entry's own colour and
# the 1 - alpha scaling of everything behind it, each at most that, with opposite signs), and
# the 1 - 1/255 change of T it causes can flip a later 1e-4 stop, one blend of at most
# 0.99 * 0.01 * c_max (the stop happens only once T < 1e-2).  Per unit of the largest colour:
AMB_ATOL_PER_C = 1.0 / 255.0 + 0.0099 + 1e-4
# Most ambiguous pixels a frame may have, per pair its compositing evaluates.  The oracle's
# margins are rigorous rounding bounds (oracle.c): near 1/255 about 7e-6 relative on alpha for
# these scenes, so a pair is flagged when ln(alpha) lies in a window about 1.4e-5 wide around
# ln(1/255); measured on a B300, 0.3e-6 to 5.8e-6 of the evaluated pairs flag their pixel
# (1.0e-6 on the 1080p city frame: 141 of its 2,073,600 pixels; the most, 5.8e-6, on scenes
# of needle-like Gaussians, whose power terms cancel and so widen the margin).  The bound
# keeps the margins honest: a looser margin would exempt more pixels from the 1e-4 check and
# fail it.
AMB_PER_PAIR_MAX = 1e-5
AMB_MIN_ALLOWED = 4  # small frames: at most this many pixels whatever the pair count


def amb_atol(rgb):
    """Error bound of an ambiguous pixel for projected colours rgb (any shape)."""
    return AMB_ATOL_PER_C * max(1.0, float(np.max(rgb))) if np.size(rgb) else AMB_ATOL_PER_C


# backwards compatible name: the bound for colours at most 1
AMB_ATOL = AMB_ATOL_PER_C


def fp16_rounded(scene):
    """The scene with scale, rotation and SH rounded to IEEE half and widened back to FP32:
    the values the FP16 attribute storage variant computes with."""
    out = dict(scene)
    for k in ("scale", "quat", "sh"):
        out[k] = np.asarray(scene[k], np.float32).astype(np.float16).astype(np.float32)
    return out


def gpu_render(scene, cams, tile=16, batch=None, n_cap=None, k_cap=None, view_block=None, levels=None,
               n_mad=None, cfg_kw=None, fp16=False):
    ds = ta.DeviceScene(scene, fp16=fp16)
    if n_mad is not None:
        ds.compute_block_bounds(n_mad)
    cfg = ta.make_config(tile=tile, batch=batch, **(cfg_kw or {}))
    W, H = cams[0]["width"], cams[0]["height"]
    n_cap = n_cap or max(1, ds.n * len(cams))
    k_cap = k_cap or max(1024, 64 * n_cap)
    k_cap = min(k_cap, (1 << 30) - 1)
    frame = ta.Frame(len(cams), W, H, tile, ds.n_blocks, n_cap, k_cap)
    d_cams = ta.cameras_device(cams)
    vb = None if view_block is None else torch.as_tensor(np.asarray(view_block, np.int32)).cuda()
    lv = None if levels is None else torch.as_tensor(np.asarray(levels, np.int8)).cuda()
    img, T, nc = ta.render_forward(ds, frame, cfg, d_cams, vb, lv)
    st, counts = frame.status()
    return {"ds": ds, "cfg": cfg, "frame": frame, "cams": d_cams, "image": img, "final_T": T, "n_contrib": nc,
            "status": st, "counts": counts, "view_block": vb, "levels": lv}


def frame_arrays(g, n_sel=None, k=None):
    fr = g["frame"]
    n_sel = n_sel if n_sel is not None else g["counts"][0]
    k = k if k is not None else g["counts"][2]
    out = {
        "tiles_touched": fr.buffer(cgs.BUF_TILES_TOUCHED, torch.int32, count=n_sel).cpu().numpy().view(np.uint32),
        "scene_index": fr.buffer(cgs.BUF_SCENE_INDEX, torch.int32, count=n_sel).cpu().numpy().view(np.uint32),
        "records": fr.buffer(cgs.BUF_RECORDS, torch.float32, (12,), count=n_sel).cpu().numpy(),
        "keys": fr.buffer(cgs.BUF_TILE_KEYS, torch.int32, count=k).cpu().numpy().view(np.uint32),
        "vals": fr.buffer(cgs.BUF_TILE_VALS, torch.int32, count=k).cpu().numpy().view(np.uint32),
        "depth_keys": fr.buffer(cgs.BUF_DEPTH_KEYS, torch.int64, count=n_sel).cpu().numpy().view(np.uint64),
        "rects": fr.buffer(cgs.BUF_RECTS, torch.int32, (2,), count=n_sel).cpu().numpy().view(np.uint32),
    }
    V, T = fr.n_views, ((fr.width + fr.tile - 1) // fr.tile) * ((fr.height + fr.tile - 1) // fr.tile)
    out["ranges"] = fr.buffer(cgs.BUF_RANGES, torch.int32, (2,), count=V * T).cpu().numpy().view(np.uint32)
    return out


def canonical_ranges(r, first=0):
    """Per-tile [start, end) with empty tiles written as [0, 0] (the oracle's form; the GPU
    leaves an empty tile at [e, e], the running offset, which is equally empty)."""
    r = np.asarray(r, np.int64)
    return np.where(r[:, 1:] > r[:, :1], r - first, 0)


def compare_image(gimg, gT, gnc, o, rgb_max=None, label=""):
    """Pixels within PIX_ATOL and n_contrib equal where the oracle saw no near-threshold
    decision; ambiguous pixels within amb_atol and at most AMB_PER_PAIR_MAX per evaluated pair.  Prints
    and returns the counts: ambiguous pixels, and those among them that actually differ."""
    amb = o["ambiguous"].astype(bool)
    img = gimg.detach().cpu().numpy()
    T = gT.detach().cpu().numpy()
    nc = gnc.detach().cpu().numpy()
    oi = o["image"].astype(np.float32)
    ok = ~amb
    err = np.abs(img - oi).max(axis=0)
    assert err[ok].max(initial=0.0) <= PIX_ATOL, (err[ok].max(), np.argwhere(err > PIX_ATOL)[:5])
    assert np.abs(T - o["final_T"])[ok].max(initial=0.0) <= PIX_ATOL
    bad = (nc != o["n_contrib"]) & ok
    assert not bad.any(), np.argwhere(bad)[:5]
    n_amb = int(amb.sum())
    if rgb_max is None:
        rgb_max = o["proj"]["rgb"] if "proj" in o else 1.0
    lim = amb_atol(rgb_max)
    differ = amb & ((err > PIX_ATOL) | (nc != o["n_contrib"]))
    if n_amb:
        assert err[amb].max() <= lim, (err[amb].max(), lim)
        assert np.abs(T - o["final_T"])[amb].max() <= lim
    assert n_amb <= max(AMB_MIN_ALLOWED, AMB_PER_PAIR_MAX * o["pairs"]), (n_amb, o["pairs"])
    print(f"[parity{(' ' + label) if label else ''}] pixels {amb.size}, ambiguous {n_amb} "
          f"({n_amb / amb.size:.2e} of pixels, {n_amb / max(1, o['pairs']):.2e} per evaluated pair), "
          f"of which differing {int(differ.sum())}, "
          f"max error there {err[amb].max(initial=0.0):.3g} (bound {lim:.3g})")
    return n_amb
