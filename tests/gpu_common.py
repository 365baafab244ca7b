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
# An ambiguous pixel can differ by one entry at the 1/255 threshold or one blend at the
# 1e-4 transmittance stop: alpha * T * c <= 0.99 * 0.01 * c behind the stop, 1/255 at the skip.
AMB_ATOL = 0.03


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


def compare_image(gimg, gT, gnc, o):
    """Pixels within PIX_ATOL and n_contrib equal where the oracle saw no near-threshold
    decision; ambiguous pixels within AMB_ATOL.  Returns the number of ambiguous pixels."""
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
    if amb.any():
        assert err[amb].max() <= AMB_ATOL
    return int(amb.sum())
