"""GPU parity of the block-LoD workload at its full size, in the benchmark's launch
configuration: the 20M-Gaussian, 8 x 8-block, 3-level city (Sec. 3.3) rendered top-down at
1920x1080 from 50 to 2000 m with MAD block bounds (Eq. 7, n_MAD = 4), distance intervals
200 / 600 m, 16 x 16 tiles and batches of 128.  Block bounds and every view's selected list
are compared whole and bit-exact; two heights also compare every tile key, value and range,
and the pixels of a band of tile rows, against the oracle.  The 64-pose queue, batched as the
benchmark batches it, is checked view by view against one-view renders."""
import numpy as np
import pytest
import torch

import oracle
from paper_2404_01133_b300 import cgs, synth
from paper_2404_01133_b300 import torch_api as ta
from gpu_common import AMB_MIN_ALLOWED, AMB_PER_PAIR_MAX, PIX_ATOL, amb_atol, canonical_ranges

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def city():
    from paper_2404_01133_b300 import build
    build.build()
    sc, cams = synth.workload_city_lod()
    ds = ta.DeviceScene(sc)
    aabb = ds.compute_block_bounds(4.0).cpu().numpy()
    return sc, cams, ds, aabb


def render_view(ds, cam, exact=False):
    cfg = ta.make_config(tile=16, batch=128, lod_dist=(200.0, 600.0), exact=exact)
    sel, ent = ta.frame_counts(ds, [cam], 1920, 1080, cfg=cfg)
    fr = ta.Frame(1, 1920, 1080, 16, ds.n_blocks, int(sel[0] * 1.02) + 1024, int(ent[0] * 1.05) + 65536)
    img, T, nc = ta.render_forward(ds, fr, cfg, ta.cameras_device([cam]))
    torch.cuda.synchronize()
    st, counts = fr.status()
    assert st == 0, cgs.cgs_status_string(st)
    return fr, counts, img, T, nc


def test_full_size_block_bounds_20m(city):
    sc, _, _, aabb = city
    np.testing.assert_array_equal(aabb, oracle.block_bounds(sc, 4.0))


def test_full_size_selection_every_height_20m(city):
    """Each height's selected list (the concatenation of the chosen blocks' levels) equals the
    oracle's LoD choice on the oracle's bounds, index for index."""
    sc, cams, ds, aabb = city
    for cam in cams:
        fr, counts, *_ = render_view(ds, cam)
        idx = oracle.concat(sc, oracle.lod_select(sc, aabb, cam))
        assert counts[0] == len(idx)
        got = fr.buffer(cgs.BUF_SCENE_INDEX, torch.int32, count=int(counts[0])).cpu().numpy().view(np.uint32)
        np.testing.assert_array_equal(got.astype(np.int64), idx.astype(np.int64))


@pytest.mark.parametrize("height", [200.0, 2000.0])
def test_full_size_lod_frame_20m(city, height):
    """Tile keys, values and ranges of the whole frame bit-exact; the pixels of the central
    eighth of the tile rows within the forward tolerance, and, rendered by the compositing
    kernels' parity build (cgs_config.exact), equal to the oracle's on every pixel of the band,
    those the fast build exempts as ambiguous included."""
    sc, cams, ds, aabb = city
    cam = [c for c in cams if abs(float(c["campos"][2]) - height) < 1e-6][0]
    fr, counts, img, T, nc = render_view(ds, cam)
    idx = oracle.concat(sc, oracle.lod_select(sc, aabb, cam))
    cfg = oracle.make_config(tile=16)
    pr = oracle.project(sc, cam, cfg, idx=idx)
    srt = oracle.bin_and_sort(pr, cam, cfg)
    k = int(counts[2])
    assert k == pr["n_entries"] and counts[1] == int((pr["tiles_touched"] > 0).sum())
    keys = fr.buffer(cgs.BUF_TILE_KEYS, torch.int32, count=k).cpu().numpy().view(np.uint32)
    vals = fr.buffer(cgs.BUF_TILE_VALS, torch.int32, count=k).cpu().numpy().view(np.uint32)
    ranges = fr.buffer(cgs.BUF_RANGES, torch.int32, (2,), count=fr_tiles(fr)).cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(keys.astype(np.int64), (srt["keys"] >> np.uint64(32)).astype(np.int64))
    np.testing.assert_array_equal(vals.astype(np.int64), srt["vals"].astype(np.int64))
    np.testing.assert_array_equal(canonical_ranges(ranges), srt["ranges"])
    # a band of tile rows through the middle of the image
    tx, ty = (1920 + 15) // 16, (1080 + 15) // 16
    rows = ty // 8
    r0 = (ty - rows) // 2
    tm = np.zeros((ty, tx), np.uint8)
    tm[r0:r0 + rows] = 1
    o = oracle.composite(pr, srt, cam, cfg, tile_mask=tm.reshape(-1))
    y0, y1 = 16 * r0, min(1080, 16 * (r0 + rows))
    amb = o["ambiguous"][y0:y1].astype(bool)
    gi = img[0, :, y0:y1].cpu().numpy()
    err = np.abs(gi - o["image"][:, y0:y1]).max(axis=0)
    assert err[~amb].max(initial=0.0) <= PIX_ATOL
    lim = amb_atol(pr["rgb"][pr["tiles_touched"] > 0])
    assert err[amb].max(initial=0.0) <= lim
    assert np.abs(T[0, y0:y1].cpu().numpy() - o["final_T"][y0:y1])[~amb].max(initial=0.0) <= PIX_ATOL
    ncb = nc[0, y0:y1].cpu().numpy()
    bad = (ncb != o["n_contrib"][y0:y1]) & ~amb
    assert not bad.any(), np.argwhere(bad)[:5]
    n_amb = int(amb.sum())
    assert n_amb <= max(AMB_MIN_ALLOWED, AMB_PER_PAIR_MAX * o["pairs"]), (n_amb, o["pairs"])
    differ = amb & ((err > PIX_ATOL) | (ncb != o["n_contrib"][y0:y1]))
    print(f"[parity 20M LoD frame at {height:g} m, central band] pixels {amb.size}, ambiguous {n_amb} "
          f"({n_amb / amb.size:.2e} of pixels, {n_amb / max(1, o['pairs']):.2e} per evaluated pair), "
          f"of which differing {int(differ.sum())}, "
          f"max error there {err[amb].max(initial=0.0):.3g} (bound {lim:.3g})")
    # the parity build: no pixel exempt
    _, _, img_x, T_x, nc_x = render_view(ds, cam, exact=True)
    gx, tx_ = img_x[0, :, y0:y1].cpu().numpy(), T_x[0, y0:y1].cpu().numpy()
    np.testing.assert_array_equal(nc_x[0, y0:y1].cpu().numpy(), o["n_contrib"][y0:y1])
    oi = o["image"][:, y0:y1].astype(np.float32)
    assert np.abs(gx - oi).max() <= PIX_ATOL and np.abs(tx_ - o["final_T"][y0:y1]).max() <= PIX_ATOL
    # only a falloff whose two FP64 exponentials round to different FP32 values can differ
    n_diff = int(((gx != oi).any(axis=0) | (tx_ != o["final_T"][y0:y1])).sum())
    assert n_diff <= 8, n_diff
    print(f"[exact 20M LoD frame at {height:g} m, central band] n_contrib equal on all {amb.size} pixels, "
          f"{n_diff} not bit-identical")


def fr_tiles(fr):
    return fr.n_views * ((fr.width + fr.tile - 1) // fr.tile) * ((fr.height + fr.tile - 1) // fr.tile)


def test_full_size_pose_queue_batched_equals_single_views(city):
    """The 64-pose queue over the 20M city rendered as batched frames (views grouped by
    capacity, as the benchmark does): every sampled view equals its own one-view render bit for
    bit (image, T, n_contrib), and the batched selections add up to the per-view ones."""
    sc, _, ds, _ = city
    cams = synth.lod_pose_queue(sc["side"])
    cfg = ta.make_config(tile=16, batch=128, lod_dist=(200.0, 600.0))
    sel, ent = ta.frame_counts(ds, cams, 1920, 1080, cfg=cfg)
    groups = ta.waves(sel, ent, n_cap_max=200_000_000, k_cap_max=(1 << 30) - 1)
    sample = {0, 17, 40, 63}
    for views, n_cap, k_cap in groups:
        fr = ta.Frame(len(views), 1920, 1080, 16, ds.n_blocks, n_cap, min((1 << 30) - 1, k_cap))
        img, T, nc = ta.render_forward(ds, fr, cfg, ta.cameras_device([cams[v] for v in views]))
        torch.cuda.synchronize()
        st, counts = fr.status()
        assert st == 0, cgs.cgs_status_string(st)
        assert counts[0] == sum(sel[v] for v in views) and counts[2] == sum(ent[v] for v in views)
        for i, v in enumerate(views):
            if v not in sample:
                continue
            _, c1, img1, T1, nc1 = render_view(ds, cams[v])
            assert c1[0] == sel[v]
            assert torch.equal(img[i], img1[0]) and torch.equal(T[i], T1[0]) and torch.equal(nc[i], nc1[0]), v
        del fr, img, T, nc
