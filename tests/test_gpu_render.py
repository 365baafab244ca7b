"""GPU parity of the forward hot path against the CPU oracle, through the C ABI:
projection records, tile keys / values / ranges (bit-exact), pixels (FP32 tolerance),
LoD selection and MAD bounds (bit-exact), batched views, edge cases."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2404_01133_b300 import cgs, synth
from paper_2404_01133_b300 import torch_api as ta
from gpu_common import canonical_ranges, compare_image, frame_arrays, gpu_render

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2404_01133_b300 import build
    build.build()
    assert torch.cuda.is_available()


def check_against_oracle(scene, cam, g, tile, idx=None, view=0):
    cfg = oracle.make_config(tile=tile)
    o = oracle.render(scene, cam, cfg, idx=idx)
    pr, srt = o["proj"], o["sort"]
    n_sel = pr["depth"].shape[0]
    assert g["status"] == 0, cgs.cgs_status_string(g["status"])
    fr = g["frame"]
    vb = fr.buffer(cgs.BUF_VIEW_BASE, torch.int32, count=fr.n_views + 1).cpu().numpy().astype(np.int64)
    a = frame_arrays(g, n_sel=int(vb[-1]))
    j0, j1 = vb[view], vb[view + 1]
    assert j1 - j0 == n_sel
    if fr.n_views == 1:
        assert g["counts"][1] == int((pr["tiles_touched"] > 0).sum())
        assert g["counts"][2] == pr["n_entries"]
    gidx = a["scene_index"][j0:j1].astype(np.int64)
    exp_idx = np.arange(n_sel) if idx is None else np.asarray(idx)
    np.testing.assert_array_equal(gidx, exp_idx)
    np.testing.assert_array_equal(a["tiles_touched"][j0:j1], pr["tiles_touched"].astype(np.uint32))
    vis = pr["tiles_touched"] > 0
    rec = a["records"][j0:j1]
    # key path and values: bit-exact with the FP32 oracle
    np.testing.assert_array_equal(rec[vis, 0], pr["xy"][vis, 0])
    np.testing.assert_array_equal(rec[vis, 1], pr["xy"][vis, 1])
    np.testing.assert_array_equal(rec[vis, 2], pr["arrays"][0][vis, 3])
    dk = a["depth_keys"][j0:j1][vis]
    np.testing.assert_array_equal(dk & np.uint64(0xFFFFFFFF), pr["depth"][vis].view(np.uint32).astype(np.uint64))
    np.testing.assert_array_equal(dk >> np.uint64(32), np.full(int(vis.sum()), view, np.uint64))
    rc = a["rects"][j0:j1][vis].astype(np.int64)
    np.testing.assert_array_equal(rc[:, 0] & 0xFFFF, pr["rect"][vis, 0])
    np.testing.assert_array_equal(rc[:, 0] >> 16, pr["rect"][vis, 1])
    np.testing.assert_array_equal(rc[:, 1] & 0xFFFF, pr["rect"][vis, 2])
    np.testing.assert_array_equal(rc[:, 1] >> 16, pr["rect"][vis, 3])
    np.testing.assert_array_equal(rec[vis, 4:7], pr["conic"][vis])
    np.testing.assert_array_equal(rec[vis, 8:11], pr["rgb"][vis])
    # sorted (tile, depth, index) entries and ranges: bit-exact
    T = ((cam["width"] + tile - 1) // tile) * ((cam["height"] + tile - 1) // tile)
    keys = a["keys"].astype(np.int64)
    sel = (keys // T) == view
    np.testing.assert_array_equal(keys[sel] - view * T, (srt["keys"] >> np.uint64(32)).astype(np.int64))
    np.testing.assert_array_equal(a["vals"][sel].astype(np.int64) - j0, srt["vals"].astype(np.int64))
    r = a["ranges"].astype(np.int64)[view * T:(view + 1) * T]
    first = int(np.flatnonzero(sel)[0]) if sel.any() else 0
    np.testing.assert_array_equal(np.where(r[:, 1:] > r[:, :1], r - first, 0), srt["ranges"])
    namb = compare_image(g["image"][view], g["final_T"][view], g["n_contrib"][view], o)
    return o, namb


@pytest.mark.parametrize("tile,batch", [(16, 256), (16, 64), (16, 32), (8, 64), (8, 32)])
def test_small_scene_parity(tile, batch):
    sc, cams = synth.workload_small()
    g = gpu_render(sc, cams, tile=tile, batch=batch)
    o, namb = check_against_oracle(sc, cams[0], g, tile)
    assert namb < 0.01 * 128 * 128
    pairs_gpu = g["counts"][3]
    assert abs(pairs_gpu - o["pairs"]) <= int(o["n_visited"][o["ambiguous"].astype(bool)].sum()) + 0


def test_depth_tie_broken_by_index():
    sc, cams = synth.workload_small()
    o = oracle.project(sc, cams[0])
    d = o["depth"][o["tiles_touched"] > 0]
    assert len(np.unique(d)) < len(d), "the 2,000-Gaussian workload has an FP32 depth tie"
    g = gpu_render(sc, cams, tile=16)
    check_against_oracle(sc, cams[0], g, 16)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_ragged_image_and_sh_degrees(seed):
    deg = seed % 4
    sc = synth.single_block(synth.random_cube_scene(3000, seed=seed, sh_degree=deg, log_scale_mu=-2.5))
    cam = synth.small_scene_camera(100, 75, f=90.0, dist=3.5)
    for tile in (16, 8):
        g = gpu_render(sc, [cam], tile=tile)
        check_against_oracle(sc, cam, g, tile)


@pytest.mark.parametrize("tile", [16, 8])
def test_elongated_and_opaque_gaussians(tile):
    """Needle-like covariances (one tiny axis), opacities near 1 and below 1/255: the warp
    skip must never drop a pair the per-pixel test would blend."""
    r = np.random.default_rng(31)
    sc = synth.random_cube_scene(1500, seed=31, sh_degree=0, log_scale_mu=-2.5)
    sc["scale"][:500, 0] = np.float32(1e-4)          # flat / needle Gaussians
    sc["scale"][500:700, :2] = np.float32(2e-4)
    sc["mean_opac"][:300, 3] = r.uniform(0.95, 0.9999, size=300).astype(np.float32)
    sc["mean_opac"][1200:1300, 3] = r.uniform(0.0, 1.0 / 255.0, size=100).astype(np.float32)
    sc = synth.single_block(sc)
    cam = synth.small_scene_camera(120, 90, f=110.0, dist=3.2)
    g = gpu_render(sc, [cam], tile=tile)
    check_against_oracle(sc, cam, g, tile)


@pytest.mark.parametrize("n", [2049, 7001, 9000])
def test_long_tile_lists_use_the_merge_path(n):
    """Tiles with more entries than one shared-memory radix sort holds (2048) are sorted by
    chunks and merge rounds; keys, values and ranges stay bit-exact."""
    sc = synth.single_block(synth.random_cube_scene(n, seed=n, sh_degree=0, extent=0.25, log_scale_mu=-2.0))
    cam = synth.small_scene_camera(40, 36, f=60.0, dist=3.0)
    g = gpu_render(sc, [cam])
    o, _ = check_against_oracle(sc, cam, g, 16)
    lens = o["sort"]["ranges"][:, 1] - o["sort"]["ranges"][:, 0]
    assert lens.max() > 2048


@pytest.mark.parametrize("n", [1, 31, 32, 33, 64, 65, 128, 129, 255, 256, 257, 512, 513, 2048, 2049, 4096, 4097])
def test_tile_lengths_at_sort_path_bounds(n):
    """One 16 x 16 tile holding every Gaussian: lengths on both sides of the ranking sort (128
    keys), the short-tile bitonic sort (256), the long-tile kernel's register bitonic sort (512)
    and its shared-memory radix sort (2048, beyond which it merges chunks) stay bit-exact."""
    sc = synth.single_block(synth.random_cube_scene(n, seed=100 + n, sh_degree=0, extent=0.2, log_scale_mu=-2.5))
    cam = synth.small_scene_camera(16, 16, f=30.0, dist=3.0)
    g = gpu_render(sc, [cam])
    o, _ = check_against_oracle(sc, cam, g, 16)
    assert o["sort"]["ranges"][0, 1] - o["sort"]["ranges"][0, 0] == n


@pytest.mark.parametrize("n", [300, 600, 1500, 5000])
def test_long_tiles_with_equal_depths_keep_index_order(n):
    """Long tiles whose Gaussians share depths exactly (four planes facing the camera): the
    radix sort orders by depth bits, then puts each run of equal depth in index order, across
    the chunk merges too; bit-exact against the oracle's (depth, index) order."""
    sc = synth.random_cube_scene(n, seed=7 + n, sh_degree=0, extent=0.2, log_scale_mu=-2.5)
    sc["mean_opac"][:, 2] = np.random.default_rng(n).choice(np.float32([-0.1, 0.0, 0.05, 0.1]), size=n)
    sc = synth.single_block(sc)
    cam = synth.small_scene_camera(16, 16, f=30.0, dist=3.0)
    g = gpu_render(sc, [cam])
    o, _ = check_against_oracle(sc, cam, g, 16)
    assert len(np.unique(o["sort"]["keys"])) == 4   # one tile, four depths: long runs of ties


@pytest.mark.parametrize("n", [5, 40, 100, 128, 200])
def test_short_tiles_with_equal_depths_keep_index_order(n):
    """Tiles of up to 256 keys whose Gaussians share depths exactly (four planes facing the
    camera): the ranking path orders by depth bits first and puts keys of equal depth in index
    order, the register bitonic path compares whole keys; bit-exact against the oracle."""
    sc = synth.random_cube_scene(n, seed=11 + n, sh_degree=0, extent=0.2, log_scale_mu=-2.5)
    sc["mean_opac"][:, 2] = np.random.default_rng(n + 1).choice(np.float32([-0.1, 0.0, 0.05, 0.1]), size=n)
    sc = synth.single_block(sc)
    cam = synth.small_scene_camera(16, 16, f=30.0, dist=3.0)
    g = gpu_render(sc, [cam])
    o, _ = check_against_oracle(sc, cam, g, 16)
    keys = o["sort"]["keys"]   # (tile, depth bits) of every entry: one tile here
    assert len(keys) == n and len(np.unique(keys)) < n   # ties present


def test_all_culled_view_gives_background():
    sc, cams = synth.workload_small()
    cam = synth.camera_from_rt(np.diag([-1.0, 1.0, -1.0]), [0.0, 0.0, -10.0], 150, 150, 63.5, 63.5, 128, 128)
    g = gpu_render(sc, [cam], cfg_kw={"bg": (0.25, 0.5, 0.75)})
    assert g["status"] == 0 and g["counts"][1] == 0 and g["counts"][2] == 0
    img = g["image"][0].cpu().numpy()
    for ch, v in enumerate((0.25, 0.5, 0.75)):
        assert np.all(img[ch] == np.float32(v))
    assert torch.all(g["final_T"] == 1.0) and torch.all(g["n_contrib"] == 0)


def test_capacity_overflow_is_reported_not_faulted():
    sc, cams = synth.workload_small()
    g = gpu_render(sc, cams, k_cap=1000)
    assert g["status"] == cgs.CGS_ERR_CAPACITY
    assert g["counts"][2] > 1000
    g = gpu_render(sc, cams, n_cap=500, k_cap=100000)
    assert g["status"] == cgs.CGS_ERR_CAPACITY
    assert g["counts"][0] == 2000


def test_batched_views_equal_single_views():
    sc, _ = synth.workload_small()
    cams = [synth.look_at((x, 0.5, -4.0), (0, 0, 0), (0, -1, 0), 150, 150, 128, 128) for x in (-1.0, 0.0, 1.5)]
    gb = gpu_render(sc, cams)
    assert gb["status"] == 0
    for v, cam in enumerate(cams):
        gs = gpu_render(sc, [cam])
        assert torch.equal(gb["image"][v], gs["image"][0])
        assert torch.equal(gb["final_T"][v], gs["final_T"][0])
        assert torch.equal(gb["n_contrib"][v], gs["n_contrib"][0])
    # and each view of the batch matches the oracle
    check_against_oracle(sc, cams[2], gb, 16, view=2)


def lod_scene(n=60000, grid=4, seed=7):
    return synth.build_blocks(synth.city_scene(n, 0.4, seed, sh_degree=1), grid)


def test_block_bounds_bit_exact():
    sc = lod_scene()
    ds = ta.DeviceScene(sc)
    got = ds.compute_block_bounds(4.0).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.block_bounds(sc, 4.0))
    got2 = ds.compute_block_bounds(2.5).cpu().numpy()
    np.testing.assert_array_equal(got2, oracle.block_bounds(sc, 2.5))


def lod_cameras(side, n=12, seed=11):
    rng = np.random.default_rng(seed)
    cams = []
    for k in range(n):
        x, y = rng.uniform(-side / 2, side / 2, size=2)
        z = math.exp(rng.uniform(math.log(20.0), math.log(1500.0)))
        pitch = rng.uniform(0.3, math.pi / 2)
        cams.append(synth.pitched_camera((x, y, z), rng.uniform(0, 2 * math.pi), pitch, 300.0, 300.0, 320, 240))
    return cams


@pytest.mark.parametrize("dist", [(200.0, 600.0), (200.0, 400.0)])
def test_lod_selection_bit_exact(dist):
    sc = lod_scene()
    ds = ta.DeviceScene(sc)
    ds.compute_block_bounds(4.0)
    aabb = oracle.block_bounds(sc, 4.0)
    cams = lod_cameras(sc["side"])
    cfg = ta.make_config(lod_dist=dist)
    lv = torch.empty((len(cams), ds.n_blocks), dtype=torch.int8, device="cuda")
    cgs.cgs_lod_select(ds.struct(), cfg, ta.cameras_device(cams), len(cams), lv)
    got = lv.cpu().numpy()
    for v, cam in enumerate(cams):
        np.testing.assert_array_equal(got[v], oracle.lod_select(sc, aabb, cam, dist=dist))
    assert (got == -1).any() and (got >= 0).any()


def test_one_view_selection_matches_oracle():
    """One view of a four-block scene: the selected list the renderer builds (the scene index
    of every selected Gaussian, in segment order), its count and the view prefix equal the
    oracle's LoD selection and concatenation, for cameras that cull blocks, use every level and
    mix levels in one frame; one mixed frame is rendered in full."""
    sc = lod_scene(n=20000, grid=2)
    aabb = oracle.block_bounds(sc, 4.0)
    cams = lod_cameras(sc["side"])
    seen, mixed = set(), None
    for cam in cams:
        lev = np.asarray(oracle.lod_select(sc, aabb, cam)).ravel()
        idx = np.asarray(oracle.concat(sc, lev), np.int64)
        g = gpu_render(sc, [cam], n_mad=4.0)
        assert g["status"] == 0
        assert g["counts"][0] == len(idx)
        gidx = g["frame"].buffer(cgs.BUF_SCENE_INDEX, torch.int32, count=len(idx)).cpu().numpy()
        np.testing.assert_array_equal(gidx.astype(np.int64), idx)
        vb = g["frame"].buffer(cgs.BUF_VIEW_BASE, torch.int32, count=2).cpu().numpy()
        assert list(vb) == [0, len(idx)]
        seen.update(int(x) for x in lev)
        if mixed is None and len(set(int(x) for x in lev if x >= 0)) > 1:
            mixed = (cam, idx)
    assert seen == {-1, 0, 1, 2} and mixed is not None
    cam, idx = mixed
    check_against_oracle(sc, cam, gpu_render(sc, [cam], n_mad=4.0), 16, idx=idx)


def test_lod_render_matches_oracle_on_concatenated_selection():
    sc = lod_scene()
    aabb = oracle.block_bounds(sc, 4.0)
    cams = [synth.pitched_camera((30.0, -40.0, 120.0), 0.3, 0.6, 300.0, 300.0, 320, 240),
            synth.pitched_camera((-150.0, 100.0, 400.0), 2.0, 1.2, 300.0, 300.0, 320, 240)]
    g = gpu_render(sc, cams, n_mad=4.0)
    assert g["status"] == 0
    for v, cam in enumerate(cams):
        lev = oracle.lod_select(sc, aabb, cam)
        idx = oracle.concat(sc, lev)
        assert 0 < len(idx) < sc["mean_opac"].shape[0]
        gv = gpu_render(sc, [cam], n_mad=4.0)
        check_against_oracle(sc, cam, gv, 16, idx=idx)
        assert torch.equal(gv["image"][0], g["image"][v])


@pytest.mark.parametrize("dist", [(200.0, 600.0), (100.0, 250.0)])
def test_pointwise_lod_baseline_matches_oracle(dist):
    """The point-wise level baseline: per-Gaussian distance levels, no block culling."""
    sc = lod_scene()
    cam = synth.pitched_camera((30.0, -40.0, 120.0), 0.3, 0.6, 300.0, 300.0, 320, 240)
    g = gpu_render(sc, [cam], cfg_kw={"lod_mode": cgs.CGS_LOD_POINT, "lod_dist": dist})
    assert g["status"] == 0
    idx = oracle.pointwise_select(sc, cam, dist=dist)
    o = oracle.render(sc, cam, idx=idx)
    a = frame_arrays(g, n_sel=g["counts"][0])
    np.testing.assert_array_equal(a["keys"].astype(np.int64), (o["sort"]["keys"] >> np.uint64(32)).astype(np.int64))
    np.testing.assert_array_equal(a["scene_index"][a["vals"]].astype(np.int64), idx[o["sort"]["vals"]])
    np.testing.assert_array_equal(canonical_ranges(a["ranges"]), o["sort"]["ranges"])
    compare_image(g["image"][0], g["final_T"][0], g["n_contrib"][0], o)
    assert g["counts"][1] == int((o["proj"]["tiles_touched"] > 0).sum())


def test_explicit_levels_and_view_block_modes():
    sc = lod_scene()
    cam = synth.pitched_camera((0.0, 0.0, 300.0), 0.0, 1.0, 300.0, 300.0, 320, 240)
    nb = sc["level_offset"].shape[0]
    lev = np.array([(b % 4) - 1 for b in range(nb)], np.int8)  # -1, 0, 1, 2 repeating
    g = gpu_render(sc, [cam], levels=lev[None, :])
    check_against_oracle(sc, cam, g, 16, idx=oracle.concat(sc, lev))
    g = gpu_render(sc, [cam], view_block=[5])
    lev = np.full(nb, -1, np.int8)
    lev[5] = 0
    check_against_oracle(sc, cam, g, 16, idx=oracle.concat(sc, lev))
