"""GPU tests of the boundary calls around the hot path, through the C ABI: the library's scene
upload (Sec. 3.1 attributes with Sec. 3.3.2's per-block levels and Eq. 7 bounds) renders exactly
as a scene uploaded by torch; the pose-to-block decision (Eqs. 3-5) equals its definition; the
autotuner times every (tile, batch) candidate on the real step, returns the fastest eligible one,
skips candidates the frame cannot hold, and reads and writes its cache."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2404_01133_b300 import cgs, synth
from paper_2404_01133_b300 import torch_api as ta

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2404_01133_b300 import build
    build.build()
    assert torch.cuda.is_available()


def _lod_scene():
    sc = synth.build_blocks(synth.city_scene(120_000, 0.06, seed=31, sh_degree=3), 4)
    cams = [synth.pitched_camera((x, y, z), 0.3, np.radians(55.0), 400.0, 400.0, 320, 200)
            for x, y, z in ((0.0, -60.0, 90.0), (40.0, 30.0, 160.0))]
    return sc, cams


@pytest.mark.parametrize("fp16", [False, True])
def test_library_upload_renders_as_the_torch_upload(fp16):
    sc, cams = _lod_scene()
    ds = ta.DeviceScene(sc, fp16=fp16)
    ds.compute_block_bounds(4.0)
    up = ta.UploadedScene(sc, n_mad=4.0, fp16=fp16)
    # Eq. 7 bounds written by the upload equal the oracle's
    np.testing.assert_array_equal(up.block_aabb.cpu().numpy(), oracle.block_bounds(sc, 4.0))
    torch.testing.assert_close(up.mean_opac, ds.mean_opac, rtol=0, atol=0)
    torch.testing.assert_close(up.sh, ds.sh, rtol=0, atol=0)
    cfg = ta.make_config(tile=16, batch=128, lod_dist=(60.0, 150.0))
    outs = []
    for scene in (ds, up):
        fr = ta.Frame(len(cams), 320, 200, 16, scene.n_blocks, scene.n * len(cams), 40 * scene.n)
        img, T, nc = ta.render_forward(scene, fr, cfg, ta.cameras_device(cams))
        torch.cuda.synchronize()
        st, counts = fr.status()
        assert st == 0 and counts[1] > 1000
        outs.append((img, T, nc, counts[:3]))
    (i0, T0, n0, c0), (i1, T1, n1, c1) = outs
    assert c0 == c1
    assert torch.equal(i0, i1) and torch.equal(T0, T1) and torch.equal(n0, n1)


def test_pose_assign_decision_equals_its_definition():
    rng = np.random.default_rng(5)
    P, nb, eps = 37, 19, 0.05
    s = rng.uniform(0.8, 1.0, size=(P, nb)).astype(np.float32)
    s[0, :4] = np.float32(1.0) - np.float32(eps)                  # exactly at the threshold: not above it
    pb = rng.integers(-1, nb, size=P).astype(np.int32)
    d_s, d_pb = torch.as_tensor(s).cuda(), torch.as_tensor(pb).cuda()
    b1, b2, b = (torch.empty((P, nb), dtype=torch.uint8, device="cuda") for _ in range(3))
    cgs.cgs_pose_assign(d_s, d_pb, P, nb, eps, b1, b2, b)
    want1 = (np.float32(1.0) - s) > np.float32(eps)
    want2 = pb[:, None] == np.arange(nb)[None, :]
    np.testing.assert_array_equal(b1.cpu().numpy().astype(bool), want1)
    np.testing.assert_array_equal(b2.cpu().numpy().astype(bool), want2)
    np.testing.assert_array_equal(b.cpu().numpy().astype(bool), want1 | want2)
    assert want1.any() and not want1.all() and (pb < 0).any()
    # one output only
    only = torch.full((P, nb), 7, dtype=torch.uint8, device="cuda")
    cgs.cgs_pose_assign(d_s, d_pb, P, nb, eps, None, None, only)
    np.testing.assert_array_equal(only.cpu().numpy().astype(bool), want1 | want2)


def test_autotune_times_every_candidate_and_caches(tmp_path):
    sc, cams = synth.workload_small()
    ds = ta.DeviceScene(sc)
    d_cams = ta.cameras_device(cams)
    W, H = cams[0]["width"], cams[0]["height"]
    cfg, ms = ta.autotune_library(ds, d_cams, W, H, ds.n, 64 * ds.n, reps=3)
    assert set(ms) == set(cgs.TUNE_ORDER)
    assert all(v > 0 for v in ms.values())                          # all fit this frame
    assert (cfg.tile, cfg.batch) == min(ms, key=ms.get)
    # the chosen configuration renders as the oracle at its tile size (the batch depth never
    # changes results; the tile size does, through the 3-sigma truncation of each tile list)
    o = oracle.render(sc, cams[0], oracle.make_config(tile=cfg.tile))
    fr = ta.Frame(1, W, H, cfg.tile, 1, ds.n, 64 * ds.n)
    img, T, nc = ta.render_forward(ds, fr, cfg, d_cams)
    torch.cuda.synchronize()
    assert fr.status()[0] == 0
    assert np.abs(img[0].cpu().numpy() - o["image"]).max(axis=0)[~o["ambiguous"].astype(bool)].max() <= 1e-4
    # cache: written, then read back without timing (ms left at -1)
    path = str(tmp_path / "tune.txt")
    cfg1, _ = ta.autotune_library(ds, d_cams, W, H, ds.n, 64 * ds.n, reps=2, cache_path=path, cache_key="small 2k")
    assert os.path.exists(path) and "small_2k" in open(path).read()
    cfg2, ms2 = ta.autotune_library(ds, d_cams, W, H, ds.n, 64 * ds.n, reps=2, cache_path=path,
                                    cache_key="small 2k")
    assert (cfg2.tile, cfg2.batch) == (cfg1.tile, cfg1.batch)
    assert all(v == -1 for v in ms2.values())


def test_autotune_skips_candidates_the_frame_cannot_hold():
    """Entry capacity between the 16 x 16 and the 8 x 8 tile counts: the 8 x 8 candidates
    overflow (device status CGS_ERR_CAPACITY) and are not eligible."""
    sc, cams = synth.workload_small()
    ds = ta.DeviceScene(sc)
    d_cams = ta.cameras_device(cams)
    W, H = cams[0]["width"], cams[0]["height"]
    pr = oracle.project(sc, cams[0])
    k16 = pr["n_entries"]
    k8 = oracle.project(sc, cams[0], oracle.make_config(tile=8))["n_entries"]
    assert k8 > k16 + 100
    cfg, ms = ta.autotune_library(ds, d_cams, W, H, ds.n, k16 + 50, reps=2, backward=False)
    for (t, b), v in ms.items():
        assert (v > 0) == (t == 16), (t, b, v)
    assert cfg.tile == 16
