"""GPU parity of the detail-level generation (Sec. 3.3.1): per-pixel hit counts accumulated by
the forward render, and the per-block significance ranking with nested level counts, against
the oracle through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
from paper_2404_01133_b300 import cgs, synth
from paper_2404_01133_b300 import torch_api as ta
from gpu_common import fp16_rounded, gpu_render

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2404_01133_b300 import build
    build.build()
    assert torch.cuda.is_available()


def gpu_hits(scene, cams, tile=16, batch=None, levels=None):
    g = gpu_render(scene, cams, tile=tile, batch=batch, levels=levels)
    hits = torch.zeros(g["ds"].n, dtype=torch.int32, device="cuda")
    img, T, nc = ta.render_forward_hits(g["ds"], g["frame"], g["cfg"], g["cams"], hits, levels=g["levels"])
    torch.cuda.synchronize()
    # the hit-counting forward renders exactly the same image
    assert torch.equal(img, g["image"]) and torch.equal(nc, g["n_contrib"])
    return hits.cpu().numpy().view(np.uint32).astype(np.int64), g


@pytest.mark.parametrize("tile,batch", [(16, 256), (16, 64), (8, 32)])
def test_hit_counts_match_oracle(tile, batch):
    sc = synth.single_block(synth.random_cube_scene(1500, seed=6, sh_degree=1, log_scale_mu=-2.4))
    cams = [synth.small_scene_camera(96, 80, f=80.0, dist=3.0), synth.small_scene_camera(96, 80, f=60.0, dist=3.5)]
    cfg = oracle.make_config(tile=tile)
    h, amb = oracle.hit_counts(sc, cams, cfg)
    gh, _ = gpu_hits(sc, cams, tile=tile, batch=batch)
    sure = amb == 0
    np.testing.assert_array_equal(gh[sure], h[sure])
    assert (np.abs(gh - h) <= amb).all()
    assert sure.mean() > 0.5 and h.sum() > 10000


def test_hit_counts_of_a_lod_selection():
    sc = synth.build_blocks(synth.city_scene(40_000, 0.01, seed=4, sh_degree=1), 4)
    cam = synth.pitched_camera((0.0, -90.0, 60.0), 0.0, np.radians(35.0), 200.0, 200.0, 128, 96)
    nb = sc["level_offset"].shape[0]
    levels = np.zeros((1, nb), np.int8)
    levels[0, ::2] = 1
    levels[0, 3] = -1
    idx = oracle.concat(sc, levels[0])
    h, amb = oracle.hit_counts(sc, [cam], idx=idx)
    gh, _ = gpu_hits(sc, [cam], levels=levels)
    np.testing.assert_array_equal(gh[amb == 0], h[amb == 0])
    assert (np.abs(gh - h) <= amb).all()
    outside = np.ones(len(h), bool)
    outside[idx] = False
    assert (gh[outside] == 0).all() and h.sum() > 1000


def grouped_scene(n, counts, seed, fp16=False, ties=False):
    rng = np.random.default_rng(seed)
    sc = synth.single_block(synth.random_cube_scene(n, seed=seed, sh_degree=0))
    if ties:
        sc["mean_opac"][:, 3] = rng.choice([0.25, 0.5, 1.0], size=n).astype(np.float32)
        sc["scale"][:, :3] = rng.choice([0.5, 1.0, 2.0], size=(n, 3)).astype(np.float32)
    if fp16:
        sc = fp16_rounded(sc)
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    sc["level_offset"] = off[:-1, None]
    sc["level_count"] = np.asarray(counts, np.int64)[:, None]
    return sc, off


@pytest.mark.parametrize("nb,fp16,use_hits,ties", [(64, False, False, False), (64, True, True, False),
                                                  (1, False, True, True), (1000, False, False, True),
                                                  (300, True, False, True)])
def test_generate_levels_matches_oracle(nb, fp16, use_hits, ties):
    rng = np.random.default_rng(nb)
    counts = rng.integers(0, 400, size=nb)
    counts[::7] = 0                                   # empty blocks
    n = int(counts.sum())
    sc, off = grouped_scene(n, counts, seed=nb, fp16=fp16, ties=ties)
    hits = rng.integers(0, 3000, size=n).astype(np.int64) if use_hits else None
    if use_hits:
        hits[::5] = 0
    rates = [1.0, 0.5, 0.34, 0.25]
    operm, olc = oracle.generate_levels(sc, rates, hits=hits)
    ds = ta.DeviceScene(sc, fp16=fp16)
    d_off = torch.as_tensor(off).cuda()
    d_hits = None if hits is None else torch.as_tensor(hits.astype(np.int32)).cuda()
    perm, lc = ta.generate_levels(ds, d_off, rates, hits=d_hits)
    np.testing.assert_array_equal(perm.cpu().numpy().astype(np.int64), operm)
    np.testing.assert_array_equal(lc.cpu().numpy(), olc)


def test_generate_levels_empty_and_single():
    sc, off = grouped_scene(1, [0, 1, 0], seed=1)
    ds = ta.DeviceScene(sc)
    perm, lc = ta.generate_levels(ds, torch.as_tensor(off).cuda(), [1.0, 0.5])
    assert perm.cpu().tolist() == [0]
    assert lc.cpu().tolist() == [[0, 0], [1, 0], [0, 0]]


def test_levels_pipeline_renders_like_the_oracle():
    """Partition, gather, count hits over aerial views, rank, gather again, and render the
    generated 3-level scene with the block LoD: every step against the oracle."""
    sc, box = synth.unbounded_city(80_000, seed=8, sh_degree=1, area_km2=0.04, bg_frac=0.02)
    grid = (4, 4, 1)
    nb = 16
    d_pos = torch.as_tensor(sc["mean_opac"]).cuda()
    block, off, perm, _ = ta.partition(d_pos, box[0], box[1], grid)
    o = oracle.partition_assign(sc["mean_opac"], box[0], box[1], grid)
    operm, ooff = oracle.partition_order(o["block"], nb)
    np.testing.assert_array_equal(perm.cpu().numpy(), operm)
    grouped = {k: ta.gather_rows(torch.as_tensor(np.ascontiguousarray(sc[k], np.float32)).cuda(), perm)
               for k in ("mean_opac", "scale", "quat", "sh")}
    gsc = {k: v.cpu().numpy() for k, v in grouped.items()}
    gsc.update({"sh_degree": sc["sh_degree"], "level_offset": ooff[:nb, None], "level_count": np.diff(ooff)[:, None],
                "block_cell": np.zeros((nb, 4), np.float32)})
    cams = [synth.pitched_camera((x, -120.0, 80.0), 0.0, np.radians(35.0), 250.0, 250.0, 160, 120)
            for x in (-40.0, 0.0, 40.0)]
    h, amb = oracle.hit_counts(gsc, cams)
    gh, _ = gpu_hits(gsc, cams, levels=np.zeros((len(cams), nb), np.int8))
    np.testing.assert_array_equal(gh[amb == 0], h[amb == 0])
    # rank with the oracle's hit counts on both sides (the ranking itself is bit-exact)
    rates = [1.0, 0.5, 0.25]
    lperm, lc = oracle.generate_levels(gsc, rates, hits=h)
    ds = ta.DeviceScene(gsc)
    dperm, dlc = ta.generate_levels(ds, torch.as_tensor(ooff).cuda(), rates,
                                    hits=torch.as_tensor(h.astype(np.int32)).cuda())
    np.testing.assert_array_equal(dperm.cpu().numpy(), lperm)
    np.testing.assert_array_equal(dlc.cpu().numpy(), lc)
    final = {k: ta.gather_rows(v, dperm).cpu().numpy() for k, v in grouped.items()}
    final.update({"sh_degree": sc["sh_degree"], "level_offset": np.repeat(ooff[:nb, None], 3, axis=1),
                  "level_count": lc, "block_cell": np.zeros((nb, 4), np.float32)})
    lv = np.array([[0, 1, 2, 1] * 4], np.int8)
    g = gpu_render(final, cams[1:2], levels=lv)
    idx = oracle.concat(final, lv[0])
    from gpu_common import compare_image
    compare_image(g["image"][0], g["final_T"][0], g["n_contrib"][0], oracle.render(final, cams[1], idx=idx))
