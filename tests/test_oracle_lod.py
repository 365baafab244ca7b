"""Pins of the oracle's block-wise LoD (Sec. 3.3.2, Eq. 7): MAD bounds against numpy's
median, selection against hand-derived cases, fusion by concatenation.  CPU only."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2404_01133_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def outward(lo, hi):
    lo_f, hi_f = np.float32(lo), np.float32(hi)
    if float(lo_f) > lo:
        lo_f = np.nextafter(lo_f, np.float32(-np.inf))
    if float(hi_f) < hi:
        hi_f = np.nextafter(hi_f, np.float32(np.inf))
    return lo_f, hi_f


def mad_bounds_numpy(v, n_mad):
    v = v.astype(np.float64)
    med = np.median(v)
    mad = np.median(np.abs(v - med))
    return outward(max(v.min(), med - n_mad * mad), min(v.max(), med + n_mad * mad))


@pytest.mark.parametrize("count", [1, 2, 7, 1000, 1001])
def test_mad_bounds_match_numpy_median(count, rng):
    nb = 3
    pts = [rng.normal(loc=(100.0 * b, 0.0, 10.0), scale=(5.0, 8.0, 3.0), size=(count, 3)) for b in range(nb)]
    for b in range(nb):
        if count > 10:
            pts[b][:5] += rng.normal(0, 500.0, size=(5, 3))   # floaters
    mo = np.zeros((nb * count, 4), np.float32)
    mo[:, :3] = np.concatenate(pts)
    sc = {"mean_opac": mo, "level_offset": (np.arange(nb) * count)[:, None].repeat(3, 1).astype(np.int64),
          "level_count": np.array([[count, count // 2, count // 4]] * nb, np.int64)}
    got = oracle.block_bounds(sc, 4.0)
    for b in range(nb):
        for ax in range(3):
            lo, hi = mad_bounds_numpy(mo[b * count:(b + 1) * count, ax], 4.0)
            assert got[b, ax] == lo and got[b, 3 + ax] == hi


def test_mad_bounds_ignore_floaters(rng):
    core = rng.normal(size=(5000, 3)) * 10.0
    floaters = rng.normal(size=(50, 3)) * 10.0 + 1e4
    mo = np.zeros((5050, 4), np.float32)
    mo[:, :3] = np.concatenate([core, floaters])
    sc = {"mean_opac": mo, "level_offset": np.zeros((1, 1), np.int64), "level_count": np.full((1, 1), 5050, np.int64)}
    bb = oracle.block_bounds(sc, 4.0)[0]
    assert (bb[3:] < 100.0).all() and (bb[:3] > -100.0).all()
    assert (bb[3:] > 20.0).all()


def test_lod_hand_cases():
    g = json.load(open(os.path.join(GOLDEN, "lod_hand_cases.json")))
    scene = {"level_count": np.full((2, 3), 10, np.int64), "block_cell": np.array(g["cell"], np.float32)}
    aabb = np.array(g["aabb"], np.float32)
    for case in g["cases"]:
        R = np.array(g[case["R"]], np.float64).reshape(3, 3)
        pos = np.array(case["pos"], np.float64)
        W, H = case["wh"]
        cam = synth.camera_from_rt(R, -R @ pos, case["f"], case["f"], (W - 1) / 2.0, (H - 1) / 2.0, W, H)
        lev = oracle.lod_select(scene, aabb, cam, dist=case["dist"])
        assert list(lev) == case["expect"], case["name"]


def test_paper_hyperparameters_are_the_defaults():
    g = json.load(open(os.path.join(GOLDEN, "paper_hyperparams.json")))
    assert g["n_mad"] == 4 and g["levels"] == 3
    assert g["distance_interval_matrixcity_m"] == [200, 400]


def test_empty_block_is_never_selected():
    scene = {"level_count": np.array([[0, 0, 0], [5, 2, 1]], np.int64),
             "block_cell": np.array([[0, 100, 0, 100], [100, 200, 0, 100]], np.float32)}
    aabb = np.array([[0, 0, 0, 100, 100, 10], [100, 0, 0, 200, 100, 10]], np.float32)
    R = np.diag([1.0, -1.0, -1.0])
    cam = synth.camera_from_rt(R, -R @ np.array([50.0, 50.0, 300.0]), 100, 100, 99.5, 99.5, 200, 200)
    assert list(oracle.lod_select(scene, aabb, cam)) == [-1, 1]


def test_concatenation_of_selected_segments():
    sc = synth.build_blocks(synth.city_scene(20000, 0.25, seed=1, sh_degree=0), grid=4)
    lev = np.array([0, -1, 1, 2] * 4, np.int8)
    idx = oracle.concat(sc, lev)
    exp = np.concatenate([np.arange(sc["level_offset"][b, lev[b]], sc["level_offset"][b, lev[b]] + sc["level_count"][b, lev[b]])
                          for b in range(16) if lev[b] >= 0])
    np.testing.assert_array_equal(idx, exp)
    assert (np.diff(idx) > 0).all()


def test_levels_are_nested_prefixes_ranked_by_opacity_volume():
    base = synth.city_scene(5000, 0.1, seed=2, sh_degree=0)
    sc = synth.build_blocks(base, grid=2)
    for b in range(4):
        off = sc["level_offset"][b]
        cnt = sc["level_count"][b]
        assert (off == off[0]).all() and cnt[0] >= cnt[1] >= cnt[2]
        assert cnt[1] == cnt[0] // 2 and cnt[2] == cnt[0] // 4
        seg = slice(off[0], off[0] + cnt[0])
        s = sc["scale"][seg].astype(np.float64)
        score = sc["mean_opac"][seg, 3].astype(np.float64) * s[:, 0] * s[:, 1] * s[:, 2]
        assert (np.diff(score) <= 0).all()


def test_pointwise_selection_by_hand():
    # one block of 8 Gaussians on the x axis, levels 8 / 4 / 2 (nested prefixes); camera at the origin
    mo = np.zeros((8, 4), np.float32)
    mo[:, 0] = [10, 250, 700, 150, 500, 900, 30, 650]
    mo[:, 3] = 0.5
    sc = {"mean_opac": mo, "level_offset": np.zeros((1, 3), np.int64), "level_count": np.array([[8, 4, 2]], np.int64)}
    cam = synth.camera_from_rt(np.eye(3), [0.0, 0.0, 0.0], 100, 100, 49.5, 49.5, 100, 100)
    # ranks 0..7 at distances 10, 250, 700, 150, 500, 900, 30, 650 -> levels 0,1,2,0,1,2,0,2
    # kept iff rank < count[level]: r0 (0<8), r1 (1<4), r2 (2<2 no), r3 (3<8), r4 (4<4 no),
    # r5 (5<2 no), r6 (6<8), r7 (7<2 no)
    assert list(oracle.pointwise_select(sc, cam, dist=(200.0, 600.0))) == [0, 1, 3, 6]
