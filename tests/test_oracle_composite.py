"""Pins of the oracle's binning, sorting and compositing (Eq. 1, Sec. 3.1) against closed
forms, brute force and library sorts.  CPU only."""
import math

import numpy as np
import pytest

import oracle
from paper_2404_01133_b300 import synth
from test_oracle_projection import make_scene


def test_single_isotropic_gaussian_closed_form():
    W = H = 64
    cam = synth.small_scene_camera(W, H, f=150.0, dist=4.0)
    s, o = 0.04, 0.8
    c = np.array([0.9, 0.4, 0.1])
    f0 = (c - 0.5) * 2 * math.sqrt(math.pi)
    sc = make_scene([[0, 0, 0]], [[s, s, s]], [[1, 0, 0, 0]], [o], sh=f0.reshape(1, 1, 3))
    out = oracle.render(sc, cam, real="f64")
    sig2 = (150.0 * s / 4.0) ** 2 + 0.3
    jj, ii = np.mgrid[0:H, 0:W].astype(np.float64)
    r2 = (ii - cam["cx"]) ** 2 + (jj - cam["cy"]) ** 2
    alpha = np.minimum(0.99, o * np.exp(-0.5 * r2 / sig2))
    alpha[alpha < 1.0 / 255.0] = 0.0
    # pixels outside the binned rect are never evaluated; the rect covers 3 sigma, where alpha < 1/255
    for ch in range(3):
        np.testing.assert_allclose(out["image"][ch], c[ch] * alpha, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(out["final_T"], 1.0 - alpha, rtol=1e-12, atol=1e-14)
    assert out["n_contrib"].max() == 1


def test_opaque_stack_stops_on_transmittance():
    W = H = 33
    cam = synth.small_scene_camera(W, H, f=100.0, dist=4.0)
    cols = np.array([[0.9, 0.2, 0.3], [0.1, 0.8, 0.5], [0.6, 0.6, 0.9]])
    f0 = ((cols - 0.5) * 2 * math.sqrt(math.pi)).reshape(3, 1, 3)
    sc = make_scene([[0, 0, 0.0], [0, 0, 0.5], [0, 0, 1.0]], [[0.2] * 3] * 3, [[1, 0, 0, 0]] * 3, [1.0] * 3, sh=f0)
    out = oracle.render(sc, cam, real="f32")
    a = np.float32(0.99)
    T1 = np.float32(1.0) * (np.float32(1.0) - a)
    T2 = T1 * (np.float32(1.0) - a)
    rgb = oracle.project(sc, cam, real="f32")["rgb"]
    expect = rgb[0] * (a * np.float32(1.0))
    n_expect = 1
    if not T2 < np.float32(1e-4):
        expect = expect + rgb[1] * (a * T1)
        n_expect = 2
    centre = out["image"][:, 16, 16]
    np.testing.assert_array_equal(centre, expect.astype(np.float32))
    assert out["n_contrib"][16, 16] == n_expect
    # the third Gaussian can never contribute at the centre: T would be at most 1e-6
    assert out["final_T"][16, 16] >= np.float32(1e-4)


def test_input_order_invariance(rng):
    sc, cams = synth.workload_small()
    a = oracle.render(sc, cams[0], real="f32")
    perm = rng.permutation(sc["mean_opac"].shape[0])
    # Equal depths are ordered by index; keep every tie group in its original relative order
    depth = a["proj"]["depth"]
    for d in np.unique(depth[np.unique(depth, return_counts=True)[1][np.searchsorted(np.unique(depth), depth)] > 1]):
        slots = np.flatnonzero(depth[perm] == d)
        perm[slots] = np.sort(perm[slots])
    sp = dict(sc)
    sp["mean_opac"], sp["scale"], sp["quat"] = sc["mean_opac"][perm], sc["scale"][perm], sc["quat"][perm]
    sp["sh"] = np.ascontiguousarray(sc["sh"][perm])
    b = oracle.render(sp, cams[0], real="f32")
    np.testing.assert_array_equal(a["image"], b["image"])
    np.testing.assert_array_equal(a["final_T"], b["final_T"])
    np.testing.assert_array_equal(a["n_contrib"], b["n_contrib"])


@pytest.mark.parametrize("tile,real", [(16, "f32"), (8, "f32"), (16, "f64")])
def test_truncation_invariant_binned_equals_brute_force(tile, real):
    # Outside its binned tiles a Gaussian's Mahalanobis distance exceeds 3, so with every
    # opacity below 1/(255 e^-4.5) ~ 0.3536 binning never drops a contributing pair.
    for seed in range(4):
        r = np.random.default_rng(seed)
        n = 60
        sc = synth.random_cube_scene(n, seed=seed, sh_degree=1, log_scale_mu=-2.0)
        sc["mean_opac"][:, 3] = r.uniform(0.05, 0.3, size=n).astype(np.float32)
        cam = synth.small_scene_camera(40, 36, f=60.0, dist=3.0)
        cfg = oracle.make_config(tile=tile)
        out = oracle.render(sc, cam, cfg, real=real)
        img, T = oracle.composite_brute(out["proj"], cam, cfg, real=real)
        np.testing.assert_array_equal(out["image"], img)
        np.testing.assert_array_equal(out["final_T"], T)


@pytest.mark.parametrize("tile", [16, 8])
def test_keys_sort_ranges_brute_force(tile):
    sc, cams = synth.workload_small()
    cam = cams[0]
    cfg = oracle.make_config(tile=tile)
    pr = oracle.project(sc, cam, cfg)
    srt = oracle.bin_and_sort(pr, cam, cfg)
    W, H = cam["width"], cam["height"]
    tx_n = (W + tile - 1) // tile
    ty_n = (H + tile - 1) // tile
    pairs = []
    for i in np.flatnonzero(pr["tiles_touched"] > 0):
        u, v, r = float(pr["xy"][i, 0]), float(pr["xy"][i, 1]), int(pr["radius"][i])
        xs = sorted({x // tile for x in range(W) if abs(x - u) <= r})
        ys = sorted({y // tile for y in range(H) if abs(y - v) <= r})
        for ty in ys:
            for tx in xs:
                pairs.append((ty * tx_n + tx, i))
    pairs = np.array(pairs, dtype=np.int64)
    dbits = pr["depth"].view(np.uint32).astype(np.int64)
    order = np.lexsort((pairs[:, 1], dbits[pairs[:, 1]], pairs[:, 0]))
    exp_tile = pairs[order, 0]
    exp_idx = pairs[order, 1]
    np.testing.assert_array_equal(srt["keys"] >> np.uint64(32), exp_tile.astype(np.uint64))
    np.testing.assert_array_equal(srt["keys"] & np.uint64(0xFFFFFFFF), dbits[exp_idx].astype(np.uint64))
    np.testing.assert_array_equal(srt["vals"], exp_idx.astype(np.uint32))
    ranges = np.zeros((tx_n * ty_n, 2), np.int64)
    for k, t in enumerate(exp_tile):
        if k == 0 or exp_tile[k - 1] != t:
            ranges[t, 0] = k
        ranges[t, 1] = k + 1
    np.testing.assert_array_equal(srt["ranges"], ranges)


def test_evaluated_pair_count_and_stop_position():
    sc, cams = synth.workload_small()
    out = oracle.render(sc, cams[0], real="f32")
    lens = out["sort"]["ranges"][:, 1] - out["sort"]["ranges"][:, 0]
    tile_of = (np.arange(128)[:, None] // 16) * 8 + (np.arange(128)[None, :] // 16)
    assert (out["n_visited"] <= lens[tile_of]).all()
    assert (out["n_contrib"] <= out["n_visited"]).all()
    assert out["pairs"] == int(out["n_visited"].sum())
    # the stop rule leaves the entry that would cross 1e-4 unblended, so T never drops below it
    assert (out["final_T"] >= np.float32(1e-4)).all()
    # a pixel that visited fewer entries than its list holds must have stopped on transmittance
    short = out["n_visited"] < lens[tile_of]
    assert short.sum() > 0 and (out["final_T"][short] < np.float32(0.05)).all()


def test_l1_loss_and_gradient(rng):
    a = rng.uniform(size=(3, 7, 5)).astype(np.float32)
    b = rng.uniform(size=(3, 7, 5)).astype(np.float32)
    b[0, 0, 0] = a[0, 0, 0]
    loss, g = oracle.l1(a, b)
    assert abs(loss - np.mean(np.abs(a - b).astype(np.float64))) < 1e-12
    np.testing.assert_array_equal(g, np.sign(a - b) * (np.float32(1) / np.float32(a.size)))
