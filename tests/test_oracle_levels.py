"""Pins of the detail-level oracle (Sec. 3.3.1: nested levels from a significance ranking,
optionally weighted by per-pixel hit counts): hand-ranked blocks, a library stable sort, and
hit counts against a compositing-free count of each Gaussian's footprint."""
import numpy as np

import oracle
from paper_2404_01133_b300 import synth


def block_scene(opac, scale, counts):
    n = len(opac)
    mo = np.zeros((n, 4), np.float32)
    mo[:, 3] = opac
    sc = np.zeros((n, 4), np.float32)
    sc[:, :3] = scale
    off = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int64)
    return {"mean_opac": mo, "scale": sc, "level_offset": off[:, None], "level_count": np.asarray(counts, np.int64)[:, None]}


def test_levels_by_hand():
    # block 0: four unit-volume Gaussians, opacities 0.2, 0.5, 0.5, 0.1 -> ranks 1, 2 (tie to the
    # lower index), 0, 3; block 1: volumes 8, 1, 27 at opacity 0.5 -> 6, 4, 5; block 2 empty.
    opac = [0.2, 0.5, 0.5, 0.1, 0.5, 0.5, 0.5]
    scale = [[1, 1, 1]] * 4 + [[2, 2, 2], [1, 1, 1], [3, 3, 3]]
    sc = block_scene(opac, scale, [4, 3, 0])
    perm, lc = oracle.generate_levels(sc, [1.0, 0.5, 0.25])
    np.testing.assert_array_equal(perm, [1, 2, 0, 3, 6, 4, 5])
    np.testing.assert_array_equal(lc, [[4, 2, 1], [3, 1, 0], [0, 0, 0]])   # floor(K rate)
    # the paper's MatrixCity rates 50 / 34 / 25 %: floor(7 * 0.34) = 2
    sc7 = block_scene([0.5] * 7, [[1, 1, 1]] * 7, [7])
    np.testing.assert_array_equal(oracle.generate_levels(sc7, [0.5, 0.34, 0.25])[1], [[3, 2, 1]])


def test_hit_weighting_and_nan_by_hand():
    opac = [0.2, 0.5, 0.5, 0.1]
    sc = block_scene(opac, [[1, 1, 1]] * 4, [4])
    # scores h * o = 2.0, 0.5, 0.0, 10.0 -> 3, 0, 1, 2
    perm, _ = oracle.generate_levels(sc, [1.0], hits=np.array([10, 1, 0, 100]))
    np.testing.assert_array_equal(perm, [3, 0, 1, 2])
    sc["scale"][0, 1] = np.nan  # a NaN score ranks last, after the zero score
    perm, _ = oracle.generate_levels(sc, [1.0], hits=np.array([10, 1, 0, 100]))
    np.testing.assert_array_equal(perm, [3, 1, 2, 0])


def test_levels_are_the_stable_sort_within_blocks():
    rng = np.random.default_rng(0)
    counts = rng.integers(0, 3000, size=37)
    n = int(counts.sum())
    opac = rng.choice([0.25, 0.5, 0.75, 1.0], size=n).astype(np.float32)   # many exact ties
    scale = rng.choice([0.5, 1.0, 2.0], size=(n, 3)).astype(np.float32)
    sc = block_scene(opac, scale, counts)
    hits = rng.integers(0, 50, size=n)
    for h in (None, hits):
        perm, lc = oracle.generate_levels(sc, [1.0, 0.5, 0.25], hits=h)
        s = (scale[:, 0] * scale[:, 1]) * scale[:, 2] * opac
        if h is not None:
            s = h.astype(np.float32) * s
        off = np.concatenate([[0], np.cumsum(counts)])
        for b in range(len(counts)):
            rows = np.arange(off[b], off[b + 1])
            np.testing.assert_array_equal(perm[rows], rows[np.argsort(-s[rows], kind="stable")])
        np.testing.assert_array_equal(lc, np.floor(counts[:, None] * np.array([1.0, 0.5, 0.25])).astype(np.int64))


def test_hit_counts_equal_footprint_counts_without_occlusion():
    # sparse, translucent Gaussians: no pixel's transmittance comes near the 1e-4 stop, and
    # every opacity is below 1/(255 e^-4.5) so the 3-sigma tile coverage holds every pixel with
    # alpha >= 1/255.  A Gaussian's hit count is then the number of pixel centres where
    # o exp(power) >= 1/255, counted directly from its 2D mean and conic.
    sc = synth.single_block(synth.random_cube_scene(40, seed=2, sh_degree=0, log_scale_mu=-2.0))
    sc["mean_opac"][:, 3] = np.linspace(0.05, 0.3, 40, dtype=np.float32)
    cam = synth.small_scene_camera(96, 80, f=80.0, dist=3.0)
    hits, amb = oracle.hit_counts(sc, [cam])
    pr = oracle.project(sc, cam)
    o = oracle.render(sc, cam)
    assert o["final_T"].min() > 1e-3
    jj, ii = np.mgrid[0:80, 0:96]
    for g in range(40):
        if pr["tiles_touched"][g] == 0:
            assert hits[g] == 0
            continue
        dx = pr["xy"][g, 0].astype(np.float64) - ii
        dy = pr["xy"][g, 1].astype(np.float64) - jj
        a, b, c = pr["conic"][g].astype(np.float64)
        power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
        al = sc["mean_opac"][g, 3] * np.exp(power)
        want = int(((power <= 0) & (al >= 1 / 255)).sum())
        near = int((np.abs(al - 1 / 255) < 1e-6).sum())
        assert abs(int(hits[g]) - want) <= near, (g, hits[g], want)
    assert hits.sum() > 1000


def test_hit_counts_of_two_views_add():
    sc = synth.single_block(synth.random_cube_scene(300, seed=3, sh_degree=0, log_scale_mu=-2.4))
    c1 = synth.small_scene_camera(64, 64, f=70.0, dist=3.0)
    c2 = synth.small_scene_camera(64, 48, f=60.0, dist=3.5)
    h1, _ = oracle.hit_counts(sc, [c1])
    h2, _ = oracle.hit_counts(sc, [c2])
    h12, _ = oracle.hit_counts(sc, [c1, c2])
    np.testing.assert_array_equal(h12, h1 + h2)
