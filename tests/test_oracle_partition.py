"""Pins of the block-partition oracle (Sec. 3.2.2: normalisation, Eq. 2 contraction, the
uniform grid over the contracted cube; Eq. 4: the block of a camera pose) against closed
forms, hand-computed cases, FP64 restatements away from cell bounds and a library stable
sort."""
import numpy as np
import pytest

import oracle
from paper_2404_01133_b300 import synth

BOX = (np.zeros(3, np.float32), np.full(3, 2.0, np.float32))  # foreground [0, 2]^3: h = p - 1


def test_normalisation_maps_box_corners_and_centre():
    lo = np.array([-750.0, -750.0, -10.0], np.float32)
    hi = np.array([750.0, 750.0, 100.0], np.float32)
    pts = np.stack([lo, hi, (lo + hi) / 2, np.array([lo[0], hi[1], 45.0], np.float32)])
    c = oracle.contract(pts, lo, hi)
    np.testing.assert_array_equal(c[0], [-1, -1, -1])
    np.testing.assert_array_equal(c[1], [1, 1, 1])
    np.testing.assert_array_equal(c[2], [0, 0, 0])
    np.testing.assert_array_equal(c[3], [-1, 1, 0])


@pytest.mark.parametrize("p,want", [
    # h = p - 1 with the [0, 2] box; values chosen so every step is exact in binary
    ((3.0, 1.0, 1.0), (1.5, 0.0, 0.0)),             # ||h|| = 2: (2 - 1/2) * (1, 0, 0)
    ((5.0, 2.0, 1.0), (1.75, 0.4375, 0.0)),         # ||h|| = 4: 1.75 * (1, 1/4, 0)
    ((-15.0, 1.5, 2.0), (-1.9375, 0.060546875, 0.12109375)),  # ||h|| = 16: (31/16) (-1, 1/32, 1/16)
    ((1.0, 1.0, -7.0), (0.0, 0.0, -1.875)),         # ||h|| = 8 along -z
    ((1.5, 0.25, 2.0), (0.5, -0.75, 1.0)),          # inside: the identity (Eq. 2, first case)
])
def test_contraction_closed_forms(p, want):
    c = oracle.contract(np.array([p], np.float32), *BOX)[0]
    np.testing.assert_array_equal(c, np.array(want, np.float32))


def test_contraction_properties_fp64():
    rng = np.random.default_rng(0)
    h = rng.normal(size=(20000, 3)) * np.exp(rng.uniform(-3, 8, size=(20000, 1)))
    p = (h + 1.0).astype(np.float32)
    hh = p.astype(np.float64) - 1.0
    c = oracle.contract(p, *BOX).astype(np.float64)
    m = np.abs(hh).max(axis=1)
    inside = m <= 1.0
    # identity inside the foreground box
    np.testing.assert_allclose(c[inside], hh[inside], rtol=0, atol=1e-6)
    # outside: the infinity norm becomes 2 - 1/m, the direction is kept, and the result stays
    # inside the open cube (-2, 2)
    out = ~inside
    cm = np.abs(c[out]).max(axis=1)
    np.testing.assert_allclose(cm, 2.0 - 1.0 / m[out], rtol=3e-7)
    np.testing.assert_allclose(c[out], (2.0 - 1.0 / m[out])[:, None] * hh[out] / m[out][:, None], rtol=1e-6,
                               atol=1e-6)
    assert (np.abs(c) < 2.0).all()
    # continuity at the box boundary
    e = np.array([[2.0 + 2 ** -20, 1.0, 1.0], [2.0, 1.0, 1.0]], np.float32)
    ce = oracle.contract(e, *BOX)
    assert abs(float(ce[0, 0]) - float(ce[1, 0])) < 1e-5


def test_contraction_is_monotone_along_a_ray():
    t = np.linspace(0.0, 5000.0, 4001)
    d = np.array([0.6, -0.3, 0.2])
    p = (1.0 + t[:, None] * d[None, :]).astype(np.float32)
    c = oracle.contract(p, *BOX)
    assert (np.diff(c[:, 0]) >= 0).all() and (np.diff(c[:, 1]) <= 0).all()
    assert c[-1, 0] < 2.0 and c[-1, 0] > 1.99


def grid_fp64(c, g):
    """Cell of every coordinate by floor((c + 2) g / 4) in FP64, clamped to [0, g - 1]."""
    return np.clip(np.floor((c.astype(np.float64) + 2.0) * g / 4.0), 0, g - 1).astype(np.int64)


def test_grid_matches_fp64_away_from_bounds_and_flattens_x_fastest():
    sc, box = synth.unbounded_city(200_000, seed=11, sh_degree=0)
    grid = (6, 5, 2)
    pos = sc["mean_opac"][:, :3]
    a = oracle.partition_assign(pos, *box, grid)
    c = oracle.contract(pos, *box).astype(np.float64)
    cell = np.stack([grid_fp64(c[:, k], grid[k]) for k in range(3)], axis=1)
    near = np.zeros(len(c), bool)
    for k in range(3):
        b = 4.0 * np.arange(1, grid[k]) / grid[k] - 2.0
        near |= (np.abs(c[:, k][:, None] - b[None, :]) < 1e-5).any(axis=1)
    want = cell[:, 0] + grid[0] * (cell[:, 1] + grid[1] * cell[:, 2])
    assert near.sum() < 100
    np.testing.assert_array_equal(a["block"][~near], want[~near])
    assert a["dropped"] == 0
    np.testing.assert_array_equal(a["count"], np.bincount(a["block"], minlength=60))
    # the contraction balances the blocks: the far background fills the outer ring
    assert (a["count"] > 0).sum() >= 40


def test_grid_half_open_bounds_by_hand():
    # g = 4 along x: inner bounds -1, 0, 1 of the contracted cube [-2, 2]; y, z one cell.
    # In the [0, 2] box, contracted x = p - 1 inside; outside, x = 2 - 1/(p - 1) for p > 2.
    xs = np.array([1.0, 0.0, 0.5, 2.0, -1.0, 1e30, 1.0 - 2 ** -23], np.float32)
    pos = np.stack([xs, np.ones_like(xs), np.ones_like(xs)], axis=1)
    want = [2, 1, 1, 3, 0, 3, 1]   # c = 0 -> cell 2 (b_2 = 0 <= c); c = -1 -> cell 1; c = 1 -> cell 3
    a = oracle.partition_assign(pos, *BOX, (4, 1, 1))
    np.testing.assert_array_equal(a["block"], want)


def test_non_finite_positions_have_no_block():
    pos = np.array([[np.nan, 1, 1], [np.inf, 1, 1], [1, 1, 1], [3e38, 1, 1]], np.float32)
    a = oracle.partition_assign(pos, *BOX, (2, 2, 2))
    assert a["block"][0] == -1 and a["block"][1] == -1 and a["block"][2] >= 0
    assert a["dropped"] == 2 + (a["block"][3] == -1)
    assert a["count"].sum() == 4 - a["dropped"]


def test_order_is_the_stable_sort_by_block():
    rng = np.random.default_rng(3)
    block = rng.integers(-1, 12, size=50_000).astype(np.int32)
    perm, off = oracle.partition_order(block, 12)
    keep = np.flatnonzero(block >= 0)
    want = keep[np.argsort(block[keep], kind="stable")]
    np.testing.assert_array_equal(perm, want)
    np.testing.assert_array_equal(off, np.concatenate([[0], np.cumsum(np.bincount(block[keep], minlength=12))]))
    assert len(oracle.partition_order(np.zeros(0, np.int32), 3)[0]) == 0


def test_pose_in_block_eq4():
    lo = np.array([-750.0, -750.0, -10.0], np.float32)
    hi = np.array([750.0, 750.0, 100.0], np.float32)
    # 4 x 4 x 1 grid: the inner bounds along x and y are at -1, 0, 1 of the contracted cube,
    # i.e. at the foreground box edges and at its centre line
    poses = np.array([[-300.0, -300.0, 50.0],    # inside the box: h = (-0.4, -0.4, 0.09), cell (1, 1)
                      [300.0, -300.0, 50.0],     # (2, 1)
                      [1000.0, 0.0, 50.0],       # h_x = 4/3: c_x = (2 - 3/4) = 1.25 -> (3, 2)
                      [1000.0, 0.0, 200.0],      # altitude dominates: h_z = 31/11, c_x = 0.78 -> (2, 2)
                      [-5000.0, 5000.0, 50.0]],  # far corner: (0, 3)
                     np.float32)
    b = oracle.pose_blocks(poses, lo, hi, (4, 4, 1))
    np.testing.assert_array_equal(b, [1 + 4 * 1, 2 + 4 * 1, 3 + 4 * 2, 2 + 4 * 2, 0 + 4 * 3])
