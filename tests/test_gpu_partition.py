"""GPU parity of the block partition (Sec. 3.2.2: normalisation, Eq. 2 contraction, uniform
grid, stable grouping; Eq. 4: the block of a camera pose) against the oracle, through the C
ABI.  Every output is an integer or a bit pattern decided in FP32, so all of it is compared
bit-exact."""
import numpy as np
import pytest
import torch

import oracle
from paper_2404_01133_b300 import cgs, synth
from paper_2404_01133_b300 import torch_api as ta
from gpu_common import compare_image, gpu_render

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2404_01133_b300 import build
    build.build()
    assert torch.cuda.is_available()


@pytest.fixture(scope="module")
def city():
    return synth.unbounded_city(300_000, seed=21, sh_degree=1)


def run_partition(pos, box, grid, perm=True):
    d = torch.as_tensor(np.ascontiguousarray(pos, np.float32)).cuda()
    block, off, p, ws = ta.partition(d, box[0], box[1], grid, perm=perm)
    assert cgs.cgs_partition_status(ws) == cgs.CGS_OK
    return (block.cpu().numpy(), off.cpu().numpy(), None if p is None else p.cpu().numpy().astype(np.int64))


def check_against_oracle(pos, box, grid):
    nb = int(np.prod(grid))
    gb, goff, gperm = run_partition(pos, box, grid)
    o = oracle.partition_assign(pos, box[0], box[1], grid)
    operm, ooff = oracle.partition_order(o["block"], nb)
    np.testing.assert_array_equal(gb, o["block"])
    np.testing.assert_array_equal(goff, ooff)
    np.testing.assert_array_equal(gperm, operm)
    return o


@pytest.mark.parametrize("grid", [(8, 8, 1), (6, 5, 2), (1, 1, 1), (64, 16, 1), (32, 32, 1)])
def test_partition_matches_oracle(city, grid):
    sc, box = city
    o = check_against_oracle(sc["mean_opac"], box, grid)  # stride 4: the scene's position rows
    assert o["dropped"] == 0


def test_contraction_bit_exact(city):
    sc, box = city
    d = torch.as_tensor(sc["mean_opac"]).cuda()
    out = torch.empty((d.shape[0], 3), dtype=torch.float32, device="cuda")
    cgs.cgs_contract(d, d.shape[0], 4, box[0], box[1], out)
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32),
                                  oracle.contract(sc["mean_opac"], *box).view(np.uint32))


@pytest.mark.parametrize("n", [0, 1, 31, 33, 1023, 1025, 4097])
def test_ragged_sizes_and_non_finite_points(n):
    rng = np.random.default_rng(n)
    pos = (rng.standard_cauchy(size=(n, 3)) * 50.0).astype(np.float32)
    if n > 3:
        pos[1, 0] = np.nan
        pos[2, 2] = np.inf
        pos[3, 1] = -3e38
    box = (np.array([-100, -100, -20], np.float32), np.array([100, 100, 60], np.float32))
    check_against_oracle(pos, box, (5, 7, 3))


def test_points_on_cell_bounds():
    # contracted coordinates exactly on the inner bounds, and their FP32 neighbours
    g = 8
    b = np.array([(4.0 * i) / g - 2.0 for i in range(1, g)], np.float32)
    c = np.concatenate([b, np.nextafter(b, np.float32(-3)), np.nextafter(b, np.float32(3))]).astype(np.float32)
    # the [0, 2] box makes the normalisation h = p - 1; inside [-1, 1] the contraction is the identity
    inner = c[np.abs(c) <= 1.0]
    pos = np.stack([inner + 1.0, np.ones_like(inner), np.ones_like(inner)], axis=1).astype(np.float32)
    box = (np.zeros(3, np.float32), np.full(3, 2.0, np.float32))
    check_against_oracle(pos, box, (g, 1, 1))


def test_pose_blocks_eq4(city):
    sc, box = city
    poses = synth.aerial_poses(sc["side"], 500, seed=3)
    d = torch.as_tensor(poses).cuda()
    out = torch.empty(500, dtype=torch.int32, device="cuda")
    cgs.cgs_pose_blocks(d, 500, 3, box[0], box[1], (8, 8, 1), out)
    np.testing.assert_array_equal(out.cpu().numpy(), oracle.pose_blocks(poses, box[0], box[1], (8, 8, 1)))


@pytest.mark.parametrize("fp16", [False, True])
def test_gather_rows_is_the_permutation(city, fp16):
    sc, box = city
    _, off, perm = run_partition(sc["mean_opac"], box, (8, 8, 1))
    p = torch.as_tensor(perm.astype(np.int32)).cuda()
    for k in ("mean_opac", "scale", "quat", "sh"):
        a = np.ascontiguousarray(sc[k], np.float32)
        if fp16 and k != "mean_opac":
            a = a.astype(np.float16)
        got = ta.gather_rows(torch.as_tensor(a).cuda(), p).cpu().numpy()
        np.testing.assert_array_equal(got.view(np.uint8), a[perm].view(np.uint8))


def test_partitioned_scene_renders_like_the_oracle():
    """Partition, gather into block segments, describe the segments as a one-level block
    scene, and render it: the image equals the oracle's render of the same grouped scene."""
    sc, box = synth.unbounded_city(60_000, seed=5, sh_degree=1, area_km2=0.01)
    grid = (4, 4, 1)
    _, off, perm = run_partition(sc["mean_opac"], box, grid)
    p = torch.as_tensor(perm.astype(np.int32)).cuda()
    grouped = {k: ta.gather_rows(torch.as_tensor(np.ascontiguousarray(sc[k], np.float32)).cuda(), p)
               for k in ("mean_opac", "scale", "quat", "sh")}
    nb = int(np.prod(grid))
    gsc = {k: v.cpu().numpy() for k, v in grouped.items()}
    gsc.update({"sh_degree": sc["sh_degree"], "level_offset": off[:nb].reshape(nb, 1).astype(np.int64),
                "level_count": np.diff(off).reshape(nb, 1).astype(np.int64),
                "block_cell": np.zeros((nb, 4), np.float32)})
    cam = synth.pitched_camera((0.0, -60.0, 60.0), 0.0, np.radians(40.0), 300.0, 300.0, 320, 240)
    g = gpu_render(gsc, [cam], levels=np.zeros((1, nb), np.int8))
    assert g["status"] == 0
    o = oracle.render(gsc, cam)
    compare_image(g["image"][0], g["final_T"][0], g["n_contrib"][0], o)


def test_full_size_partition_20m():
    """The 20M-Gaussian unbounded city on an 8 x 8 grid, in the benchmark's launch
    configuration: blocks, offsets and the grouped order all bit-exact."""
    sc, box = synth.unbounded_city(20_000_000, seed=3, defer_sh=True)
    check_against_oracle(sc["mean_opac"], box, (8, 8, 1))


def test_rank_is_the_inverse_and_scatter_equals_gather(city):
    sc, box = city
    pos = sc["mean_opac"].copy()
    pos[5, 0] = np.nan                                        # one point with no block
    d = torch.as_tensor(pos).cuda()
    block, off, perm, ws, rank = ta.partition(d, box[0], box[1], (8, 8, 1), rank=True)
    p = perm.cpu().numpy()
    r = rank.cpu().numpy()
    assert r[5] == -1 and len(p) == len(pos) - 1
    np.testing.assert_array_equal(r[p], np.arange(len(p)))
    for k in ("mean_opac", "sh"):
        src = torch.as_tensor(np.ascontiguousarray(sc[k], np.float32)).cuda()
        a = ta.gather_rows(src, perm)
        b = ta.scatter_rows(src, rank, len(p))
        assert torch.equal(a, b)
