"""GPU parity of the backward pass (differentiable rendering, Sec. 3.1) and of the full-size
1080p / 1M-Gaussian forward+backward workload against the CPU oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
from paper_2404_01133_b300 import cgs, synth
from paper_2404_01133_b300 import torch_api as ta
from gpu_common import canonical_ranges, compare_image, frame_arrays, gpu_render

pytestmark = pytest.mark.gpu

# Gradients: relative 1e-3 per tensor (the benchmark spec's bound, as a norm).  Per element the
# bound is 1e-3 of |g| plus 1e-3 of the tensor's largest magnitude: each element is an FP32
# sum of hundreds of per-pixel terms accumulated in a different order on each side, then
# chained through the quaternion normalisation and rotation, where terms cancel; on the
# 1080p workload the largest such difference measured 2.8e-4 of the tensor maximum, and the
# FP32 oracle itself differs from the FP64 one by up to 2.6e-4 of it.
G_RTOL = 1e-3
G_ELEM = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2404_01133_b300 import build
    build.build()
    assert torch.cuda.is_available()


def gpu_grads(g, dL):
    d = torch.as_tensor(dL, dtype=torch.float32).cuda().reshape(g["image"].shape).contiguous()
    gm, gs_, gq, gsh = ta.render_backward(g["ds"], g["frame"], g["cfg"], g["cams"], d, g["final_T"], g["n_contrib"])
    torch.cuda.synchronize()
    return {"mean": gm[:, :3].cpu().numpy(), "opac": gm[:, 3].cpu().numpy(), "scale": gs_[:, :3].cpu().numpy(),
            "quat": gq.cpu().numpy(), "sh": gsh.cpu().numpy()}


def gpu_grads_packed(g, dL, sentinel=None):
    """Packed backward rows, and the same gradients scattered into scene-indexed arrays by
    summing rows of equal index (float64 sums)."""
    d = torch.as_tensor(dL, dtype=torch.float32).cuda().reshape(g["image"].shape).contiguous()
    rows = None
    if sentinel is not None:
        fr, ds = g["frame"], g["ds"]
        cap = fr.n_cap
        rows = tuple(torch.full(sh, sentinel, dtype=torch.float32, device="cuda")
                     for sh in ((cap, 4), (cap, 4), (cap, 4), (cap,) + tuple(ds.sh.shape[1:])))
        rows = rows + (torch.full((cap,), -7, dtype=torch.int64, device="cuda"),)
    rows = ta.render_backward_packed(g["ds"], g["frame"], g["cfg"], g["cams"], d, g["final_T"], g["n_contrib"],
                                     rows=rows)
    torch.cuda.synchronize()
    st, counts = g["frame"].status()
    n_vis = int(counts[1])
    gm, gs_, gq, gsh, gi = (t.cpu().numpy() for t in rows)
    n = g["ds"].n
    dense = {}
    for k, src in (("mo", gm), ("sc", gs_), ("q", gq), ("sh", gsh)):
        acc = np.zeros((n,) + src.shape[1:], np.float64)
        np.add.at(acc, gi[:n_vis], src[:n_vis].astype(np.float64))
        dense[k] = acc
    out = {"mean": dense["mo"][:, :3], "opac": dense["mo"][:, 3], "scale": dense["sc"][:, :3], "quat": dense["q"],
           "sh": dense["sh"]}
    return out, (gm, gs_, gq, gsh, gi), n_vis


def compare_grads(gg, og, rows=None, rtol=G_RTOL, elem=G_ELEM):
    for k in ("mean", "opac", "scale", "quat", "sh"):
        a = gg[k].astype(np.float64)
        b = og[k].astype(np.float64)
        if rows is not None:
            a, b = a[rows], b[rows]
        nb = np.linalg.norm(b)
        assert np.linalg.norm(a - b) <= rtol * nb + 1e-30, (k, np.linalg.norm(a - b) / nb)
        scale = np.abs(og[k]).max()
        bad = np.abs(a - b) > elem * scale + rtol * np.abs(b)
        assert not bad.any(), (k, np.argwhere(bad)[:5], a[bad][:5], b[bad][:5])


@pytest.mark.parametrize("tile,batch,deg", [(16, 256, 3), (16, 64, 1), (8, 64, 3), (8, 32, 0)])
def test_backward_matches_oracle(tile, batch, deg):
    sc = synth.single_block(synth.random_cube_scene(800, seed=4 + deg, sh_degree=deg, log_scale_mu=-2.4))
    cam = synth.small_scene_camera(96, 80, f=80.0, dist=3.0)
    cfg = oracle.make_config(tile=tile)
    o = oracle.render(sc, cam, cfg)
    w = np.random.default_rng(9).normal(size=(3, 80, 96)).astype(np.float32)
    w[:, o["ambiguous"].astype(bool)] = 0.0  # pixels near a decision threshold carry no gradient
    og = oracle.render_backward(sc, cam, w, cfg, real="f32", fwd=o)
    g = gpu_render(sc, [cam], tile=tile, batch=batch)
    compare_image(g["image"][0], g["final_T"][0], g["n_contrib"][0], o)
    gg = gpu_grads(g, w)
    compare_grads(gg, og)
    # the FP64 oracle (pinned by finite differences) agrees to the same relative bound
    og64 = oracle.render_backward(sc, cam, w, cfg, real="f64")
    if og64["fwd"]["hash"] == o["hash"]:
        for k in ("mean", "opac", "scale", "quat", "sh"):
            assert np.linalg.norm(gg[k] - og64[k]) <= G_RTOL * np.linalg.norm(og64[k])
    st, counts = g["frame"].status()
    assert st == 0 and counts[4] > 0


def test_backward_twice_accumulates_and_state_resets():
    sc = synth.single_block(synth.random_cube_scene(400, seed=21, sh_degree=2, log_scale_mu=-2.4))
    cam = synth.small_scene_camera(64, 64, f=70.0, dist=3.0)
    g = gpu_render(sc, [cam])
    w = np.random.default_rng(3).normal(size=(3, 64, 64)).astype(np.float32)
    a = gpu_grads(g, w)
    b = gpu_grads(g, w)  # a second backward of the same forward starts from cleared state
    # (a state left over would double every gradient).  The two runs differ only in the order
    # in which warps add their FP32 moment sums to a Gaussian's accumulator, which the opacity
    # and conic factors of dL/du, dL/dv can amplify where their two terms cancel: measured up to
    # 1.4e-7 of the tensor maximum
    for k in a:
        np.testing.assert_allclose(a[k], b[k], rtol=1e-4, atol=1e-5 * np.abs(a[k]).max())


def test_backward_without_the_pair_count_gives_the_same_gradients():
    """A frame flagged CGS_FRAME_NO_PAIR_COUNT: the backward's gradients are those of the
    counting backward (up to the order of its atomic additions) and the contributing-pair
    count is left out, in a backward of an existing frame and in a fresh forward + backward."""
    sc = synth.single_block(synth.random_cube_scene(600, seed=23, sh_degree=3, log_scale_mu=-2.4))
    cam = synth.small_scene_camera(80, 64, f=70.0, dist=3.0)
    g = gpu_render(sc, [cam])
    w = np.random.default_rng(4).normal(size=(3, 64, 80)).astype(np.float32)
    a = gpu_grads(g, w)
    pairs = g["frame"].status()[1][4]
    assert pairs > 0
    g["frame"].struct.flags = cgs.CGS_FRAME_NO_PAIR_COUNT
    b = gpu_grads(g, w)
    assert g["frame"].status()[1][4] == pairs        # not counted again
    for k in a:
        np.testing.assert_allclose(b[k], a[k], rtol=1e-4, atol=1e-5 * np.abs(a[k]).max())
    ta.render_forward(g["ds"], g["frame"], g["cfg"], g["cams"], out=(g["image"], g["final_T"], g["n_contrib"]))
    c = gpu_grads(g, w)
    st, counts = g["frame"].status()
    assert st == 0 and counts[4] == 0 and counts[3] > 0
    for k in a:
        np.testing.assert_allclose(c[k], a[k], rtol=1e-4, atol=1e-5 * np.abs(a[k]).max())


def test_l1_loss_kernel():
    rng = np.random.default_rng(5)
    img = rng.uniform(size=(3, 50, 70)).astype(np.float32)
    tgt = rng.uniform(size=(3, 50, 70)).astype(np.float32)
    tgt[1, 2, 3] = img[1, 2, 3]
    loss, grad = ta.l1_loss(torch.tensor(img).cuda(), torch.tensor(tgt).cuda())
    oloss, ograd = oracle.l1(img, tgt)
    assert abs(loss.item() - oloss) <= 1e-6 * oloss
    np.testing.assert_array_equal(grad.cpu().numpy(), ograd)


def test_l1_loss_kernel_with_8bit_target():
    rng = np.random.default_rng(6)
    img = rng.uniform(size=(3, 37, 61)).astype(np.float32)
    t8 = rng.integers(0, 256, size=(3, 37, 61)).astype(np.uint8)
    img[0, 1, 2] = np.float32(t8[0, 1, 2]) / np.float32(255)   # an exact tie: gradient 0
    loss, grad = ta.l1_loss(torch.tensor(img).cuda(), torch.tensor(t8).cuda())
    # an 8-bit channel value t stands for t / 255 (FP32 quotient, correctly rounded)
    oloss, ograd = oracle.l1(img, t8.astype(np.float32) / np.float32(255))
    assert abs(loss.item() - oloss) <= 1e-6 * oloss
    np.testing.assert_array_equal(grad.cpu().numpy(), ograd)
    assert ograd[0, 1, 2] == 0.0
    # unaligned views take the one-value-per-thread path, with the same results
    big = torch.zeros(img.size + 1, device="cuda")
    big[1:] = torch.tensor(img.ravel()).cuda()
    t8b = torch.zeros(t8.size + 1, dtype=torch.uint8, device="cuda")
    t8b[1:] = torch.tensor(t8.ravel()).cuda()
    loss2, grad2 = ta.l1_loss(big[1:], t8b[1:])
    assert abs(loss2.item() - oloss) <= 1e-6 * oloss
    np.testing.assert_array_equal(grad2.cpu().numpy().reshape(img.shape), ograd)


def test_autograd_function_matches_direct_backward():
    sc = synth.single_block(synth.random_cube_scene(300, seed=8, sh_degree=1, log_scale_mu=-2.3))
    cam = synth.small_scene_camera(48, 48, f=60.0, dist=3.0)
    g = gpu_render(sc, [cam])
    ds = g["ds"]
    params = [t.clone().requires_grad_(True) for t in (ds.mean_opac, ds.scale, ds.quat, ds.sh)]
    img, T, nc = ta.RenderFn.apply(*params, ds, g["frame"], g["cfg"], g["cams"])
    w = torch.randn_like(img)
    (img * w).sum().backward()
    direct = gpu_grads(g, w.detach().cpu().numpy())
    np.testing.assert_allclose(params[0].grad[:, :3].cpu().numpy(), direct["mean"], rtol=1e-5,
                               atol=1e-6 * np.abs(direct["mean"]).max())
    np.testing.assert_allclose(params[3].grad.cpu().numpy(), direct["sh"], rtol=1e-5,
                               atol=1e-6 * np.abs(direct["sh"]).max())


def test_full_size_city_1m_forward_backward():
    """The 1920x1080, 1M-Gaussian SH-3 workload in the benchmark's launch configuration:
    every key, value and range bit-exact; every pixel; the gradients of 64 sampled visible
    Gaussians and of every attribute tensor against the FP32 and FP64 oracles."""
    sc, cams = synth.workload_city_1m()
    cam = cams[0]
    g = gpu_render(sc, cams, n_cap=1_000_000, k_cap=4_000_000)
    assert g["status"] == 0
    pr = oracle.project(sc, cam)
    srt = oracle.bin_and_sort(pr, cam)
    a = frame_arrays(g)
    assert g["counts"][2] == pr["n_entries"]
    np.testing.assert_array_equal(a["keys"].astype(np.int64), (srt["keys"] >> np.uint64(32)).astype(np.int64))
    np.testing.assert_array_equal(a["vals"].astype(np.int64), srt["vals"].astype(np.int64))
    np.testing.assert_array_equal(canonical_ranges(a["ranges"]), srt["ranges"])
    vis = pr["tiles_touched"] > 0
    np.testing.assert_array_equal(a["records"][vis, 0:2], pr["xy"][vis])
    np.testing.assert_array_equal(a["records"][vis, 8:11], pr["rgb"][vis])
    # full oracle composite (seconds), compare every pixel
    o = oracle.composite(pr, srt, cam)
    n_amb = compare_image(g["image"][0], g["final_T"][0], g["n_contrib"][0], o, rgb_max=pr["rgb"][vis],
                          label="1920x1080 city, 1M Gaussians")
    # backward of the L1 loss against the seeded target; the upstream gradient is the oracle's
    tgt = synth.target_image(1, cam["width"], cam["height"])
    _, dL = oracle.l1(o["image"], tgt)
    dL[:, o["ambiguous"].astype(bool)] = 0.0
    o["proj"], o["sort"] = pr, srt
    og = oracle.render_backward(sc, cam, dL, real="f32", fwd=o)
    gg = gpu_grads(g, dL)
    rows = np.random.default_rng(0).choice(np.flatnonzero(vis), size=64, replace=False)
    compare_grads(gg, og, rows=rows)
    compare_grads(gg, og)
    # and against the FP64 oracle, whose gradient is pinned by finite differences
    og64 = oracle.render_backward(sc, cam, dL.astype(np.float64), real="f64")
    for k in ("mean", "opac", "scale", "quat", "sh"):
        assert np.linalg.norm(gg[k] - og64[k]) <= G_RTOL * np.linalg.norm(og64[k]), k


@pytest.mark.parametrize("deg", [3, 1])
def test_packed_backward_rows_match_dense_backward(deg):
    """One view: every visible Gaussian owns one packed row, whose values are the dense
    backward's row (up to the order in which the compositing backward adds each Gaussian's
    screen-space gradient, which differs between runs in the last bits); rows past the visible
    count are left as they were; the row indices follow the visible list."""
    sc = synth.single_block(synth.random_cube_scene(900, seed=30 + deg, sh_degree=deg, log_scale_mu=-2.4))
    cam = synth.small_scene_camera(96, 80, f=80.0, dist=3.0)
    cfg = oracle.make_config(tile=16)
    o = oracle.render(sc, cam, cfg)
    w = np.random.default_rng(12).normal(size=(3, 80, 96)).astype(np.float32)
    w[:, o["ambiguous"].astype(bool)] = 0.0
    g = gpu_render(sc, [cam])
    dense = gpu_grads(g, w)
    packed, rows, n_vis = gpu_grads_packed(g, w, sentinel=np.float32(1234.5))
    gm, gs_, gq, gsh, gi = rows
    assert n_vis > 100
    # rows past n_vis untouched
    assert (gi[n_vis:] == -7).all() and (gm[n_vis:] == 1234.5).all() and (gsh[n_vis:] == 1234.5).all()
    # the visible list's scene indices, each once
    vis = g["frame"].buffer(cgs.BUF_VISIBLE, torch.int32, count=n_vis).cpu().numpy()
    sidx = g["frame"].buffer(cgs.BUF_SCENE_INDEX, torch.int32, count=g["counts"][0]).cpu().numpy()
    np.testing.assert_array_equal(gi[:n_vis], sidx[vis])
    assert len(np.unique(gi[:n_vis])) == n_vis
    for k in ("mean", "opac", "scale", "quat", "sh"):
        b = dense[k].astype(np.float64)
        np.testing.assert_allclose(packed[k], b, rtol=1e-5, atol=1e-6 * np.abs(b).max(), err_msg=k)
        assert ((packed[k] != 0) == (b != 0)).mean() > 0.999, k   # the same rows carry gradient
    assert (gs_[:n_vis, 3] == 0).all()
    # and the oracle's gradient
    og = oracle.render_backward(sc, cam, w, cfg, real="f32", fwd=o)
    compare_grads({k: v.astype(np.float32) for k, v in packed.items()}, og)


def test_packed_backward_multi_view_sums_to_dense():
    """Several views in one frame: a Gaussian seen by k views owns k rows; their sum is the
    dense backward's accumulated gradient (up to the order of FP32 additions)."""
    sc = synth.single_block(synth.random_cube_scene(700, seed=41, sh_degree=3, log_scale_mu=-2.4))
    cams = [synth.look_at((x, 0.4, -3.2), (0, 0, 0), (0, -1, 0), 60.0, 60.0, 64, 48) for x in (-0.8, 0.0, 0.9)]
    g = gpu_render(sc, cams)
    w = np.random.default_rng(13).normal(size=(3, 3, 48, 64)).astype(np.float32)
    dense = gpu_grads(g, w)
    packed, rows, n_vis = gpu_grads_packed(g, w)
    gi = rows[4][:n_vis]
    assert n_vis > len(np.unique(gi))  # some Gaussians are visible in more than one view
    for k in ("mean", "opac", "scale", "quat", "sh"):
        a, b = packed[k], dense[k].astype(np.float64)
        np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-6 * np.abs(b).max(), err_msg=k)


@pytest.mark.parametrize("case", ["small16", "small8", "city1m"])
def test_backward_replays_exactly_the_forward_blends(case):
    """The compositing backward (built with flush-to-zero) replays exactly the forward's blends:
    the number of (pixel, Gaussian) pairs its replay takes equals the forward's per-Gaussian
    blended-pixel counts summed (the two kernels take every skip and stop decision alike)."""
    if case == "city1m":
        sc, cams = synth.workload_city_1m()
        tile, batch, n_cap, k_cap = 16, 128, 1_000_000, 4_000_000
    else:
        sc = synth.single_block(synth.random_cube_scene(1500, seed=77, sh_degree=2, log_scale_mu=-2.2))
        cams = [synth.small_scene_camera(120, 90, f=90.0, dist=3.0)]
        tile, batch = (16, 64) if case == "small16" else (8, 32)
        n_cap, k_cap = None, None
    g = gpu_render(sc, cams, tile=tile, batch=batch, n_cap=n_cap, k_cap=k_cap)
    hits = torch.zeros(g["ds"].n, dtype=torch.int32, device="cuda")
    img, T, nc = ta.render_forward_hits(g["ds"], g["frame"], g["cfg"], g["cams"], hits)
    dL = torch.randn_like(img)
    ta.render_backward_packed(g["ds"], g["frame"], g["cfg"], g["cams"], dL, T, nc)
    torch.cuda.synchronize()
    st, counts = g["frame"].status()
    assert st == 0
    blends = int(hits.to(torch.int64).sum().item())
    assert blends > 0 and counts[4] == blends, (counts[4], blends)
