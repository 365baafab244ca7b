"""GPU parity of the L1 loss folded into the compositing backward (cgs_render_backward_l1): the
same loss and gradients as cgs_l1_loss followed by the backward, and the oracle's gradient of
the L1 loss (Sec. 3.2.3's L1 term, Sec. 3.1's differentiable rendering), through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
from paper_2404_01133_b300 import cgs, synth
from paper_2404_01133_b300 import torch_api as ta
from gpu_common import gpu_render
from test_gpu_backward import compare_grads, gpu_grads_packed

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2404_01133_b300 import build
    build.build()
    assert torch.cuda.is_available()


def dense_from_rows(rows, n_vis, n):
    gm, gs_, gq, gsh, gi = (t.cpu().numpy() for t in rows)
    out = {}
    for k, src in (("mo", gm), ("sc", gs_), ("q", gq), ("sh", gsh)):
        acc = np.zeros((n,) + src.shape[1:], np.float64)
        np.add.at(acc, gi[:n_vis], src[:n_vis].astype(np.float64))
        out[k] = acc
    return {"mean": out["mo"][:, :3], "opac": out["mo"][:, 3], "scale": out["sc"][:, :3], "quat": out["q"],
            "sh": out["sh"]}


def close(a, b, what):
    # the two runs differ only in the order of the backward's atomic FP32 additions
    for k in a:
        x, y = np.asarray(a[k], np.float64), np.asarray(b[k], np.float64)
        np.testing.assert_allclose(x, y, rtol=1e-4, atol=1e-5 * max(np.abs(y).max(), 1e-30), err_msg=f"{what} {k}")


@pytest.mark.parametrize("tile,batch,u8,n_views", [(16, 128, True, 1), (16, 64, False, 3), (8, 32, True, 2),
                                                   (8, 64, False, 1)])
def test_fused_l1_backward_equals_separate_loss_and_backward(tile, batch, u8, n_views):
    sc = synth.single_block(synth.random_cube_scene(900, seed=50 + tile + n_views, sh_degree=3, log_scale_mu=-2.4))
    cams = [synth.look_at((x, 0.3, -3.1), (0, 0, 0), (0, -1, 0), 70.0, 70.0, 83, 61)
            for x in (-0.7, 0.0, 0.8)[:n_views]]
    g = gpu_render(sc, cams, tile=tile, batch=batch)
    assert g["status"] == 0
    img, T, nc = g["image"], g["final_T"], g["n_contrib"]
    rng = np.random.default_rng(tile * 10 + n_views)
    if u8:
        tgt = torch.as_tensor(rng.integers(0, 256, size=tuple(img.shape)).astype(np.uint8)).cuda()
    else:
        tgt = torch.as_tensor(rng.uniform(size=tuple(img.shape)).astype(np.float32)).cuda()
        tgt.view(-1)[::97] = img.view(-1)[::97]  # exact ties: gradient 0
    # separate: loss kernel, then the packed and the scene-indexed backward
    loss_s, dL = ta.l1_loss(img, tgt)
    rows_s = ta.render_backward_packed(g["ds"], g["frame"], g["cfg"], g["cams"], dL, T, nc)
    torch.cuda.synchronize()
    n_vis = int(g["frame"].status()[1][1])
    dense_s = dense_from_rows(rows_s, n_vis, g["ds"].n)
    # fused, packed rows
    loss_f, rows_f = ta.render_backward_l1(g["ds"], g["frame"], g["cfg"], g["cams"], img, tgt, T, nc)
    torch.cuda.synchronize()
    assert int(g["frame"].status()[1][1]) == n_vis
    np.testing.assert_array_equal(rows_f[4][:n_vis].cpu().numpy(), rows_s[4][:n_vis].cpu().numpy())
    dense_f = dense_from_rows(rows_f, n_vis, g["ds"].n)
    close(dense_f, dense_s, "packed")
    assert abs(loss_f.item() - loss_s.item()) <= 2e-6 * loss_s.item()
    # the loss against the oracle's L1 of the same image
    tv = tgt.cpu().numpy().astype(np.float32)
    if u8:
        tv = tv / np.float32(255)
    oloss, _ = oracle.l1(img.cpu().numpy(), tv)
    assert abs(loss_f.item() - oloss) <= 2e-6 * oloss
    # fused, scene-indexed gradients added into arrays (twice: the second call adds the same)
    f32 = torch.float32
    ds = g["ds"]
    grads = (torch.zeros_like(ds.mean_opac), torch.zeros_like(ds.scale, dtype=f32),
             torch.zeros_like(ds.quat, dtype=f32), torch.zeros_like(ds.sh, dtype=f32))
    loss_1, _ = ta.render_backward_l1(ds, g["frame"], g["cfg"], g["cams"], img, tgt, T, nc, grads=grads)
    torch.cuda.synchronize()
    d1 = {"mean": grads[0][:, :3].cpu().numpy(), "opac": grads[0][:, 3].cpu().numpy(),
          "scale": grads[1][:, :3].cpu().numpy(), "quat": grads[2].cpu().numpy(), "sh": grads[3].cpu().numpy()}
    close(d1, dense_s, "scene-indexed")
    ta.render_backward_l1(ds, g["frame"], g["cfg"], g["cams"], img, tgt, T, nc, grads=grads)
    torch.cuda.synchronize()
    d2 = {"mean": grads[0][:, :3].cpu().numpy(), "opac": grads[0][:, 3].cpu().numpy(),
          "scale": grads[1][:, :3].cpu().numpy(), "quat": grads[2].cpu().numpy(), "sh": grads[3].cpu().numpy()}
    close(d2, {k: 2 * v for k, v in d1.items()}, "accumulated")
    assert abs(loss_1.item() - loss_s.item()) <= 2e-6 * loss_s.item()


def test_fused_l1_backward_matches_oracle():
    """The oracle's backward of its L1 gradient on the GPU image: where a pixel lies near a
    decision threshold the target is set to the rendered value there, so its L1 gradient is
    exactly zero on both sides and the two need not take the same near-threshold branch."""
    sc = synth.single_block(synth.random_cube_scene(800, seed=61, sh_degree=3, log_scale_mu=-2.4))
    cam = synth.small_scene_camera(96, 80, f=80.0, dist=3.0)
    cfg = oracle.make_config(tile=16)
    o = oracle.render(sc, cam, cfg)
    g = gpu_render(sc, [cam], tile=16, batch=128)
    img = g["image"][0].cpu().numpy()
    tgt = np.random.default_rng(62).uniform(size=img.shape).astype(np.float32)
    amb = o["ambiguous"].astype(bool)
    tgt[:, amb] = img[:, amb]
    oloss, odL = oracle.l1(img, tgt)
    assert (odL[:, amb] == 0).all()
    og = oracle.render_backward(sc, cam, odL, cfg, real="f32", fwd=o)
    loss, rows = ta.render_backward_l1(g["ds"], g["frame"], g["cfg"], g["cams"], g["image"],
                                       torch.as_tensor(tgt)[None].cuda(), g["final_T"], g["n_contrib"])
    torch.cuda.synchronize()
    n_vis = int(g["frame"].status()[1][1])
    gg = dense_from_rows(rows, n_vis, g["ds"].n)
    compare_grads({k: v.astype(np.float32) for k, v in gg.items()}, og)
    assert abs(loss.item() - oloss) <= 2e-6 * oloss


def test_fused_l1_backward_rejects_parity_config_and_bad_target_type():
    sc = synth.single_block(synth.random_cube_scene(200, seed=63, sh_degree=0, log_scale_mu=-2.4))
    cam = synth.small_scene_camera(32, 32, f=40.0, dist=3.0)
    g = gpu_render(sc, [cam], cfg_kw={"exact": 1})
    tgt = torch.zeros_like(g["image"])
    with pytest.raises(cgs.CgsError) as e:
        ta.render_backward_l1(g["ds"], g["frame"], g["cfg"], g["cams"], g["image"], tgt, g["final_T"],
                              g["n_contrib"])
    assert e.value.code == cgs.CGS_ERR_UNSUPPORTED
    g2 = gpu_render(sc, [cam])
    rows = gpu_grads_packed(g2, np.zeros((3, 32, 32), np.float32))[1]
    loss = torch.zeros(1, device="cuda")
    with pytest.raises(cgs.CgsError) as e:
        cgs.cgs_render_backward_l1(g2["ds"].struct(), g2["frame"].struct, g2["cfg"], g2["cams"], g2["image"], tgt, 2,
                                   g2["final_T"], g2["n_contrib"], loss, *[torch.as_tensor(r).cuda() for r in rows])
    assert e.value.code == cgs.CGS_ERR_INVALID_ARGUMENT
