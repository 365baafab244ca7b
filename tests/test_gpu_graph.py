"""The training step -- forward render (Eq. 1), L1 loss, packed backward (differentiable
rendering, Sec. 3.1) -- captured once into a CUDA graph with the package's capture helper and
replayed, as the benchmark times it.  The replay must equal the eager step bit for bit and the
oracle within the parity bounds, also after the camera buffer is overwritten with another pose
between replays: a step that read a count on the host while being captured, or baked a pointer
or a pose into the graph, fails here."""
import numpy as np
import pytest
import torch

import oracle
from paper_2404_01133_b300 import cgs, synth
from paper_2404_01133_b300 import torch_api as ta
from gpu_common import compare_image

pytestmark = pytest.mark.gpu

G_RTOL = 1e-3
G_ELEM = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2404_01133_b300 import build
    build.build()
    assert torch.cuda.is_available()


def _scene_and_poses():
    sc = synth.single_block(synth.random_cube_scene(3000, seed=21, sh_degree=3, log_scale_mu=-2.6))
    poses = [synth.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), (0.0, -1.0, 0.0), 150.0, 150.0, 136, 104),
             synth.look_at((0.5, -0.3, -3.7), (0.05, 0.0, 0.0), (0.0, -1.0, 0.0), 150.0, 150.0, 136, 104)]
    return sc, poses


class Step:
    """Device buffers and the step itself (forward, L1 against an FP32 target, packed backward)."""

    def __init__(self, sc, cam, target, tile=16, batch=64):
        self.ds = ta.DeviceScene(sc)
        self.cfg = ta.make_config(tile=tile, batch=batch)
        W, H = cam["width"], cam["height"]
        self.frame = ta.Frame(1, W, H, tile, 1, self.ds.n, 64 * self.ds.n)
        self.d_cams = ta.cameras_device([cam])
        self.img, self.T, self.nc = self.frame.outputs()
        self.tgt = torch.as_tensor(target).cuda()[None].contiguous()
        self.loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        self.dL = torch.empty_like(self.img)
        cap, f32 = self.frame.n_cap, torch.float32
        self.rows = (torch.empty((cap, 4), dtype=f32, device="cuda"), torch.empty((cap, 4), dtype=f32, device="cuda"),
                     torch.empty((cap, 4), dtype=f32, device="cuda"),
                     torch.empty((cap,) + tuple(self.ds.sh.shape[1:]), dtype=f32, device="cuda"),
                     torch.empty(cap, dtype=torch.int64, device="cuda"))
        self.s = self.ds.struct()

    def __call__(self):
        cur = torch.cuda.current_stream().cuda_stream
        cgs.cgs_render_forward(self.s, self.frame.struct, self.cfg, self.d_cams, None, None, self.img, self.T,
                               self.nc, cur)
        self.loss.zero_()
        cgs.cgs_l1_loss(self.img, self.tgt, self.img.numel(), self.loss, self.dL, cur)
        cgs.cgs_render_backward_packed(self.s, self.frame.struct, self.cfg, self.d_cams, self.dL, self.T, self.nc,
                                       *self.rows, cur)

    def poison(self):
        for t in (self.img, self.T, self.dL) + self.rows[:4]:
            t.fill_(float("nan"))
        self.nc.fill_(-1)
        self.loss.fill_(float("nan"))
        self.rows[4].fill_(-9)

    def snapshot(self):
        torch.cuda.synchronize()
        st, counts = self.frame.status()
        n_vis = int(counts[1])
        gi = self.rows[4][:n_vis].cpu().numpy()
        order = np.argsort(gi, kind="stable")
        rows = [r[:n_vis].cpu().numpy()[order] for r in self.rows[:4]]
        return {"status": st, "counts": list(counts[:5]), "image": self.img.clone(), "T": self.T.clone(),
                "nc": self.nc.clone(), "loss": float(self.loss.item()), "dL": self.dL.clone(), "index": gi[order],
                "rows": rows}


def dense_from_rows(snap, n):
    gm, gs_, gq, gsh = snap["rows"]
    out = {}
    for k, src in (("mo", gm), ("sc", gs_), ("q", gq), ("sh", gsh)):
        acc = np.zeros((n,) + src.shape[1:], np.float64)
        np.add.at(acc, snap["index"], src.astype(np.float64))
        out[k] = acc
    return {"mean": out["mo"][:, :3], "opac": out["mo"][:, 3], "scale": out["sc"][:, :3], "quat": out["q"],
            "sh": out["sh"]}


def assert_same_step(a, b):
    assert a["status"] == b["status"] == 0
    assert a["counts"] == b["counts"]
    for k in ("image", "T", "nc", "dL"):
        assert torch.equal(a[k], b[k]), k
    # the loss is summed with one atomic add per CTA, in scheduling order
    assert abs(a["loss"] - b["loss"]) <= 1e-6 * abs(b["loss"])
    np.testing.assert_array_equal(a["index"], b["index"])
    # the backward's screen-space sums are added in scheduling order: the last bits may differ,
    # more where terms cancel (measured up to 1.1e-4 relative on an element near zero)
    for x, y in zip(a["rows"], b["rows"]):
        np.testing.assert_allclose(x, y, rtol=1e-4, atol=1e-5 * max(1e-30, float(np.abs(y).max())))


def check_against_oracle(sc, cam, target, snap):
    o = oracle.render(sc, cam)
    compare_image(snap["image"][0], snap["T"][0], snap["nc"][0], o, label="graph-replayed step")
    loss, dL = oracle.l1(o["image"], target)
    assert abs(snap["loss"] - loss) <= 1e-5 * max(loss, 1e-6)
    # the step's upstream gradient (sign(img - target) / count) equals the oracle's wherever
    # the pixel is not ambiguous and its value is not within the pixel tolerance of the target
    amb = o["ambiguous"].astype(bool)
    sure = ~amb[None] & (np.abs(o["image"] - target) > 1e-4)
    gd = snap["dL"][0].cpu().numpy()
    np.testing.assert_array_equal(gd[sure], dL[sure])
    og = oracle.render_backward(sc, cam, dL, fwd=o)
    return o, og, bool(sure.all())


def check_keys(st, o):
    torch.cuda.synchronize()
    _, counts = st.frame.status()
    k = int(counts[2])
    keys = st.frame.buffer(cgs.BUF_TILE_KEYS, torch.int32, count=k).cpu().numpy().view(np.uint32)
    vals = st.frame.buffer(cgs.BUF_TILE_VALS, torch.int32, count=k).cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(keys.astype(np.int64), (o["sort"]["keys"] >> np.uint64(32)).astype(np.int64))
    np.testing.assert_array_equal(vals.astype(np.int64), o["sort"]["vals"].astype(np.int64))


def test_graph_replayed_step_equals_eager_and_oracle():
    sc, poses = _scene_and_poses()
    W, H = poses[0]["width"], poses[0]["height"]
    target = synth.target_image(5, W, H)
    st = Step(sc, poses[0], target)
    st()  # eager
    eager = st.snapshot()
    assert eager["status"] == 0 and eager["counts"][1] > 200
    g = ta.capture(st, warmup=1)
    for _ in range(2):
        st.poison()
        g.replay()
        assert_same_step(st.snapshot(), eager)
    o, _, _ = check_against_oracle(sc, poses[0], target, eager)
    check_keys(st, o)
    # gradients against the oracle: a second graph, forward and backward of a fixed upstream
    # gradient w (random, zero at the oracle's ambiguous pixels), replayed like the first
    w = np.random.default_rng(3).normal(size=(3, H, W)).astype(np.float32)
    w[:, o["ambiguous"].astype(bool)] = 0.0
    st.dL_fixed = torch.as_tensor(w).cuda()[None].contiguous()

    def fwd_bwd():
        cur = torch.cuda.current_stream().cuda_stream
        cgs.cgs_render_forward(st.s, st.frame.struct, st.cfg, st.d_cams, None, None, st.img, st.T, st.nc, cur)
        cgs.cgs_render_backward_packed(st.s, st.frame.struct, st.cfg, st.d_cams, st.dL_fixed, st.T, st.nc,
                                       *st.rows, cur)
    g2 = ta.capture(fwd_bwd, warmup=1)
    st.poison()
    g2.replay()
    snap = st.snapshot()
    assert snap["status"] == 0
    gg = dense_from_rows(snap, st.ds.n)
    og = oracle.render_backward(sc, poses[0], w, fwd=o)
    for k in ("mean", "opac", "scale", "quat", "sh"):
        a, b = gg[k], og[k].astype(np.float64)
        assert np.linalg.norm(a - b) <= G_RTOL * np.linalg.norm(b) + 1e-30, k
        assert not (np.abs(a - b) > G_ELEM * np.abs(b).max() + G_RTOL * np.abs(b)).any(), k


def test_graph_replay_follows_the_camera_buffer():
    """Overwrite the captured camera buffer with another pose: the replay renders that pose,
    equal to an eager step on it and to the oracle."""
    sc, poses = _scene_and_poses()
    W, H = poses[0]["width"], poses[0]["height"]
    target = synth.target_image(6, W, H)
    st = Step(sc, poses[0], target)
    g = ta.capture(st, warmup=1)
    st.d_cams.copy_(ta.cameras_device([poses[1]]))
    st.poison()
    g.replay()
    replayed = st.snapshot()
    ref = Step(sc, poses[1], target)
    ref()
    eager = ref.snapshot()
    assert_same_step(replayed, eager)
    o, _, _ = check_against_oracle(sc, poses[1], target, replayed)
    check_keys(st, o)
