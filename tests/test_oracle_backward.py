"""Pins of the oracle's analytic gradient (differentiable rendering, Sec. 3.1) against
central finite differences of its own FP64 forward.  A sample is rejected when any
discrete decision (cull, guard-band clamp, colour clamp, tile rect, skip/stop/opacity
clamp of any pixel) differs between the +h and -h renders.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_2404_01133_b300 import synth


def fd_scene(seed, n=10, deg=3):
    r = np.random.default_rng(seed)
    mo = np.zeros((n, 4))
    mo[:, 0] = r.uniform(-0.5, 0.5, n)
    mo[:, 1] = r.uniform(-0.4, 0.4, n)
    mo[:, 2] = r.uniform(-0.5, 0.5, n)
    mo[:, 3] = r.uniform(0.3, 0.9, n)
    sc = np.zeros((n, 4))
    sc[:, :3] = np.exp(r.normal(-2.3, 0.4, size=(n, 3)))
    q = r.normal(size=(n, 4))
    nc = (deg + 1) ** 2
    sh = r.normal(0, 0.3, size=(n, nc, 3))
    sh[:, 0, :] = r.uniform(-1.5, 1.5, size=(n, 3))
    return {"mean_opac": mo, "scale": sc, "quat": q, "sh": sh, "sh_degree": deg}


def fd_scene_edges():
    """Adds a large Gaussian beyond the 1.3x guard band that still reaches the image, and
    an almost opaque one whose centre pixels hit the 0.99 opacity clamp."""
    sc = fd_scene(2, n=8)
    sc["mean_opac"][0, :3] = (1.8, 0.1, 0.0)     # tx/tz = 0.6 > 1.3 * 24/60
    sc["scale"][0, :3] = (0.5, 0.4, 0.45)
    sc["mean_opac"][1, :3] = (0.0225, 0.0225, -0.3)  # projects onto the pixel centre (24, 20)
    sc["mean_opac"][1, 3] = 0.995
    sc["scale"][1, :3] = (0.08, 0.07, 0.06)
    return sc


PARAMS = [("mean_opac", a) for a in range(3)] + [("mean_opac", 3)] + [("scale", a) for a in range(3)] + \
         [("quat", a) for a in range(4)]


def signature(out):
    pr = out["proj"]
    return (out["hash"], pr["flags"].tobytes(), pr["rect"].tobytes())


def loss_of(scene, cam, w, cfg):
    out = oracle.render(scene, cam, cfg, real="f64")
    return float((out["image"] * w).sum()), signature(out)


@pytest.mark.parametrize("seed", [0, 1, "edges"])
def test_analytic_gradient_matches_central_differences(seed):
    sc = fd_scene(seed) if seed != "edges" else fd_scene_edges()
    cam = synth.small_scene_camera(48, 40, f=60.0, dist=3.0)
    cfg = oracle.make_config(tile=16)
    w = np.random.default_rng(100 + (seed if seed != "edges" else 2)).normal(size=(3, 40, 48))
    g = oracle.render_backward(sc, cam, w, cfg, real="f64")
    if seed == "edges":
        assert g["fwd"]["proj"]["flags"][0] & oracle.F_CLAMP_X and g["fwd"]["proj"]["tiles_touched"][0] > 0
        pr = g["fwd"]["proj"]
        u, v = pr["xy"][1]
        c = pr["conic"][1]
        jj, ii = np.mgrid[0:40, 0:48]
        dx, dy = u - ii, v - jj
        pw = -0.5 * (c[0] * dx * dx + c[2] * dy * dy) - c[1] * dx * dy
        assert (sc["mean_opac"][1, 3] * np.exp(pw) > 0.99).any()
    an = {"mean_opac": np.concatenate([g["mean"], g["opac"][:, None]], axis=1), "scale": g["scale"],
          "quat": g["quat"], "sh": g["sh"]}
    n = sc["mean_opac"].shape[0]
    checked = rejected = 0
    worst = 0.0
    samples = []
    for i in range(n):
        for name, a in PARAMS:
            samples.append((name, (i, a)))
        for k in range(sc["sh"].shape[1]):
            for ch in range(3):
                samples.append(("sh", (i, k, ch)))
    gmax = {k: max(np.abs(v).max(), 1e-30) for k, v in an.items()}
    for name, ix in samples:
        x0 = sc[name][ix]
        h = 1e-6 * max(abs(x0), 0.05)
        sp = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
        sp[name][ix] = x0 + h
        lp, sig_p = loss_of(sp, cam, w, cfg)
        sp[name][ix] = x0 - h
        lm, sig_m = loss_of(sp, cam, w, cfg)
        if sig_p != sig_m:
            rejected += 1
            continue
        fd = (lp - lm) / (2 * h)
        ref = an[name][ix]
        err = abs(fd - ref)
        tol = 1e-5 * abs(ref) + 1e-7 * gmax[name]
        worst = max(worst, err / tol)
        assert err <= tol, (name, ix, fd, ref)
        checked += 1
    assert checked > 0.8 * len(samples), (checked, rejected)
    assert worst <= 1.0


def test_f32_gradient_close_to_f64():
    sc = fd_scene(3, n=40)
    cam = synth.small_scene_camera(64, 48, f=70.0, dist=3.0)
    w = np.random.default_rng(7).normal(size=(3, 48, 64))
    g64 = oracle.render_backward(sc, cam, w, real="f64")
    g32 = oracle.render_backward(sc, cam, w, real="f32")
    f64, f32 = g64["fwd"], g32["fwd"]
    # compare only when the two builds took the same compositing decisions
    assert f64["hash"] == f32["hash"]
    for k in ("mean", "scale", "quat", "opac", "sh"):
        a, b = g32[k].astype(np.float64), g64[k]
        assert np.linalg.norm(a - b) <= 1e-4 * np.linalg.norm(b), k
