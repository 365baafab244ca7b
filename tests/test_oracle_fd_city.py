"""Finite-difference pin of the oracle's analytic gradient (differentiable rendering, Sec. 3.1)
at the scale of the 1920x1080, 1M-Gaussian SH-3 city workload: 64 random visible Gaussians of
that frame, the L1 loss against its seeded target (its gradient sign(img - target) / count
taken at the base point, so the check is of the vector-Jacobian product the backward
computes).  Each Gaussian's render is restricted to its own tiles and to the Gaussians binned
to them, which reproduces those tiles' pixels exactly; no other pixel depends on it (a
perturbation that changes its tile rect changes the decision signature and is rejected).
Central differences of the FP64 oracle; a sample is rejected when any discrete decision
differs between the +h and -h renders.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_2404_01133_b300 import synth

N_GAUSSIANS = 64
SH_SAMPLES = 6  # SH coefficients per Gaussian beyond the three DC ones (random, seeded)


@pytest.fixture(scope="module")
def city():
    sc, cams = synth.workload_city_1m()
    cam = cams[0]
    pr = oracle.project(sc, cam, real="f64")
    return sc, cam, pr


def _signature(out):
    pr = out["proj"]
    return (out["hash"], pr["flags"].tobytes(), pr["rect"].tobytes())


def test_fd_on_64_visible_gaussians_of_the_1080p_city(city):
    sc, cam, pr = city
    W, H = cam["width"], cam["height"]
    tx, ty = (W + 15) // 16, (H + 15) // 16
    tt = pr["tiles_touched"]
    rect = pr["rect"]
    # random visible Gaussians; ones wider than 64 tiles are left to the small-scene pins
    # (their neighbourhoods hold tens of thousands of Gaussians)
    cand = np.flatnonzero((tt > 0) & (tt <= 64))
    pick = np.random.default_rng(2024).choice(cand, size=N_GAUSSIANS, replace=False)
    target = synth.target_image(1, W, H)
    count = 3 * W * H
    cfg = oracle.make_config(tile=16)
    checked = rejected = 0
    worst = 0.0
    for gi, g in enumerate(pick):
        x0, y0, x1, y1 = (int(v) for v in rect[g])
        mask = np.zeros((ty, tx), np.uint8)
        mask[y0:y1, x0:x1] = 1
        # every Gaussian binned to a tile of the mask, in scene order (depth ties break by index)
        hit = (rect[:, 0] < x1) & (rect[:, 2] > x0) & (rect[:, 1] < y1) & (rect[:, 3] > y0) & (tt > 0)
        idx = np.flatnonzero(hit)
        me = int(np.searchsorted(idx, g))
        assert idx[me] == g
        sub = {k: np.array(sc[k][idx], dtype=np.float64) for k in ("mean_opac", "scale", "quat", "sh")}
        sub["sh_degree"] = sc["sh_degree"]
        base = oracle.render(sub, cam, cfg, real="f64", tile_mask=mask.reshape(-1))
        # the L1 loss's upstream gradient at the base point, on the mask's pixels
        pix = np.repeat(np.repeat(mask, 16, axis=0), 16, axis=1)[:H, :W].astype(bool)
        w = np.sign(base["image"] - target) / count
        w[:, ~pix] = 0.0
        g_an = oracle.render_backward(sub, cam, w, cfg, real="f64", fwd=base, tile_mask=mask.reshape(-1))
        an = {"mean_opac": np.concatenate([g_an["mean"][me], [g_an["opac"][me]]]), "scale": g_an["scale"][me],
              "quat": g_an["quat"][me], "sh": g_an["sh"][me]}
        gmax = max(max(np.abs(v).max() for v in an.values()), 1e-30)
        r = np.random.default_rng(1000 + gi)
        sh_ix = [(0, c) for c in range(3)] + [(int(k), int(c)) for k, c in
                                               zip(r.integers(1, sub["sh"].shape[1], SH_SAMPLES),
                                                   r.integers(0, 3, SH_SAMPLES))]
        samples = [("mean_opac", (a,)) for a in range(4)] + [("scale", (a,)) for a in range(3)] + \
                  [("quat", (a,)) for a in range(4)] + [("sh", ix) for ix in sh_ix]
        for name, ix in samples:
            full = (me,) + ix
            x = sub[name][full]
            h = 1e-6 * max(abs(x), 0.05)
            sp = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in sub.items()}
            sp[name][full] = x + h
            op = oracle.render(sp, cam, cfg, real="f64", tile_mask=mask.reshape(-1))
            sp[name][full] = x - h
            om = oracle.render(sp, cam, cfg, real="f64", tile_mask=mask.reshape(-1))
            if _signature(op) != _signature(om):
                rejected += 1
                continue
            fd = float(((op["image"] - om["image"]) * w).sum()) / (2 * h)
            ref = float(an[name][ix])
            tol = 1e-5 * abs(ref) + 1e-7 * gmax
            worst = max(worst, abs(fd - ref) / tol)
            assert abs(fd - ref) <= tol, (int(g), name, ix, fd, ref)
            checked += 1
    total = checked + rejected
    assert checked >= 0.8 * total, (checked, rejected)
    print(f"[fd 1080p city] {N_GAUSSIANS} Gaussians, {checked} samples checked, {rejected} rejected "
          f"(a decision changed), worst error {worst:.2f} of the tolerance")
