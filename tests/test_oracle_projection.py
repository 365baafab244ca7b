"""Pins of the oracle's projection (Eq. 1's proj, Sec. 3.1) against closed forms, finite
differences of the perspective map, a library rotation, brute-force pixel enumeration and
a library spherical-harmonics routine.  CPU only."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2404_01133_b300 import synth


def make_scene(means, scales, quats, opac, sh=None, deg=0):
    n = len(means)
    mo = np.zeros((n, 4), np.float64)
    mo[:, :3] = means
    mo[:, 3] = opac
    sc = np.zeros((n, 4), np.float64)
    sc[:, :3] = scales
    if sh is None:
        sh = np.zeros((n, (deg + 1) ** 2, 3))
    return {"mean_opac": mo, "scale": sc, "quat": np.asarray(quats, np.float64), "sh": np.asarray(sh, np.float64),
            "sh_degree": deg}


def screen_map(cam, p):
    R = cam["R"].astype(np.float64)
    t = cam["t"].astype(np.float64)
    x = R @ p + t
    return np.array([cam["fx"] * x[0] / x[2] + cam["cx"], cam["fy"] * x[1] / x[2] + cam["cy"]])


def fd_jacobian(cam, p):
    J = np.zeros((2, 3))
    for a in range(3):
        h = 1e-5 * max(1.0, abs(p[a]))
        e = np.zeros(3)
        e[a] = h
        J[:, a] = (screen_map(cam, p + e) - screen_map(cam, p - e)) / (2 * h)
    return J


def test_isotropic_on_axis_closed_form():
    cam = synth.small_scene_camera(64, 64, f=150.0, dist=4.0)
    s = 0.05
    sc = make_scene([[0, 0, 0]], [[s, s, s]], [[1, 0, 0, 0]], [0.5])
    pr = oracle.project(sc, cam, real="f64")
    sig2 = (150.0 * s / 4.0) ** 2 + 0.3
    np.testing.assert_allclose(pr["cov2d"][0], [sig2, 0.0, sig2], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(pr["conic"][0], [1 / sig2, 0.0, 1 / sig2], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(pr["xy"][0], [cam["cx"], cam["cy"]], rtol=0, atol=1e-12)


def test_sigma2d_matches_fd_jacobian_and_library_rotation(rng):
    cam = synth.look_at((3.0, -2.0, -6.0), (0.1, 0.2, 0.0), (0, -1, 0), 300.0, 280.0, 160, 120)
    n = 40
    means = rng.uniform(-0.6, 0.6, size=(n, 3))
    scales = np.exp(rng.normal(-2.0, 0.5, size=(n, 3)))
    q = rng.normal(size=(n, 4))
    sc = make_scene(means, scales, q, np.full(n, 0.5))
    pr = oracle.project(sc, cam, real="f64")
    for i in range(n):
        assert pr["flags"][i] & (oracle.F_CLAMP_X | oracle.F_CLAMP_Y) == 0
        Rm = Rotation.from_quat([q[i, 1], q[i, 2], q[i, 3], q[i, 0]]).as_matrix()
        S3 = Rm @ np.diag(scales[i] ** 2) @ Rm.T
        J = fd_jacobian(cam, means[i])
        S2 = J @ S3 @ J.T
        got = pr["cov2d"][i]
        np.testing.assert_allclose([got[0] - 0.3, got[1], got[2] - 0.3], [S2[0, 0], S2[0, 1], S2[1, 1]],
                                   rtol=1e-6, atol=1e-9 * abs(S2).max())
        np.testing.assert_allclose(pr["xy"][i], screen_map(cam, means[i]), rtol=1e-12, atol=1e-9)
        inv = np.linalg.inv(np.array([[got[0], got[1]], [got[1], got[2]]]))
        np.testing.assert_allclose(pr["conic"][i], [inv[0, 0], inv[0, 1], inv[1, 1]], rtol=1e-9)


def test_guard_band_only_changes_offscreen():
    # A Gaussian far outside the field of view gets the clamp flag; an on-screen one does not.
    cam = synth.small_scene_camera(64, 64, f=100.0, dist=4.0)
    sc = make_scene([[0.2, 0.1, 0.0], [30.0, 0.0, 0.0]], [[0.05] * 3] * 2, [[1, 0, 0, 0]] * 2, [0.5, 0.5])
    pr = oracle.project(sc, cam, real="f64")
    assert pr["flags"][0] & oracle.F_CLAMP_X == 0
    assert pr["flags"][1] & oracle.F_CLAMP_X
    assert pr["tiles_touched"][1] == 0


def test_near_plane_cull():
    cam = synth.small_scene_camera(64, 64, f=100.0, dist=4.0)
    # camera z = world z + 4: world z -3.9 -> 0.1 (culled), -3.8 -> 0.2 (culled: tz <= near), -3.7 kept
    sc = make_scene([[0, 0, -3.9], [0, 0, -3.8], [0, 0, -3.7]], [[0.01] * 3] * 3, [[1, 0, 0, 0]] * 3, [0.5] * 3)
    pr = oracle.project(sc, cam, real="f32")
    tz = np.float32(-3.8) + np.float32(4.0)
    assert pr["flags"][0] & oracle.F_CULL_NEAR
    assert bool(pr["flags"][1] & oracle.F_CULL_NEAR) == bool(tz <= np.float32(0.2))
    assert pr["flags"][2] & oracle.F_CULL_NEAR == 0
    assert pr["tiles_touched"][0] == 0


@pytest.mark.parametrize("tile", [16, 8])
def test_radius_and_rect_by_brute_force(tile):
    sc, cams = synth.workload_small()
    cam = cams[0]
    pr = oracle.project(sc, cam, oracle.make_config(tile=tile), real="f32")
    W, H = cam["width"], cam["height"]
    tx_n = (W + tile - 1) // tile
    checked = 0
    for i in np.flatnonzero((pr["flags"] & 3) == 0):
        A, B, Cc = (float(v) for v in pr["cov2d"][i])
        lam = np.linalg.eigvalsh(np.array([[A, B], [B, Cc]]))[1]
        r = int(pr["radius"][i])
        assert r >= 3.0 * math.sqrt(lam) * (1 - 1e-6)
        assert r <= 3.0 * math.sqrt(lam + 0.33) + 1
        u, v = float(pr["xy"][i, 0]), float(pr["xy"][i, 1])
        xs = [x for x in range(W) if abs(x - u) <= r]
        ys = [y for y in range(H) if abs(y - v) <= r]
        if not xs or not ys:
            assert pr["tiles_touched"][i] == 0
            continue
        tiles = {(y // tile) * tx_n + x // tile for x in xs for y in ys}
        x0, y0, x1, y1 = pr["rect"][i]
        got = {ty * tx_n + tx for ty in range(y0, y1) for tx in range(x0, x1)}
        assert got == tiles
        assert pr["tiles_touched"][i] == len(tiles)
        checked += 1
    assert checked > 1000


def real_sh_scipy(l, m, theta, phi):
    from scipy.special import sph_harm_y
    if m == 0:
        return sph_harm_y(l, 0, theta, phi).real
    y = sph_harm_y(l, abs(m), theta, phi)
    return math.sqrt(2.0) * (y.real if m > 0 else y.imag)


def test_sh_basis_matches_library(rng):
    d = rng.normal(size=(200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = oracle.sh_basis(d, 3)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    for l in range(4):
        for m in range(-l, l + 1):
            ref = real_sh_scipy(l, m, theta, phi)
            np.testing.assert_allclose(Y[:, l * l + l + m], ref, rtol=1e-10, atol=1e-12)


def test_sh_basis_orthonormal_by_quadrature():
    xg, wg = np.polynomial.legendre.leggauss(24)
    nphi = 48
    phi = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    ct, ph = np.meshgrid(xg, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    d = np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=-1).reshape(-1, 3)
    w = (wg[:, None] * np.full(nphi, 2 * np.pi / nphi)[None, :]).reshape(-1)
    Y = oracle.sh_basis(d, 3)
    G = (Y * w[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_basis_derivative_fd(rng):
    p = rng.normal(size=(20, 3))
    Y, dY = oracle.sh_basis(p, 3, with_grad=True)
    h = 1e-6
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        fd = (oracle.sh_basis(p + e, 3) - oracle.sh_basis(p - e, 3)) / (2 * h)
        np.testing.assert_allclose(dY[:, :, a], fd, rtol=1e-7, atol=1e-8)


def test_degree0_colour_is_base_colour():
    sc, cams = synth.workload_small()
    pr = oracle.project(sc, cams[0], real="f64")
    vis = (pr["flags"] & 3) == 0
    f0 = sc["sh"][:, 0, :].astype(np.float64)
    # the DC basis function is 1 / (2 sqrt(pi)); the generator stored (c - 0.5) * 2 sqrt(pi)
    np.testing.assert_allclose(pr["rgb"][vis], np.clip(f0[vis] / (2 * math.sqrt(math.pi)) + 0.5, 0, None),
                               rtol=1e-12, atol=1e-12)


def test_f32_and_f64_builds_agree_on_values():
    sc, cams = synth.workload_small()
    a = oracle.project(sc, cams[0], real="f32")
    b = oracle.project(sc, cams[0], real="f64")
    np.testing.assert_array_equal(a["rect"], b["rect"])
    np.testing.assert_array_equal(a["depth"], b["depth"])
    vis = a["tiles_touched"] > 0
    np.testing.assert_allclose(a["xy"][vis], b["xy"][vis], rtol=1e-6, atol=1e-4)
    np.testing.assert_allclose(a["conic"][vis], b["conic"][vis], rtol=2e-5, atol=1e-6)
    np.testing.assert_allclose(a["rgb"][vis], b["rgb"][vis], rtol=1e-5, atol=1e-6)
