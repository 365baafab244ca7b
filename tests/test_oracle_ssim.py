"""Pins of the SSIM oracle behind Eq. 3 (B1 pose assignment): identity and symmetry, a closed
form for constant images with the zero padding of the window, and the windowed moments
computed by scipy's Gaussian filter (11 taps of sigma 1.5, zero outside the image)."""
import numpy as np
from scipy import ndimage

import oracle

C1, C2 = 0.01 ** 2, 0.03 ** 2


def test_identity_and_symmetry():
    rng = np.random.default_rng(0)
    a = rng.uniform(size=(3, 33, 47)).astype(np.float32)
    b = np.clip(a + rng.normal(0, 0.05, size=a.shape), 0, 1).astype(np.float32)
    assert abs(oracle.ssim(a, a) - 1.0) < 1e-12
    assert abs(oracle.ssim(a, b) - oracle.ssim(b, a)) < 1e-12
    assert 0.5 < oracle.ssim(a, b) < 1.0


def test_constant_images_closed_form_with_zero_padding():
    # a = c1, b = c2 everywhere: with s the window mass inside the image at a pixel,
    # mu = c s, var = c^2 s (1 - s), cov = c1 c2 s (1 - s); s is a product of 1D partial sums
    c1, c2, H, W = 0.3, 0.7, 20, 26
    a = np.full((1, H, W), c1, np.float32)
    b = np.full((1, H, W), c2, np.float32)
    g = np.exp(-((np.arange(11) - 5.0) ** 2) / (2 * 1.5 ** 2))
    g /= g.sum()
    sx = np.array([g[max(0, 5 - x):min(11, W + 5 - x)].sum() for x in range(W)])
    sy = np.array([g[max(0, 5 - y):min(11, H + 5 - y)].sum() for y in range(H)])
    s = sy[:, None] * sx[None, :]
    a32, b32 = np.float64(np.float32(c1)), np.float64(np.float32(c2))
    ma, mb = a32 * s, b32 * s
    va, vb, cv = a32 ** 2 * s * (1 - s), b32 ** 2 * s * (1 - s), a32 * b32 * s * (1 - s)
    want = ((2 * ma * mb + C1) * (2 * cv + C2)) / ((ma ** 2 + mb ** 2 + C1) * (va + vb + C2))
    v, m = oracle.ssim(a, b, with_map=True)
    np.testing.assert_allclose(m, want, rtol=1e-12, atol=1e-14)
    # the interior value: luminance term only
    assert abs(m[10, 13] - (2 * a32 * b32 + C1) / (a32 ** 2 + b32 ** 2 + C1)) < 1e-12


def test_window_moments_match_scipy_gaussian_filter():
    rng = np.random.default_rng(3)
    a = rng.uniform(size=(2, 29, 31)).astype(np.float32)
    b = (0.5 * a + 0.5 * rng.uniform(size=a.shape)).astype(np.float32)
    f = lambda x: ndimage.gaussian_filter(x, 1.5, truncate=5 / 1.5, mode="constant", cval=0.0)
    maps = []
    for c in range(2):
        A, B = a[c].astype(np.float64), b[c].astype(np.float64)
        ma, mb = f(A), f(B)
        va, vb, cv = f(A * A) - ma ** 2, f(B * B) - mb ** 2, f(A * B) - ma * mb
        maps.append(((2 * ma * mb + C1) * (2 * cv + C2)) / ((ma ** 2 + mb ** 2 + C1) * (va + vb + C2)))
    want = np.mean(maps, axis=0)
    v, m = oracle.ssim(a, b, with_map=True)
    np.testing.assert_allclose(m, want, rtol=0, atol=1e-12)
    assert abs(v - want.mean()) < 1e-12


def test_pose_assignment_b1_threshold():
    rng = np.random.default_rng(4)
    full = rng.uniform(size=(3, 24, 24)).astype(np.float32)
    same = full.copy()
    changed = full.copy()
    changed[:, 4:20, 4:20] = 0.0
    b1 = oracle.pose_assign_b1(full, [same, changed], eps=0.05)
    np.testing.assert_array_equal(b1, [False, True])
    assert not oracle.pose_assign_b1(full, [changed], eps=1.0)[0]
