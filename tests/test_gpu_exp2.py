"""The falloff exponential of the compositing kernels (Eq. 1's exp, evaluated as 2^p by the
hardware base-2 exponential) measured against exact values: the oracle's ambiguity margins
assume its relative error is at most 2^-21 wherever the result is a normal FP32 number; this
test pins that assumption on the device the parity tests run on."""
import numpy as np
import pytest
import torch

from paper_2404_01133_b300 import cgs

pytestmark = pytest.mark.gpu

EXP2_REL_ASSUMED = 2.0 ** -21  # AMB_EXP2_REL in oracle.c


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2404_01133_b300 import build
    build.build()
    assert torch.cuda.is_available()


def device_exp2(p):
    d_p = torch.as_tensor(p, dtype=torch.float32).cuda().contiguous()
    d_g = torch.empty_like(d_p)
    cgs.cgs_debug_exp2(d_p, d_p.numel(), d_g)
    torch.cuda.synchronize()
    return d_g.cpu().numpy()


def test_exp2_relative_error_within_the_assumed_bound():
    rng = np.random.default_rng(0)
    # every FP32 value in [-1, 0] spaced 2^-20 apart, a dense grid over [-126, 0] (the powers of
    # Eq. 1 are never positive), random points, and the integers
    p = np.concatenate([
        np.arange(-(1 << 20), 1, dtype=np.int64).astype(np.float64) / (1 << 20),
        np.linspace(-126.0, 0.0, 1 << 22),
        rng.uniform(-126.0, 0.0, size=1 << 21),
        np.arange(-126, 1, dtype=np.float64),
    ]).astype(np.float32)
    g = device_exp2(p).astype(np.float64)
    exact = np.exp2(p.astype(np.float64))
    rel = np.abs(g - exact) / exact
    worst = float(rel.max())
    print(f"[exp2] {p.size} points in [-126, 0]: max relative error {worst:.3e} "
          f"({worst / 2.0 ** -23:.2f} FP32 ulp-equivalents), assumed bound {EXP2_REL_ASSUMED:.3e}")
    assert worst <= EXP2_REL_ASSUMED


def test_exp2_results_below_the_normal_range_are_zero_or_tiny():
    """Results that would be subnormal are flushed to zero: o * 2^p is then below 1/255 on any
    evaluation, so the skip decision cannot depend on it."""
    p = np.linspace(-160.0, -126.5, 4096).astype(np.float32)
    g = device_exp2(p)
    assert np.all((g == 0.0) | (np.abs(g) < 2.0 ** -125))
