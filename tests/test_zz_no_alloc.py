"""The allocation-free entry point cgs_render_forward_static, for callers that cannot call
cudaMalloc or keep a workspace (an application that owns all device memory and forbids
allocation in its frame loop, or a plugin handed only its inputs and outputs).  Its output
must match the workspace-based cgs_render_forward on two calls in a row; the shared static
array is reused by the second call.  Collected last on purpose."""
import numpy as np
import pytest
import torch

from paper_2404_01133_b300 import cgs, synth
from paper_2404_01133_b300 import torch_api as ta
from gpu_common import PIX_ATOL, gpu_render

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2404_01133_b300 import build
    build.build()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("tile", [16, 8])
def test_static_forward_matches_workspace_forward_twice(tile):
    sc, cams = synth.workload_small()
    cam = cams[0]
    ref = gpu_render(sc, cams, tile=tile)
    assert ref["status"] == cgs.CGS_OK
    ds, cfg, d_cam = ref["ds"], ref["cfg"], ref["cams"]
    W, H = cam["width"], cam["height"]
    for _ in range(2):
        img = torch.full((1, 3, H, W), -1.0, device="cuda")
        T = torch.full((1, H, W), -1.0, device="cuda")
        nc = torch.full((1, H, W), -1, dtype=torch.int32, device="cuda")
        status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        rc = cgs.cgs_render_forward_static(ds.struct(), cfg, d_cam, W, H, None, None, img, T, nc, status)
        assert rc == cgs.CGS_OK, cgs.cgs_status_string(rc)
        torch.cuda.synchronize()
        assert int(status.item()) == cgs.CGS_OK
        assert (img - ref["image"]).abs().max().item() <= PIX_ATOL
        assert (T - ref["final_T"]).abs().max().item() <= PIX_ATOL
        assert torch.equal(nc, ref["n_contrib"])


def test_static_forward_rejects_requests_beyond_its_limits():
    sc, cams = synth.workload_small()
    ref = gpu_render(sc, cams)
    ds, cfg, d_cam = ref["ds"], ref["cfg"], ref["cams"]
    img = torch.empty((1, 3, 600, 600), device="cuda")
    T = torch.empty((1, 600, 600), device="cuda")
    nc = torch.empty((1, 600, 600), dtype=torch.int32, device="cuda")
    rc = cgs.cgs_render_forward_static(ds.struct(), cfg, d_cam, 600, 600, None, None, img, T, nc)
    assert rc == cgs.CGS_ERR_TOO_LARGE
    assert "limits" in cgs.cgs_status_string(rc)
