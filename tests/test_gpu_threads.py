"""Forward renders issued concurrently from several host threads, each on its own stream and
frame workspace, equal the same render issued from one thread.  The forward runs its long-tile
sort on a side stream the library keeps per host thread and device, forked from the caller's
stream after the entries are binned and joined back before compositing (the depth sort of
Sec. 3.1's rasterizer); a side stream or event shared between threads would let one thread's
long-tile sort start before its own entries are binned, or its compositing before its sort
ends.  The scene puts tiles on both sides of the long-tile bound (256 entries), so both sort
kernels have work."""
import threading

import numpy as np
import pytest
import torch

from paper_2404_01133_b300 import cgs, synth
from paper_2404_01133_b300 import torch_api as ta

pytestmark = pytest.mark.gpu

N_THREADS = 4
ROUNDS = 12


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2404_01133_b300 import build
    build.build()
    assert torch.cuda.is_available()


def _scene():
    # a dense cluster (tiles of thousands of entries) inside a sparse cube (short tiles)
    sc = synth.random_cube_scene(6000, seed=41, sh_degree=1, log_scale_mu=-2.6)
    sc["mean_opac"][:3000, :3] *= np.float32(0.12)
    return synth.single_block(sc), synth.small_scene_camera(96, 80, f=90.0, dist=3.0)


def _render(ds, cam, stream):
    cfg = ta.make_config(tile=16, batch=128)
    with torch.cuda.stream(stream):  # the workspace is zero-filled and the camera copied on this stream
        fr = ta.Frame(1, cam["width"], cam["height"], 16, ds.n_blocks, ds.n, 400 * ds.n)
        img, T, nc = ta.render_forward(ds, fr, cfg, ta.cameras_device([cam]), stream=stream)
    stream.synchronize()
    st, counts = fr.status()
    vals = fr.buffer(cgs.BUF_TILE_VALS, torch.int32, count=int(counts[2])).cpu().numpy()
    return st, img.cpu().numpy(), nc.cpu().numpy(), vals


def test_concurrent_host_threads_equal_one_thread():
    sc, cam = _scene()
    ds = ta.DeviceScene(sc)
    torch.cuda.synchronize()
    ref_st, ref_img, ref_nc, ref_vals = _render(ds, cam, torch.cuda.Stream())
    assert ref_st == 0
    # the scene has long tiles (the side-stream kernel has work) and short ones
    cfg = ta.make_config(tile=16, batch=128)
    fr = ta.Frame(1, cam["width"], cam["height"], 16, ds.n_blocks, ds.n, 400 * ds.n)
    ta.render_forward(ds, fr, cfg, ta.cameras_device([cam]))
    torch.cuda.synchronize()
    tiles = ((cam["width"] + 15) // 16) * ((cam["height"] + 15) // 16)
    ranges = fr.buffer(cgs.BUF_RANGES, torch.int32, (2,), count=tiles).cpu().numpy()
    lengths = ranges[:, 1] - ranges[:, 0]
    assert lengths.max() > 256 and ((lengths > 0) & (lengths <= 256)).any()

    results, errors = [], []

    def worker():
        try:
            s = torch.cuda.Stream()
            for _ in range(ROUNDS):
                results.append(_render(ds, cam, s))
        except Exception as e:  # reported by the main thread
            errors.append(repr(e))

    threads = [threading.Thread(target=worker) for _ in range(N_THREADS)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    assert len(results) == N_THREADS * ROUNDS
    for st, img, nc, vals in results:
        assert st == 0
        np.testing.assert_array_equal(vals, ref_vals)
        np.testing.assert_array_equal(nc, ref_nc)
        np.testing.assert_array_equal(img, ref_img)
