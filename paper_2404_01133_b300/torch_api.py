"""Torch-facing helpers around the C ABI: device scenes, frames (workspaces), cameras and a
``torch.autograd.Function`` whose forward and backward are the library's kernels.

PyTorch only provides device memory and streams here; all rendering work is done by
libcgs.so through :mod:`paper_2404_01133_b300.cgs`.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import cgs as _c


def camera_struct(cam):
    s = _c.cgs_camera()
    s.R[:] = [float(v) for v in np.asarray(cam["R"], np.float32).reshape(9)]
    s.t[:] = [float(v) for v in np.asarray(cam["t"], np.float32).reshape(3)]
    s.campos[:] = [float(v) for v in np.asarray(cam["campos"], np.float32).reshape(3)]
    s.fx, s.fy, s.cx, s.cy = cam["fx"], cam["fy"], cam["cx"], cam["cy"]
    s.width, s.height = cam["width"], cam["height"]
    return s


def cameras_host(cams):
    """Pinned host uint8 tensor holding the packed cgs_camera array."""
    arr = (_c.cgs_camera * len(cams))(*[camera_struct(c) for c in cams])
    t = torch.frombuffer(bytearray(bytes(arr)), dtype=torch.uint8).clone()
    return t.pin_memory() if torch.cuda.is_available() else t


def cameras_device(cams, device="cuda"):
    return cameras_host(cams).to(device, non_blocking=False)


def make_config(tile=16, batch=None, near_z=0.2, bg=(0.0, 0.0, 0.0), lod_dist=(200.0, 600.0), lod_mode=0,
                exact=False):
    """exact=True selects the compositing kernels' parity build (cgs_config.exact)."""
    c = _c.cgs_config()
    c.lod_mode = lod_mode
    c.exact = 1 if exact else 0
    c.tile = tile
    c.batch = batch if batch is not None else (256 if tile == 16 else 64)
    c.near_z = near_z
    c.bg[:] = list(bg)
    c.lod_dist[:] = list(lod_dist)
    return c


class DeviceScene:
    """A synth-format scene uploaded to the device, with its cgs_scene descriptor."""

    def __init__(self, scene, device="cuda", attrs=None, fp16=False):
        dev = torch.device(device)
        self.attr_fp16 = 1 if fp16 else 0
        if attrs is None:
            attrs = {k: torch.from_numpy(np.ascontiguousarray(scene[k], np.float32)).to(dev)
                     for k in ("mean_opac", "scale", "quat", "sh")}
            if fp16:
                for k in ("scale", "quat", "sh"):
                    attrs[k] = attrs[k].to(torch.float16).contiguous()
        self.mean_opac, self.scale, self.quat, self.sh = (attrs["mean_opac"], attrs["scale"], attrs["quat"],
                                                          attrs["sh"])
        self.sh_degree = int(scene["sh_degree"])
        lo = np.ascontiguousarray(scene["level_offset"], np.int64)
        lc = np.ascontiguousarray(scene["level_count"], np.int64)
        self.n_blocks, self.n_levels = lo.shape
        self.level_offset = torch.from_numpy(lo).to(dev)
        self.level_count = torch.from_numpy(lc).to(dev)
        self.block_cell = torch.from_numpy(np.ascontiguousarray(scene["block_cell"], np.float32)).to(dev)
        self.block_aabb = torch.zeros((self.n_blocks, 6), dtype=torch.float32, device=dev)
        self.n = int(self.mean_opac.shape[0])
        self.device = dev

    def struct(self, attrs=None):
        a = attrs or {}
        s = _c.cgs_scene()
        s.mean_opac = a.get("mean_opac", self.mean_opac).data_ptr()
        s.scale = a.get("scale", self.scale).data_ptr()
        s.quat = a.get("quat", self.quat).data_ptr()
        s.sh = a.get("sh", self.sh).data_ptr()
        s.n = self.n
        s.sh_degree = self.sh_degree
        s.n_blocks = self.n_blocks
        s.n_levels = self.n_levels
        s.attr_fp16 = self.attr_fp16
        s.level_offset = self.level_offset.data_ptr()
        s.level_count = self.level_count.data_ptr()
        s.block_aabb = self.block_aabb.data_ptr()
        s.block_cell = self.block_cell.data_ptr()
        return s

    def compute_block_bounds(self, n_mad=4.0, stream=None):
        """Eq. 7 MAD bounds of every block, written into self.block_aabb by the library."""
        _c.cgs_block_bounds(self.struct(), n_mad, self.block_aabb, None, 0, stream)
        return self.block_aabb


class UploadedScene:
    """A synth-format scene uploaded by the library (cgs_scene_upload) into one device buffer
    from torch; same interface as DeviceScene for rendering (struct(), n, n_blocks, ...)."""

    def __init__(self, scene, device="cuda", n_mad=-1.0, fp16=False, stream=None):
        dev = torch.device(device)
        self.attr_fp16 = 1 if fp16 else 0
        hdt = np.float16 if fp16 else np.float32
        self._host = {"mean_opac": np.ascontiguousarray(scene["mean_opac"], np.float32),
                      "scale": np.ascontiguousarray(scene["scale"], hdt), "quat": np.ascontiguousarray(scene["quat"], hdt),
                      "sh": np.ascontiguousarray(scene["sh"], hdt),
                      "level_offset": np.ascontiguousarray(scene["level_offset"], np.int64),
                      "level_count": np.ascontiguousarray(scene["level_count"], np.int64),
                      "block_cell": np.ascontiguousarray(scene["block_cell"], np.float32)}
        h = self._host
        self.n = int(h["mean_opac"].shape[0])
        self.sh_degree = int(scene["sh_degree"])
        self.n_blocks, self.n_levels = h["level_offset"].shape
        nbytes = _c.cgs_scene_bytes(self.n, self.sh_degree, self.n_blocks, self.n_levels, self.attr_fp16)
        if nbytes < 0:
            raise ValueError("invalid scene dimensions")
        self.mem = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self._s = _c.cgs_scene_upload(self.mem, nbytes, h["mean_opac"], h["scale"], h["quat"], h["sh"], self.n,
                                      self.sh_degree, self.attr_fp16, h["level_offset"], h["level_count"],
                                      h["block_cell"], n_mad, stream)
        torch.cuda.synchronize(dev)  # the host arrays may be released after the copies
        self.device = dev
        # tensor views of the uploaded attributes and bounds (inside self.mem)
        base = self.mem.data_ptr()
        adt = torch.float16 if fp16 else torch.float32
        nco = (self.sh_degree + 1) ** 2

        def view(ptr, dtype, shape):
            off = ptr - base
            cnt = int(np.prod(shape))
            elem = torch.tensor([], dtype=dtype).element_size()
            return self.mem[off:off + cnt * elem].view(dtype).view(shape)
        sc = self._s
        self.mean_opac = view(sc.mean_opac, torch.float32, (self.n, 4))
        self.scale = view(sc.scale, adt, (self.n, 4))
        self.quat = view(sc.quat, adt, (self.n, 4))
        self.sh = view(sc.sh, adt, (self.n, nco, 3))
        self.block_aabb = view(sc.block_aabb, torch.float32, (self.n_blocks, 6))

    def struct(self, attrs=None):
        if attrs:
            raise ValueError("an uploaded scene renders its own attributes")
        return self._s


class Frame:
    """Workspace of a batch of equally sized views (device memory from torch)."""

    def __init__(self, n_views, width, height, tile, n_blocks, n_cap, k_cap, device="cuda", count_pairs=True):
        nbytes = _c.cgs_frame_workspace_bytes(n_views, width, height, tile, n_blocks, n_cap, k_cap)
        if nbytes <= 0:
            raise ValueError("invalid frame dimensions")
        self.ws = torch.zeros(nbytes, dtype=torch.uint8, device=device)  # zero-filled once (cgs_frame)
        f = _c.cgs_frame()
        f.ws = self.ws.data_ptr()
        f.ws_bytes = nbytes
        f.n_views, f.width, f.height, f.tile, f.n_blocks = n_views, width, height, tile, n_blocks
        f.n_cap, f.k_cap = n_cap, k_cap
        f.flags = 0 if count_pairs else _c.CGS_FRAME_NO_PAIR_COUNT
        self.struct = f
        self.n_views, self.width, self.height, self.tile = n_views, width, height, tile
        self.n_cap, self.k_cap = n_cap, k_cap

    def outputs(self, device=None):
        dev = device or self.ws.device
        V, H, W = self.n_views, self.height, self.width
        return (torch.empty((V, 3, H, W), dtype=torch.float32, device=dev),
                torch.empty((V, H, W), dtype=torch.float32, device=dev),
                torch.empty((V, H, W), dtype=torch.int32, device=dev))

    def status(self, stream=None):
        return _c.cgs_frame_status(self.struct, stream)

    def buffer(self, which, dtype, shape_tail=(), count=None):
        """Copy of an internal array (see cgs_frame_buffer) as a torch tensor."""
        ptr, cap = _c.cgs_frame_buffer(self.struct, which)
        n = cap if count is None else count
        elem = torch.tensor([], dtype=dtype).element_size()
        width = int(np.prod(shape_tail)) if shape_tail else 1
        nbytes = n * width * elem
        off = ptr - self.ws.data_ptr()
        raw = self.ws[off:off + nbytes]
        return raw.view(dtype).reshape((n,) + tuple(shape_tail)).clone()


def render_forward(dscene, frame, cfg, d_cams, view_block=None, levels=None, out=None, attrs=None, stream=None):
    img, T, nc = out if out is not None else frame.outputs()
    _c.cgs_render_forward(dscene.struct(attrs), frame.struct, cfg, d_cams, view_block, levels, img, T, nc, stream)
    return img, T, nc


def render_backward(dscene, frame, cfg, d_cams, dL_dimage, final_T, n_contrib, grads=None, attrs=None, stream=None):
    if grads is None:
        f32 = torch.float32
        grads = (torch.zeros_like(dscene.mean_opac), torch.zeros_like(dscene.scale, dtype=f32),
                 torch.zeros_like(dscene.quat, dtype=f32), torch.zeros_like(dscene.sh, dtype=f32))
    g_mo, g_sc, g_q, g_sh = grads
    _c.cgs_render_backward(dscene.struct(attrs), frame.struct, cfg, d_cams, dL_dimage.contiguous(), final_T,
                           n_contrib, g_mo, g_sc, g_q, g_sh, stream)
    return grads


def render_backward_packed(dscene, frame, cfg, d_cams, dL_dimage, final_T, n_contrib, rows=None, attrs=None,
                           stream=None):
    """Backward with one gradient row per visible (view, Gaussian) pair (cgs_render_backward_packed):
    returns (g_mean_opac, g_scale, g_quat, g_sh, g_index), each with frame.n_cap rows of which the
    first n_vis (frame.status()[1][1]) are written."""
    if rows is None:
        f32, dev, cap = torch.float32, dscene.device, frame.n_cap
        rows = (torch.empty((cap, 4), dtype=f32, device=dev), torch.empty((cap, 4), dtype=f32, device=dev),
                torch.empty((cap, 4), dtype=f32, device=dev),
                torch.empty((cap,) + tuple(dscene.sh.shape[1:]), dtype=f32, device=dev),
                torch.empty(cap, dtype=torch.int64, device=dev))
    g_mo, g_sc, g_q, g_sh, g_idx = rows
    _c.cgs_render_backward_packed(dscene.struct(attrs), frame.struct, cfg, d_cams, dL_dimage.contiguous(), final_T,
                                  n_contrib, g_mo, g_sc, g_q, g_sh, g_idx, stream)
    return rows


class RenderFn(torch.autograd.Function):
    """image = render(mean_opac, scale, quat, sh) for the views of `frame`.

    Inputs are activated attributes (linear scales, opacity in (0, 1)); apply exp / sigmoid
    / normalisation in torch before calling.  Gradients come from cgs_render_backward.
    """

    @staticmethod
    def forward(ctx, mean_opac, scale, quat, sh, dscene, frame, cfg, d_cams, view_block=None, levels=None):
        attrs = {"mean_opac": mean_opac.contiguous(), "scale": scale.contiguous(), "quat": quat.contiguous(),
                 "sh": sh.contiguous()}
        img, T, nc = render_forward(dscene, frame, cfg, d_cams, view_block, levels, attrs=attrs)
        ctx.save_for_backward(T, nc)
        ctx.attrs = attrs
        ctx.meta = (dscene, frame, cfg, d_cams)
        ctx.mark_non_differentiable(T, nc)
        return img, T, nc

    @staticmethod
    def backward(ctx, g_img, g_T, g_nc):
        T, nc = ctx.saved_tensors
        dscene, frame, cfg, d_cams = ctx.meta
        a = ctx.attrs
        grads = (torch.zeros_like(a["mean_opac"]), torch.zeros_like(a["scale"]), torch.zeros_like(a["quat"]),
                 torch.zeros_like(a["sh"]))
        render_backward(dscene, frame, cfg, d_cams, g_img.contiguous(), T, nc, grads=grads, attrs=a)
        return grads + (None, None, None, None, None, None)


def render_backward_l1(dscene, frame, cfg, d_cams, img, target, final_T, n_contrib, grads=None, rows=None,
                       attrs=None, stream=None):
    """L1 loss and backward in one pass (cgs_render_backward_l1): returns (loss, gradients).  With
    `rows` (or neither `grads` nor `rows`) the gradients are packed rows as render_backward_packed
    returns them; with `grads` they are added into those scene-indexed arrays."""
    loss = torch.zeros(1, dtype=torch.float32, device=img.device)
    u8 = 1 if target.dtype == torch.uint8 else 0
    if grads is not None:
        g_mo, g_sc, g_q, g_sh = grads
        _c.cgs_render_backward_l1(dscene.struct(attrs), frame.struct, cfg, d_cams, img, target.contiguous(), u8,
                                  final_T, n_contrib, loss, g_mo, g_sc, g_q, g_sh, None, stream)
        return loss, grads
    if rows is None:
        f32, dev, cap = torch.float32, dscene.device, frame.n_cap
        rows = (torch.empty((cap, 4), dtype=f32, device=dev), torch.empty((cap, 4), dtype=f32, device=dev),
                torch.empty((cap, 4), dtype=f32, device=dev),
                torch.empty((cap,) + tuple(dscene.sh.shape[1:]), dtype=f32, device=dev),
                torch.empty(cap, dtype=torch.int64, device=dev))
    g_mo, g_sc, g_q, g_sh, g_idx = rows
    _c.cgs_render_backward_l1(dscene.struct(attrs), frame.struct, cfg, d_cams, img, target.contiguous(), u8,
                              final_T, n_contrib, loss, g_mo, g_sc, g_q, g_sh, g_idx, stream)
    return loss, rows


def l1_loss(img, target, stream=None):
    """L1 loss and its gradient; target is float32, or uint8 (t stands for t / 255)."""
    loss = torch.zeros(1, dtype=torch.float32, device=img.device)
    grad = torch.empty_like(img)
    if target.dtype == torch.uint8:
        _c.cgs_l1_loss_u8(img, target, img.numel(), loss, grad, stream)
    else:
        _c.cgs_l1_loss(img, target, img.numel(), loss, grad, stream)
    return loss, grad


# ---------------------------------------------------------------------------------------
# capacity calibration, CUDA graphs, autotuning
# ---------------------------------------------------------------------------------------
def frame_counts(dscene, cams, width, height, tile=16, view_block=None, levels=None, device="cuda",
                 n_cap=None, k_cap=None, cfg=None):
    """Selected Gaussians and tile entries of each view, rendered one view at a time.

    Used to size batched frames: returns two lists (selected, entries) per view.  The entry
    count is exact even past the counting frame's capacity (the projection counts every entry
    and drops the ones that do not fit), so the counting frame stays small."""
    n_cap = n_cap or max(1, dscene.n)
    k_cap = k_cap or min((1 << 30) - 1, 4 * n_cap + (1 << 20))
    fr = Frame(1, width, height, tile, dscene.n_blocks, n_cap, k_cap, device)
    cfg = cfg or make_config(tile=tile)
    sel, ent = [], []
    out = fr.outputs()
    for v in range(len(cams)):
        d_cam = cameras_device([cams[v]], device)
        vb = None if view_block is None else view_block[v:v + 1]
        lv = None if levels is None else levels[v:v + 1]
        render_forward(dscene, fr, cfg, d_cam, vb, lv, out=out)
        st, c = fr.status()
        if st not in (_c.CGS_OK, _c.CGS_ERR_CAPACITY):
            raise _c.CgsError(st, "frame_counts")
        sel.append(int(c[0]))
        ent.append(int(c[2]))
    del fr, out
    torch.cuda.empty_cache()
    return sel, ent


def waves(sel, ent, n_cap_max=(1 << 31) - 1, k_cap_max=(1 << 30) - 1, slack=1.05):
    """Splits views into consecutive groups whose summed counts fit the frame capacities."""
    groups, cur, s_sum, e_sum = [], [], 0, 0
    for v, (s, e) in enumerate(zip(sel, ent)):
        s2, e2 = int(s * slack) + 1024, int(e * slack) + 4096
        if cur and (s_sum + s2 > n_cap_max or e_sum + e2 > k_cap_max):
            groups.append((cur, s_sum, e_sum))
            cur, s_sum, e_sum = [], 0, 0
        cur.append(v)
        s_sum += s2
        e_sum += e2
    if cur:
        groups.append((cur, s_sum, e_sum))
    return groups


def capture(fn, warmup=2, stream=None):
    """Runs fn() `warmup` times, then captures one call into a CUDA graph and returns it."""
    s = stream or torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(warmup):
            fn()
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        fn()
    return g


def autotune(run_step, candidates, reps=5, cache_path=None, key=None):
    """Times run_step(tile, batch) for every (tile, batch) candidate with CUDA events (median of
    `reps` after one warm-up) and returns (best, {candidate: ms}).  With cache_path and key,
    the choice is read from / written to a JSON cache keyed by GPU name and workload."""
    import json
    import os
    gpu = torch.cuda.get_device_name()
    full_key = f"{gpu}|{key}" if key else None
    if cache_path and full_key and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
            if full_key in cache:
                t, b = cache[full_key]["choice"]
                return (t, b), cache[full_key]["ms"]
        except (ValueError, KeyError, TypeError):
            pass
    times = {}
    for tile, batch in candidates:
        run_step(tile, batch)
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            run_step(tile, batch)
            b_.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b_))
        times[(tile, batch)] = sorted(ms)[len(ms) // 2]
    best = min(times, key=times.get)
    if cache_path and full_key:
        cache = {}
        if os.path.exists(cache_path):
            try:
                cache = json.load(open(cache_path))
            except ValueError:
                cache = {}
        cache[full_key] = {"choice": list(best), "ms": {f"{t}x{b}": v for (t, b), v in times.items()}}
        json.dump(cache, open(cache_path, "w"), indent=1)
    return best, {f"{t}x{b}": v for (t, b), v in times.items()}


TUNE_CANDIDATES = [(16, 256), (16, 128), (16, 64), (8, 64), (8, 32)]


def autotune_library(dscene, d_cams, width, height, n_cap, k_cap, cfg=None, view_block=None, levels=None,
                     backward=True, reps=3, cache_path=None, cache_key=None, stream=None):
    """The library's autotuner (cgs_autotune): times the real step for every (tile, batch)
    candidate in a workspace from torch and returns (config with the choice, {candidate: ms})."""
    cfg = cfg or make_config()
    n_views = d_cams.numel() // 96
    mode = _c.CGS_TUNE_FORWARD_BACKWARD if backward else _c.CGS_TUNE_FORWARD
    nbytes = _c.cgs_autotune_workspace_bytes(n_views, width, height, dscene.n_blocks, n_cap, k_cap, dscene.sh_degree,
                                             mode)
    if nbytes < 0:
        raise ValueError("invalid autotune dimensions")
    ws = torch.empty(nbytes, dtype=torch.uint8, device=dscene.device)
    ms = _c.cgs_autotune(dscene.struct(), d_cams, n_views, width, height, view_block, levels, n_cap, k_cap, mode, reps,
                         ws, nbytes, cfg, cache_path, cache_key, stream)
    del ws
    return cfg, ms


def partition(pos, pmin, pmax, grid, perm=True, rank=False, stream=None):
    """Block partition of the positions (rows of a float32 device tensor, xyz first): block
    per row, block offsets and (optionally) the stable grouped order.  Returns
    (block int32 [n], offset int64 [n_blocks + 1], perm int32 [offset[-1]] or None, workspace),
    plus rank int32 [n] (the inverse permutation, -1 for no block) when ``rank``; with perm the
    call synchronises to read the number of grouped points."""
    n, stride = pos.shape[0], pos.shape[1]
    assert pos.dtype == torch.float32 and pos.is_contiguous()
    nb = int(np.prod(grid))
    ws_bytes = _c.cgs_partition_workspace_bytes(n, grid)
    if ws_bytes < 0:
        raise ValueError("invalid partition grid")
    dev = pos.device
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    block = torch.empty(max(1, n), dtype=torch.int32, device=dev)
    offset = torch.empty(nb + 1, dtype=torch.int64, device=dev)
    p = torch.empty(max(1, n), dtype=torch.int32, device=dev) if perm else None
    r = torch.empty(max(1, n), dtype=torch.int32, device=dev) if rank else None
    _c.cgs_partition(pos, n, stride, pmin, pmax, grid, block, offset, p, r, ws, ws_bytes, stream)
    if p is not None:
        # only the first offset[n_blocks] entries are written (points with no block are left out)
        p = p[:int(offset[-1].item())]
    if rank:
        return block[:n], offset, p, ws, r[:n]
    return block[:n], offset, p, ws


def gather_rows(src, perm, out=None, stream=None):
    """Rows of src (any dtype, contiguous) in the order perm (int32 device tensor)."""
    n = perm.shape[0]
    out = out if out is not None else torch.empty((n,) + tuple(src.shape[1:]), dtype=src.dtype, device=src.device)
    row_bytes = src[0].numel() * src.element_size() if src.shape[0] else 4
    _c.cgs_gather_rows(src, out, row_bytes, perm, n, stream)
    return out


def render_forward_hits(dscene, frame, cfg, d_cams, hits, view_block=None, levels=None, out=None, stream=None):
    """Forward render that also adds each scene Gaussian's blended-pixel count to ``hits``
    (uint32 stored in an int32 device tensor of scene length)."""
    img, T, nc = out if out is not None else frame.outputs()
    _c.cgs_render_forward_hits(dscene.struct(), frame.struct, cfg, d_cams, view_block, levels, img, T, nc, hits,
                               stream)
    return img, T, nc


def generate_levels(dscene, block_offset, rates, hits=None, stream=None):
    """Ranked permutation (int32 [n]) and level counts (int64 [n_blocks][len(rates)]) of the
    block-grouped device scene (block b = rows [block_offset[b], block_offset[b + 1]))."""
    n = dscene.n
    nb = block_offset.shape[0] - 1
    ws_bytes = _c.cgs_levels_workspace_bytes(n, nb)
    if ws_bytes < 0:
        raise ValueError("invalid level generation size")
    dev = dscene.device
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    perm = torch.empty(max(1, n), dtype=torch.int32, device=dev)
    lc = torch.empty((nb, len(rates)), dtype=torch.int64, device=dev)
    _c.cgs_generate_levels(dscene.mean_opac, dscene.scale, dscene.attr_fp16, n, block_offset, nb, hits, rates, perm,
                           lc, ws, ws_bytes, stream)
    if _c.cgs_levels_status(ws, stream) != _c.CGS_OK:
        raise RuntimeError("cgs_generate_levels: a bounded wait gave up")
    return perm[:n], lc


def scatter_rows(src, rank, n_out, out=None, stream=None):
    """Rows of src moved to rows rank[r] of a new [n_out, ...] tensor (rank < 0 skipped)."""
    out = out if out is not None else torch.empty((n_out,) + tuple(src.shape[1:]), dtype=src.dtype, device=src.device)
    row_bytes = src[0].numel() * src.element_size() if src.shape[0] else 4
    _c.cgs_scatter_rows(src, out, row_bytes, rank, src.shape[0], stream)
    return out


def ssim(a, b, with_map=False, stream=None):
    """Mean SSIM of image pairs: a [C, H, W] (compared with every b) or [n, C, H, W], b
    [n, C, H, W] (float32 device tensors); returns [n] (and the [n, H, W] map)."""
    if b.dim() == 3:
        b = b[None]
    n, c, h, w = b.shape
    a_stride = 0 if a.dim() == 3 else c * h * w
    out = torch.empty(n, dtype=torch.float32, device=b.device)
    m = torch.empty((n, h, w), dtype=torch.float32, device=b.device) if with_map else None
    _c.cgs_ssim(a.contiguous(), a_stride, b.contiguous(), n, c, w, h, out, m, stream)
    return (out, m) if with_map else out


def pose_assign(dscene, cams, pmin, pmax, grid, eps, tile=16, batch=None):
    """Pose-to-block assignment of Sec. 3.2.2: B1 (Eq. 3) where the SSIM loss between the render
    with every block and the render without block j exceeds eps; B2 (Eq. 4) where the camera
    centre lies in block j after normalisation and contraction; B = B1 + B2 (Eq. 5, read as a
    logical or).  The scene's blocks are its block table (level 0 of each block); the renders of
    one pose are one batched frame of n_blocks + 1 views, split into waves that fit the frame
    capacities.  Returns (B1, B2, B) as [n_poses, n_blocks] bool tensors and the SSIM values."""
    nb = dscene.n_blocks
    P = len(cams)
    W, H = cams[0]["width"], cams[0]["height"]
    dev = dscene.device
    cfg = make_config(tile=tile, batch=batch)
    campos = torch.tensor(np.asarray([c["campos"] for c in cams], np.float32), device=dev)
    pb = torch.empty(P, dtype=torch.int32, device=dev)
    _c.cgs_pose_blocks(campos, P, 3, pmin, pmax, grid, pb)
    lv_all = torch.zeros((nb + 1, nb), dtype=torch.int8, device=dev)
    lv_all[torch.arange(1, nb + 1), torch.arange(nb)] = -1
    s_all = torch.empty((P, nb), dtype=torch.float32, device=dev)
    for i, cam in enumerate(cams):
        sel, ent = frame_counts(dscene, [cam], W, H, tile=tile, levels=lv_all[:1], cfg=cfg)
        per_sel, per_ent = sel[0], ent[0]
        full = None
        # frames of at most ~64M selected Gaussians (a few GB of workspace), at least one view
        groups = waves([per_sel] * (nb + 1), [per_ent] * (nb + 1), n_cap_max=max(1 << 26, 2 * per_sel + 4096),
                       k_cap_max=min((1 << 30) - 1, max(1 << 28, 2 * per_ent + 8192)))
        for views, n_cap, k_cap in groups:
            views = list(views)
            fr = Frame(len(views), W, H, tile, nb, n_cap, k_cap, dev)
            d_cams = cameras_device([cam] * len(views), dev)
            img, T, nc = render_forward(dscene, fr, cfg, d_cams, None, lv_all[views].contiguous())
            st, _ = fr.status()
            if st != _c.CGS_OK:
                raise _c.CgsError(st, "pose_assign")
            if views[0] == 0:
                full = img[0].clone()
                img, views = img[1:], views[1:]
            if views:
                s_all[i, torch.tensor(views, device=dev) - 1] = ssim(full, img)
    # Eqs. 3-5 in the library: B1 from the SSIM losses, B2 from the poses' blocks, B = B1 or B2
    b1u = torch.empty((P, nb), dtype=torch.uint8, device=dev)
    b2u = torch.empty_like(b1u)
    bu = torch.empty_like(b1u)
    _c.cgs_pose_assign(s_all, pb, P, nb, eps, b1u, b2u, bu)
    return b1u.bool(), b2u.bool(), bu.bool(), s_all
