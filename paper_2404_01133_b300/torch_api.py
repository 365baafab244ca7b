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


def make_config(tile=16, batch=None, near_z=0.2, bg=(0.0, 0.0, 0.0), lod_dist=(200.0, 600.0)):
    c = _c.cgs_config()
    c.tile = tile
    c.batch = batch if batch is not None else (256 if tile == 16 else 64)
    c.near_z = near_z
    c.bg[:] = list(bg)
    c.lod_dist[:] = list(lod_dist)
    return c


class DeviceScene:
    """A synth-format scene uploaded to the device, with its cgs_scene descriptor."""

    def __init__(self, scene, device="cuda", attrs=None):
        dev = torch.device(device)
        if attrs is None:
            attrs = {k: torch.from_numpy(np.ascontiguousarray(scene[k], np.float32)).to(dev)
                     for k in ("mean_opac", "scale", "quat", "sh")}
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
        s.level_offset = self.level_offset.data_ptr()
        s.level_count = self.level_count.data_ptr()
        s.block_aabb = self.block_aabb.data_ptr()
        s.block_cell = self.block_cell.data_ptr()
        return s

    def compute_block_bounds(self, n_mad=4.0, stream=None):
        """Eq. 7 MAD bounds of every block, written into self.block_aabb by the library."""
        _c.cgs_block_bounds(self.struct(), n_mad, self.block_aabb, None, 0, stream)
        return self.block_aabb


class Frame:
    """Workspace of a batch of equally sized views (device memory from torch)."""

    def __init__(self, n_views, width, height, tile, n_blocks, n_cap, k_cap, device="cuda"):
        nbytes = _c.cgs_frame_workspace_bytes(n_views, width, height, tile, n_blocks, n_cap, k_cap)
        if nbytes <= 0:
            raise ValueError("invalid frame dimensions")
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=device)
        f = _c.cgs_frame()
        f.ws = self.ws.data_ptr()
        f.ws_bytes = nbytes
        f.n_views, f.width, f.height, f.tile, f.n_blocks = n_views, width, height, tile, n_blocks
        f.n_cap, f.k_cap = n_cap, k_cap
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
        dev = dscene.device
        grads = (torch.zeros_like(dscene.mean_opac), torch.zeros_like(dscene.scale),
                 torch.zeros_like(dscene.quat), torch.zeros_like(dscene.sh))
    g_mo, g_sc, g_q, g_sh = grads
    _c.cgs_render_backward(dscene.struct(attrs), frame.struct, cfg, d_cams, dL_dimage.contiguous(), final_T,
                           n_contrib, g_mo, g_sc, g_q, g_sh, stream)
    return grads


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


def l1_loss(img, target, stream=None):
    loss = torch.zeros(1, dtype=torch.float32, device=img.device)
    grad = torch.empty_like(img)
    _c.cgs_l1_loss(img, target, img.numel(), loss, grad, stream)
    return loss, grad
