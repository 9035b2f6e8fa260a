"""Device-resident scenes and a frame renderer over the C ABI.

torch provides device memory and streams; every step of the frame runs in
libgs3's CUDA kernels.  `DeviceScene` uploads a host scene (structure of
arrays) once; `Renderer` owns a workspace and renders frames into a device
image, exposing the workspace's intermediate buffers for inspection.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _native as N


def camera_struct(cam) -> N.gs3_camera:
    c = N.gs3_camera()
    c.R = (C.c_float * 9)(*np.asarray(cam.R, dtype=np.float32).reshape(-1).tolist())
    c.t = (C.c_float * 3)(*np.asarray(cam.t, dtype=np.float32).tolist())
    c.pos = (C.c_float * 3)(*np.asarray(cam.pos, dtype=np.float32).tolist())
    c.fx, c.fy, c.cx, c.cy = cam.fx, cam.fy, cam.cx, cam.cy
    c.width, c.height = cam.width, cam.height
    return c


def light_struct(light) -> N.gs3_light:
    d = getattr(light, "dir", None)
    d = (0.0, 0.0, 0.0) if d is None else np.asarray(d, dtype=np.float32).tolist()
    return N.gs3_light((C.c_float * 3)(*np.asarray(light.pos, dtype=np.float32).tolist()),
                       float(light.intensity), int(getattr(light, "type", 0)), (C.c_float * 3)(*d),
                       float(getattr(light, "extent", 0.0)))


def opts_struct(ablate: int = 0, falloff: int = 1, **kw) -> N.gs3_render_opts:
    o = N.gs3_default_opts()
    o.ablate = ablate
    o.falloff = falloff
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class DeviceScene:
    """Scene parameters resident on the GPU plus the library's scene handle."""

    ARRAYS_DEV = N.GRAD_FIELDS

    def __init__(self, scene, device="cuda", mlp_dtype: int = N.GS3_MLP_FP32):
        self.n, self.k = scene.n, scene.k
        dev = torch.device(device)
        self.t = {}
        for a in scene.ARRAYS:
            arr = np.ascontiguousarray(getattr(scene, a), dtype=np.float32)
            if arr.size == 0:
                arr = np.zeros(4, dtype=np.float32)
            self.t[a] = torch.from_numpy(arr).to(dev)
        for nm in ("phi", "psi"):
            w, b = getattr(scene, nm).packed()
            self.t[nm + "_w"] = torch.from_numpy(w).to(dev)
            self.t[nm + "_b"] = torch.from_numpy(b).to(dev)
        d = N.gs3_scene_desc()
        d.n, d.k = scene.n, scene.k
        for a in scene.ARRAYS:
            setattr(d, a, self.t[a].data_ptr())
        for nm in ("phi", "psi"):
            m = getattr(scene, nm)
            setattr(d, nm, N.gs3_mlp_desc(m.in_dim, m.width, m.n_hidden, m.out_dim, m.act,
                                          self.t[nm + "_w"].data_ptr(), self.t[nm + "_b"].data_ptr()))
        d.mlp_dtype = mlp_dtype
        d.lobe_shared = int(getattr(scene, "lobe_shared", False))
        self.desc = d
        self.handle = N.gs3_create_scene(d)

    def close(self):
        if self.handle:
            N.gs3_destroy_scene(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Renderer:
    """One workspace sized for (n, width, height, key_capacity)."""

    def __init__(self, dscene: DeviceScene, width: int, height: int, key_capacity: int,
                 device="cuda"):
        self.scene = dscene
        self.width, self.height, self.cap = width, height, int(key_capacity)
        nbytes = N.gs3_workspace_size(dscene.n, width, height, self.cap)
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        pad = (-self.ws.data_ptr()) % 256
        self.ws = self.ws[pad:pad + nbytes]
        self.layout = N.gs3_workspace_layout(dscene.n, width, height, self.cap)
        self.image = torch.empty((height, width, 3), dtype=torch.float32, device=device)

    def render(self, cam, light, opts=None, out=None, stream=None):
        opts = opts if opts is not None else opts_struct()
        out = self.image if out is None else out
        s = torch.cuda.current_stream() if stream is None else stream
        N.gs3_render(self.scene.handle, camera_struct(cam), light_struct(light), opts, out, self.ws,
                     self.cap, s.cuda_stream)
        return out

    def env_workspace(self, count: int):
        """The 256-byte aligned workspace of an environment render of `count` lights."""
        nbytes = N.gs3_environment_workspace_size(self.scene.n, self.width, self.height, max(count, 1),
                                                  self.cap)
        have = getattr(self, "env_ws", None)
        if have is None or have.numel() < nbytes:
            raw = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.ws.device)
            pad = (-raw.data_ptr()) % 256
            self.env_ws = raw[pad:pad + nbytes]
        return self.env_ws

    def render_environment(self, cam, lights, weights, opts=None, out=None, stream=None):
        """Sec. 4.5: sum_l weights[l] * render(lights[l]) (directional lights), one batched frame."""
        opts = opts if opts is not None else opts_struct()
        out = self.image if out is None else out
        ws = self.env_workspace(len(lights))
        s = torch.cuda.current_stream() if stream is None else stream
        N.gs3_render_environment(self.scene.handle, camera_struct(cam), [light_struct(L) for L in lights],
                                 weights, opts, out, ws, self.cap, s.cuda_stream)
        return out

    def render_stages(self, cam, light, stages: int, opts=None, out=None, stream=None):
        opts = opts if opts is not None else opts_struct()
        out = self.image if out is None else out
        s = torch.cuda.current_stream() if stream is None else stream
        N.gs3_render_stages(self.scene.handle, camera_struct(cam), light_struct(light), opts, out,
                            self.ws, self.cap, stages, s.cuda_stream)
        return out

    def backward(self, cam, light, dl_drgb, opts=None, stream=None) -> dict:
        """Gradients of every scene parameter for dL/d(image) of the last
        render() of the same (cam, light, opts); arrays shaped like the scene's."""
        opts = opts if opts is not None else opts_struct()
        s = torch.cuda.current_stream() if stream is None else stream
        if getattr(self, "bws", None) is None:
            nb = N.gs3_backward_workspace_size(self.scene.handle)
            self.bws = torch.empty(nb, dtype=torch.uint8, device=self.ws.device)
        grads = {f: torch.zeros_like(self.scene.t[f]) for f in self.scene.ARRAYS_DEV}
        N.gs3_render_backward(self.scene.handle, camera_struct(cam), light_struct(light), opts,
                              dl_drgb.contiguous(), self.ws, self.cap, self.bws, grads, s.cuda_stream)
        return grads

    def header(self, stream=None) -> N.gs3_ws_header:
        s = torch.cuda.current_stream() if stream is None else stream
        return N.gs3_workspace_read_header(self.ws, s.cuda_stream)

    def env_header(self, stream=None) -> N.gs3_ws_header:
        """Header of the last environment render (status, camera and largest light pair counts)."""
        s = torch.cuda.current_stream() if stream is None else stream
        return N.gs3_workspace_read_header(self.env_ws, s.cuda_stream)

    def check(self):
        h = self.header()
        if h.status != N.GS3_OK:
            raise N.GS3Error(h.status, f"device status (pairs needed: camera {h.pairs_cam_needed}, "
                                       f"light {h.pairs_light_needed}, capacity {self.cap})")
        return h

    # -- inspection views ------------------------------------------------------
    def _view(self, off: int, count: int, dtype) -> torch.Tensor:
        nb = count * torch.empty((), dtype=dtype).element_size()
        return self.ws[off:off + nb].view(dtype)

    def stage(self, name: str, splat: int = 0) -> torch.Tensor:
        L, n = self.layout, self.scene.n
        ntiles = ((self.width + 15) // 16) * ((self.height + 15) // 16)
        if name == "key":
            return self._view(L.key[splat], n, torch.int32)
        if name == "order":
            return self._view(L.order[splat], n, torch.int32)
        if name == "tile_start":
            return self._view(L.tile_start[splat], ntiles + 1, torch.int32)
        if name == "list":
            return self._view(L.list[splat], self.cap, torch.int32)
        if name == "rect":
            return self._view(L.rect[splat], 4 * n, torch.int32).view(n, 4)
        if name == "shade":
            return self._view(L.shade, 4 * n, torch.float32).view(n, 4)
        if name == "T":
            return self._view(L.shadow, n, torch.float32)
        if name == "Tp":
            return self._view(L.shadow_refined, n, torch.float32)
        if name == "res":
            return self._view(L.residual, 4 * n, torch.float32).view(n, 4)
        if name == "final_t":
            return self._view(L.final_t, self.width * self.height, torch.float32).view(self.height, self.width)
        if name == "n_contrib":
            return self._view(L.n_contrib, self.width * self.height, torch.int32).view(self.height, self.width)
        if name == "light_final":
            return self._view(L.light_final, self.width * self.height, torch.float32).view(self.height, self.width)
        if name == "light_stop":
            return self._view(L.light_stop, self.width * self.height, torch.int32).view(self.height, self.width)
        raise KeyError(name)


class Server:
    """Continuous-batching server (gs3_server_*) over device-resident scenes."""

    def __init__(self, hbm_budget: int, max_inflight: int = 4, device: int = 0,
                 inject_alloc_failures: int = 0, initial_pairs: float = 0.0, max_batch: int = 0,
                 light_cache: int = 0):
        """max_inflight slots, each rendering up to max_batch requests together
        (0 or 1: every request alone on its slot's streams); light_cache: shadow
        values kept for that many (scene, light, size, options) keys."""
        self.handle = N.gs3_server_create(hbm_budget, max_inflight, device, inject_alloc_failures,
                                          initial_pairs, max_batch, light_cache)
        self.scenes = []

    def add_scene(self, dscene: DeviceScene) -> int:
        self.scenes.append(dscene)  # keep the parameters alive
        return N.gs3_server_add_scene(self.handle, dscene.handle)

    def submit(self, scene_id: int, cam, light, out, opts=None) -> int:
        """Queue a frame into `out` (device [H, W, 3] float32).  The server's
        streams do not wait for torch's: no pending kernel may write `out`,
        and it must stay alive until the request completes."""
        opts = opts if opts is not None else opts_struct()
        return N.gs3_server_submit(self.handle, scene_id, camera_struct(cam), light_struct(light),
                                   opts, out)

    def wait(self, ticket: int, timeout_s: float = 120.0):
        return N.gs3_server_wait(self.handle, ticket, timeout_s)

    def poll(self, ticket: int):
        return N.gs3_server_poll(self.handle, ticket)

    def stats(self):
        return N.gs3_server_stats(self.handle)

    def reset_counters(self):
        N.gs3_server_reset_counters(self.handle)

    def close(self):
        if self.handle:
            N.gs3_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class RenderFunction(torch.autograd.Function):
    """Differentiable frame: forward gs3_render, backward gs3_render_backward.

    Inputs after (renderer, cam, light, opts) are the scene's device tensors
    in N.GRAD_FIELDS order; they are read by the library through the scene
    handle, and their gradients come from the hand-written backward."""

    @staticmethod
    def forward(ctx, renderer, cam, light, opts, *params):
        img = renderer.render(cam, light, opts).clone()
        ctx.renderer, ctx.cam, ctx.light, ctx.opts = renderer, cam, light, opts
        return img

    @staticmethod
    def backward(ctx, grad_img):
        g = ctx.renderer.backward(ctx.cam, ctx.light, grad_img, ctx.opts)
        return (None, None, None, None) + tuple(g[f] for f in N.GRAD_FIELDS)


def render_differentiable(renderer, cam, light, opts=None):
    """Image tensor whose backward flows into renderer.scene.t[...] tensors."""
    sc = renderer.scene
    opts = opts if opts is not None else opts_struct()
    return RenderFunction.apply(renderer, cam, light, opts, *[sc.t[f] for f in N.GRAD_FIELDS])


def loss_l1_dssim(img, target, lam: float = 0.2, stream=None):
    """(loss tensor [1], dL/d(img)) of (1 - lam) L1 + lam (1 - SSIM), on the GPU."""
    s = torch.cuda.current_stream() if stream is None else stream
    h, w = img.shape[0], img.shape[1]
    scratch = torch.empty(N.gs3_loss_scratch_size(w, h), dtype=torch.uint8, device=img.device)
    loss = torch.empty(1, dtype=torch.float32, device=img.device)
    dimg = torch.empty_like(img)
    N.gs3_loss_l1_dssim(img.contiguous(), target.contiguous(), lam, loss, dimg, scratch, s.cuda_stream)
    return loss, dimg
