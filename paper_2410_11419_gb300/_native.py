"""ctypes binding of libgs3 (include/gs3.h): argument marshalling only.

Every function here has the name of the C entry point it calls.  Device
buffers are passed as torch CUDA tensors (their data pointers); camera,
light and options as the ctypes structures below.  There is no CPU fallback:
if libgs3.so is missing or a call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgs3.so")

GS3_OK, GS3_ERR_INVALID_ARG, GS3_ERR_OOM, GS3_ERR_CAPACITY, GS3_ERR_CUDA, GS3_ERR_TIMEOUT, \
    GS3_ERR_UNSUPPORTED = range(7)
GS3_ACT_RELU, GS3_ACT_LEAKY_RELU = 0, 1
GS3_MLP_FP32, GS3_MLP_BF16, GS3_MLP_FP8_E4M3 = 0, 1, 2
GS3_ABLATE_SHADOW_SPLAT, GS3_ABLATE_PHI, GS3_ABLATE_PSI, GS3_ABLATE_SPECULAR = 1, 2, 4, 8
GS3_STAGE_PREP, GS3_STAGE_CAMERA_BIN, GS3_STAGE_LIGHT_BIN, GS3_STAGE_SHADOW_COMPOSITE, \
    GS3_STAGE_SHADOW_REDUCE, GS3_STAGE_MLP, GS3_STAGE_CAMERA, GS3_STAGE_ALL = 1, 2, 4, 8, 16, 32, 64, 127

STATUS_NAMES = {0: "GS3_OK", 1: "GS3_ERR_INVALID_ARG", 2: "GS3_ERR_OOM", 3: "GS3_ERR_CAPACITY",
                4: "GS3_ERR_CUDA", 5: "GS3_ERR_TIMEOUT", 6: "GS3_ERR_UNSUPPORTED"}


class GS3Error(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_FP = C.POINTER(C.c_float)


class gs3_mlp_desc(C.Structure):
    _fields_ = [("in_dim", C.c_int32), ("width", C.c_int32), ("n_hidden", C.c_int32),
                ("out_dim", C.c_int32), ("act", C.c_int32), ("w", C.c_void_p), ("b", C.c_void_p)]


class gs3_scene_desc(C.Structure):
    _fields_ = [("n", C.c_int32), ("k", C.c_int32)] + [
        (a, C.c_void_p) for a in ("mean_op", "scale", "rot", "shade_rot", "albedo_d", "albedo_s",
                                  "latent", "lobe_rot", "lobe_sigma", "lobe_amp")] + [
        ("phi", gs3_mlp_desc), ("psi", gs3_mlp_desc), ("mlp_dtype", C.c_int32),
                ("lobe_shared", C.c_int32)]


class gs3_camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("pos", C.c_float * 3),
                ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("width", C.c_int32), ("height", C.c_int32)]


GS3_LIGHT_POINT, GS3_LIGHT_DIRECTIONAL = 0, 1


class gs3_light(C.Structure):
    _fields_ = [("pos", C.c_float * 3), ("intensity", C.c_float), ("type", C.c_int32),
                ("dir", C.c_float * 3), ("extent", C.c_float)]


class gs3_render_opts(C.Structure):
    _fields_ = [("near_z", C.c_float), ("lowpass", C.c_float), ("frustum", C.c_float),
                ("shadow_bias", C.c_float), ("alpha_min", C.c_float), ("alpha_max", C.c_float),
                ("t_stop", C.c_float), ("target", C.c_float * 3), ("falloff", C.c_int32),
                ("tile", C.c_int32), ("ablate", C.c_int32)]


class gs3_ws_header(C.Structure):
    _fields_ = [("status", C.c_uint32), ("pairs_cam", C.c_uint32), ("pairs_light", C.c_uint32),
                ("pairs_cam_needed", C.c_uint32), ("pairs_light_needed", C.c_uint32),
                ("reserved", C.c_uint32 * 3), ("light_R", C.c_float * 9), ("light_t", C.c_float * 3),
                ("light_ortho", C.c_float)]


class gs3_ws_layout(C.Structure):
    _fields_ = [("total", C.c_size_t), ("header", C.c_size_t), ("key", C.c_size_t * 2),
                ("order", C.c_size_t * 2), ("tile_start", C.c_size_t * 2), ("list", C.c_size_t * 2),
                ("rect", C.c_size_t * 2), ("shade", C.c_size_t), ("shadow", C.c_size_t),
                ("shadow_refined", C.c_size_t), ("residual", C.c_size_t), ("final_t", C.c_size_t),
                ("n_contrib", C.c_size_t), ("light_final", C.c_size_t), ("light_stop", C.c_size_t)]


class gs3_scene(C.Structure):
    pass


GRAD_FIELDS = ("mean_op", "scale", "rot", "shade_rot", "albedo_d", "albedo_s", "latent", "lobe_rot",
               "lobe_sigma", "lobe_amp", "phi_w", "phi_b", "psi_w", "psi_b")


class gs3_grads(C.Structure):
    _fields_ = [(f, C.c_void_p) for f in GRAD_FIELDS]


class gs3_server(C.Structure):
    pass


class gs3_server_opts(C.Structure):
    _fields_ = [("hbm_budget", C.c_size_t), ("max_inflight", C.c_int32), ("device", C.c_int32),
                ("inject_alloc_failures", C.c_int32), ("initial_pairs", C.c_float), ("max_batch", C.c_int32),
                ("light_cache", C.c_int32)]


class gs3_server_counters(C.Structure):
    _fields_ = [(f, C.c_uint64) for f in ("completed", "failed", "retries", "queued", "in_flight",
                                          "max_in_flight", "bytes_in_use", "peak_bytes_in_use")] + [
        ("device_span_ms", C.c_double), ("batches", C.c_uint64), ("max_batch", C.c_uint64),
        ("light_reuse", C.c_uint64)]


GS3_REQ_QUEUED, GS3_REQ_RUNNING, GS3_REQ_DONE, GS3_REQ_FAILED = 0, 1, 2, 3
_SERVER_P = C.POINTER(gs3_server)


_SCENE_P = C.POINTER(gs3_scene)

# name -> (restype, argtypes); every symbol include/gs3.h declares
SIGNATURES = {
    "gs3_default_opts": (None, [C.POINTER(gs3_render_opts)]),
    "gs3_create_scene": (C.c_int, [C.POINTER(gs3_scene_desc), C.POINTER(_SCENE_P)]),
    "gs3_destroy_scene": (C.c_int, [_SCENE_P]),
    "gs3_scene_mlp_scales": (C.c_int, [_SCENE_P, C.c_int32, C.POINTER(C.c_float), C.c_int32]),
    "gs3_workspace_size": (C.c_size_t, [C.c_int32, C.c_int32, C.c_int32, C.c_size_t]),
    "gs3_workspace_layout": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_size_t,
                                       C.POINTER(gs3_ws_layout)]),
    "gs3_render": (C.c_int, [_SCENE_P, C.POINTER(gs3_camera), C.POINTER(gs3_light),
                             C.POINTER(gs3_render_opts), C.c_void_p, C.c_void_p, C.c_size_t,
                             C.c_size_t, C.c_void_p]),
    "gs3_render_stages": (C.c_int, [_SCENE_P, C.POINTER(gs3_camera), C.POINTER(gs3_light),
                                    C.POINTER(gs3_render_opts), C.c_void_p, C.c_void_p, C.c_size_t,
                                    C.c_size_t, C.c_uint32, C.c_void_p]),
    "gs3_workspace_read_header": (C.c_int, [C.c_void_p, C.POINTER(gs3_ws_header), C.c_void_p]),
    "gs3_adam_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_float,
                                C.c_float, C.c_float, C.c_float, C.c_int32, C.c_float, C.c_void_p]),
    "gs3_render_environment": (C.c_int, [_SCENE_P, C.POINTER(gs3_camera), C.POINTER(gs3_light),
                                         C.POINTER(C.c_float), C.c_int32, C.POINTER(gs3_render_opts),
                                         C.c_void_p, C.c_void_p, C.c_size_t, C.c_size_t, C.c_void_p]),
    "gs3_environment_workspace_size": (C.c_size_t, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_size_t]),
    "gs3_backward_workspace_size": (C.c_size_t, [_SCENE_P]),
    "gs3_loss_scratch_size": (C.c_size_t, [C.c_int32, C.c_int32]),
    "gs3_loss_l1_dssim": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_float, C.c_void_p,
                                    C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "gs3_render_backward": (C.c_int, [_SCENE_P, C.POINTER(gs3_camera), C.POINTER(gs3_light),
                                      C.POINTER(gs3_render_opts), C.c_void_p, C.c_void_p, C.c_size_t,
                                      C.c_size_t, C.c_void_p, C.c_size_t, C.POINTER(gs3_grads),
                                      C.c_void_p]),
    "gs3_server_create": (C.c_int, [C.POINTER(gs3_server_opts), C.POINTER(_SERVER_P)]),
    "gs3_server_add_scene": (C.c_int, [_SERVER_P, _SCENE_P, C.POINTER(C.c_int32)]),
    "gs3_server_submit": (C.c_int, [_SERVER_P, C.c_int32, C.POINTER(gs3_camera), C.POINTER(gs3_light),
                                    C.POINTER(gs3_render_opts), C.c_void_p, C.POINTER(C.c_uint64)]),
    "gs3_server_poll": (C.c_int, [_SERVER_P, C.c_uint64, C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
    "gs3_server_wait": (C.c_int, [_SERVER_P, C.c_uint64, C.c_double, C.POINTER(C.c_double)]),
    "gs3_server_stats": (C.c_int, [_SERVER_P, C.POINTER(gs3_server_counters)]),
    "gs3_server_reset_counters": (C.c_int, [_SERVER_P]),
    "gs3_server_destroy": (C.c_int, [_SERVER_P]),
    "gs3_depth_order_static": (C.c_int, [C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p]),
    "gs3_selftest_wait_timeout": (C.c_int, [C.c_uint32, C.POINTER(C.c_uint32)]),
    "gs3_selftest_shadow_wait": (C.c_int, [_SCENE_P, C.POINTER(gs3_camera), C.POINTER(gs3_light),
                                           C.POINTER(gs3_render_opts), C.c_void_p, C.c_size_t, C.c_size_t,
                                           C.POINTER(C.c_uint32)]),
    "gs3_kernel_launches": (C.c_uint64, []),
    "gs3_measure_alu_peak": (C.c_int, [C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "gs3_last_error": (C.c_char_p, []),
}

_lib = None


def lib():
    """Load libgs3.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libgs3.so not built at {LIB_PATH}; run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(st: int, what: str):
    if st != GS3_OK:
        raise GS3Error(st, f"{what}: {lib().gs3_last_error().decode()}")


def _ptr(t) -> int:
    if t is None:
        return 0
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    return t.data_ptr()


def gs3_default_opts() -> gs3_render_opts:
    o = gs3_render_opts()
    lib().gs3_default_opts(C.byref(o))
    return o


def gs3_create_scene(desc: gs3_scene_desc):
    out = _SCENE_P()
    _check(lib().gs3_create_scene(C.byref(desc), C.byref(out)), "gs3_create_scene")
    return out


def gs3_scene_mlp_scales(scene, which: int, n_hidden: int):
    """FP8 scene: [(sx_l, sw_l)] for every hidden layer of Phi (0) or Psi (1)."""
    buf = (C.c_float * (2 * n_hidden))()
    _check(lib().gs3_scene_mlp_scales(scene, which, buf, 2 * n_hidden), "gs3_scene_mlp_scales")
    return [(buf[2 * l], buf[2 * l + 1]) for l in range(n_hidden)]


def gs3_destroy_scene(scene) -> None:
    _check(lib().gs3_destroy_scene(scene), "gs3_destroy_scene")


def gs3_workspace_size(n: int, width: int, height: int, key_capacity: int) -> int:
    return int(lib().gs3_workspace_size(n, width, height, key_capacity))


def gs3_workspace_layout(n: int, width: int, height: int, key_capacity: int) -> gs3_ws_layout:
    out = gs3_ws_layout()
    _check(lib().gs3_workspace_layout(n, width, height, key_capacity, C.byref(out)),
           "gs3_workspace_layout")
    return out


def gs3_adam_step(param, grad, m, v, lr: float, beta1: float, beta2: float, eps: float, step: int,
                  lower_bound: float, stream: int) -> None:
    n = param.numel()
    assert grad.numel() == n and m.numel() == n and v.numel() == n
    _check(lib().gs3_adam_step(_ptr(param), _ptr(grad), _ptr(m), _ptr(v), n, lr, beta1, beta2, eps, step,
                               lower_bound, stream), "gs3_adam_step")


def gs3_environment_workspace_size(n: int, width: int, height: int, count: int, key_capacity: int) -> int:
    return int(lib().gs3_environment_workspace_size(n, width, height, count, key_capacity))


def gs3_render_environment(scene, camera: gs3_camera, lights, weights, opts: gs3_render_opts, out_rgb,
                           workspace, key_capacity: int, stream: int) -> None:
    n = len(lights)
    la = (gs3_light * max(n, 1))(*lights)
    wa = (C.c_float * max(n, 1))(*[float(w) for w in weights])
    _check(lib().gs3_render_environment(scene, C.byref(camera), la, wa, n, C.byref(opts), _ptr(out_rgb),
                                        _ptr(workspace), workspace.numel() * workspace.element_size(),
                                        key_capacity, stream),
           "gs3_render_environment")


def gs3_render(scene, camera: gs3_camera, light: gs3_light, opts: gs3_render_opts, out_rgb,
               workspace, key_capacity: int, stream: int) -> None:
    _check(lib().gs3_render(scene, C.byref(camera), C.byref(light), C.byref(opts), _ptr(out_rgb),
                            _ptr(workspace), workspace.numel() * workspace.element_size(),
                            key_capacity, stream), "gs3_render")


def gs3_render_stages(scene, camera: gs3_camera, light: gs3_light, opts: gs3_render_opts, out_rgb,
                      workspace, key_capacity: int, stages: int, stream: int) -> None:
    _check(lib().gs3_render_stages(scene, C.byref(camera), C.byref(light), C.byref(opts),
                                   _ptr(out_rgb), _ptr(workspace),
                                   workspace.numel() * workspace.element_size(), key_capacity,
                                   stages, stream), "gs3_render_stages")


def gs3_loss_scratch_size(width: int, height: int) -> int:
    return int(lib().gs3_loss_scratch_size(width, height))


def gs3_loss_l1_dssim(img, target, lam: float, loss_out, dimg_out, scratch, stream: int) -> None:
    h, w = img.shape[0], img.shape[1]
    _check(lib().gs3_loss_l1_dssim(_ptr(img), _ptr(target), w, h, lam, _ptr(loss_out), _ptr(dimg_out),
                                   _ptr(scratch), scratch.numel() * scratch.element_size(), stream),
           "gs3_loss_l1_dssim")


def gs3_backward_workspace_size(scene) -> int:
    return int(lib().gs3_backward_workspace_size(scene))


def gs3_render_backward(scene, camera: gs3_camera, light: gs3_light, opts: gs3_render_opts, dl_drgb,
                        workspace, key_capacity: int, bwd_ws, grads: dict, stream: int) -> None:
    g = gs3_grads(*[_ptr(grads[f]) for f in GRAD_FIELDS])
    _check(lib().gs3_render_backward(scene, C.byref(camera), C.byref(light), C.byref(opts),
                                     _ptr(dl_drgb), _ptr(workspace),
                                     workspace.numel() * workspace.element_size(), key_capacity,
                                     _ptr(bwd_ws), bwd_ws.numel() * bwd_ws.element_size(),
                                     C.byref(g), stream), "gs3_render_backward")


def gs3_workspace_read_header(workspace, stream: int) -> gs3_ws_header:
    h = gs3_ws_header()
    _check(lib().gs3_workspace_read_header(_ptr(workspace), C.byref(h), stream),
           "gs3_workspace_read_header")
    return h


def gs3_server_create(hbm_budget: int, max_inflight: int, device: int = 0,
                      inject_alloc_failures: int = 0, initial_pairs: float = 0.0, max_batch: int = 0,
                      light_cache: int = 0):
    out = _SERVER_P()
    o = gs3_server_opts(hbm_budget, max_inflight, device, inject_alloc_failures, initial_pairs, max_batch,
                        light_cache)
    _check(lib().gs3_server_create(C.byref(o), C.byref(out)), "gs3_server_create")
    return out


def gs3_server_add_scene(server, scene) -> int:
    sid = C.c_int32()
    _check(lib().gs3_server_add_scene(server, scene, C.byref(sid)), "gs3_server_add_scene")
    return sid.value


def gs3_server_submit(server, scene_id: int, camera: gs3_camera, light: gs3_light,
                      opts: gs3_render_opts, out_rgb) -> int:
    t = C.c_uint64()
    _check(lib().gs3_server_submit(server, scene_id, C.byref(camera), C.byref(light), C.byref(opts),
                                   _ptr(out_rgb), C.byref(t)), "gs3_server_submit")
    return t.value


def gs3_server_poll(server, ticket: int):
    """(state, latency_ms, status); never raises for a failed request."""
    st = C.c_int32()
    lat = C.c_double()
    rc = lib().gs3_server_poll(server, ticket, C.byref(st), C.byref(lat))
    if rc == GS3_ERR_INVALID_ARG and st.value == 0:
        _check(rc, "gs3_server_poll")
    return st.value, lat.value, rc


def gs3_server_wait(server, ticket: int, timeout_s: float = 60.0):
    """(status, latency_ms)."""
    lat = C.c_double()
    rc = lib().gs3_server_wait(server, ticket, timeout_s, C.byref(lat))
    return rc, lat.value


def gs3_server_stats(server) -> gs3_server_counters:
    out = gs3_server_counters()
    _check(lib().gs3_server_stats(server, C.byref(out)), "gs3_server_stats")
    return out


def gs3_server_reset_counters(server) -> None:
    _check(lib().gs3_server_reset_counters(server), "gs3_server_reset_counters")


def gs3_server_destroy(server) -> None:
    _check(lib().gs3_server_destroy(server), "gs3_server_destroy")


GS3_STATIC_SORT_MAX_KEYS = 1048576


def gs3_depth_order_static(keys, n: int, order_out, stream: int) -> None:
    _check(lib().gs3_depth_order_static(_ptr(keys), n, _ptr(order_out), stream),
           "gs3_depth_order_static")


def gs3_selftest_wait_timeout(n: int) -> int:
    """The status word of a look-back sort pass whose waits can never end."""
    out = C.c_uint32(0)
    _check(lib().gs3_selftest_wait_timeout(n, C.byref(out)), "gs3_selftest_wait_timeout")
    return int(out.value)


def gs3_selftest_shadow_wait(scene, cam, light, opts, workspace, ws_bytes: int, cap: int) -> int:
    """The workspace status after a shadow chain whose predecessors never publish."""
    out = C.c_uint32(0)
    _check(lib().gs3_selftest_shadow_wait(scene, C.byref(cam), C.byref(light), C.byref(opts), _ptr(workspace),
                                          ws_bytes, cap, C.byref(out)), "gs3_selftest_shadow_wait")
    return int(out.value)


def gs3_measure_alu_peak(repeats: int = 5):
    """(FP32 FMA TFLOP/s, ex2 G ops/s) of the current device, measured."""
    f, x = C.c_double(0.0), C.c_double(0.0)
    _check(lib().gs3_measure_alu_peak(repeats, C.byref(f), C.byref(x)), "gs3_measure_alu_peak")
    return float(f.value), float(x.value)


def gs3_kernel_launches() -> int:
    return int(lib().gs3_kernel_launches())


def gs3_last_error() -> str:
    return lib().gs3_last_error().decode()
