"""ctypes binding of the FP64 CPU oracle (gs3_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the library.  It takes scenes, cameras
and lights as plain objects with the attribute names of the seeded generator
(duck-typed; nothing here imports the library package).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gs3_oracle.c")
LIB = os.path.join(HERE, "libgs3_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with IEEE FP32 semantics for the key recipe."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-fopenmp", "-D_GNU_SOURCE", SRC, "-o", LIB + ".tmp", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


class _MLP(C.Structure):
    _fields_ = [("in_dim", C.c_int), ("width", C.c_int), ("n_hidden", C.c_int),
                ("out_dim", C.c_int), ("act", C.c_int),
                ("w", C.POINTER(C.c_float)), ("b", C.POINTER(C.c_float))]


_FP = C.POINTER(C.c_float)


class _Scene(C.Structure):
    _fields_ = [("n", C.c_int), ("k", C.c_int)] + [
        (a, _FP) for a in ("mean_op", "scale", "rot", "shade_rot", "albedo_d", "albedo_s",
                           "latent", "lobe_rot", "lobe_sigma", "lobe_amp")] + [
        ("phi", _MLP), ("psi", _MLP), ("lobe_shared", C.c_int)]


class _Camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("pos", C.c_float * 3),
                ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("width", C.c_int), ("height", C.c_int)]


class _Light(C.Structure):
    _fields_ = [("pos", C.c_float * 3), ("intensity", C.c_float), ("type", C.c_int),
                ("dir", C.c_float * 3), ("extent", C.c_float)]


class _Opts(C.Structure):
    _fields_ = [("near_z", C.c_float), ("lowpass", C.c_float), ("frustum", C.c_float),
                ("shadow_bias", C.c_float), ("alpha_min", C.c_float), ("alpha_max", C.c_float),
                ("t_stop", C.c_float), ("target", C.c_float * 3), ("falloff", C.c_int),
                ("tile", C.c_int), ("ablate", C.c_int), ("threads", C.c_int),
                ("margin_alpha", C.c_double), ("margin_tstop", C.c_double),
                ("crop", C.c_int * 4), ("flip", C.POINTER(C.c_int64)), ("nflip", C.c_int),
                ("record_amb", C.c_int)]


_U32 = C.POINTER(C.c_uint32)
_I32 = C.POINTER(C.c_int32)
_D = C.POINTER(C.c_double)


class _Frame(C.Structure):
    _fields_ = [("n", C.c_int), ("width", C.c_int), ("height", C.c_int), ("gx", C.c_int),
                ("gy", C.c_int), ("ntiles", C.c_int), ("light_R", C.c_float * 9),
                ("light_t", C.c_float * 3), ("light_ortho", C.c_float),
                ("key", _U32 * 2), ("rect", _I32 * 2), ("uv_f32", _FP * 2), ("uv", _D * 2),
                ("conic", _D * 2), ("opacity", _D), ("P", C.c_uint32 * 2),
                ("tile_start", _U32 * 2), ("list", _U32 * 2),
                ("shade", _D), ("T", _D), ("T_bound", _D), ("Tp", _D), ("Tp_bound", _D),
                ("res", _D), ("img", _D), ("img_bound", _D), ("final_T", _D),
                ("n_contrib", _I32), ("S", _D), ("Sh", _D), ("Rimg", _D),
                ("shadow_evals", C.c_int64), ("shadow_pass", C.c_int64),
                ("camera_evals", C.c_int64), ("amb_shadow", C.c_int64),
                ("amb_camera", C.c_int64), ("camera_pass", C.c_int64), ("t_prep", C.c_double), ("t_bin", C.c_double),
                ("t_shadow", C.c_double), ("t_mlp", C.c_double), ("t_camera", C.c_double),
                ("amb", C.POINTER(C.c_int64)), ("namb", C.c_int64), ("amb_cap", C.c_int64),
                ("sacc", _D), ("wi", _D), ("wo", _D)]

# kinds of decision-ambiguous cases (the top bits of a decision code)
AMB_SHADOW_ALPHA, AMB_CAMERA_ALPHA, AMB_CAMERA_STOP = 0, 1, 2


def amb_code(kind: int, pixel: int, pos: int) -> int:
    return (kind << 60) | (pixel << 32) | pos


def amb_split(codes: np.ndarray):
    """(kind, pixel, list position) of decision codes."""
    codes = np.asarray(codes, dtype=np.int64)
    return codes >> 60, (codes >> 32) & ((1 << 28) - 1), codes & 0xFFFFFFFF


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.go_render.restype = C.POINTER(_Frame)
        _lib.go_render.argtypes = [C.POINTER(_Scene), C.POINTER(_Camera), C.POINTER(_Light),
                                   C.POINTER(_Opts)]
        _lib.go_frame_free.argtypes = [C.POINTER(_Frame)]
        _lib.go_begin.restype = C.POINTER(_Frame)
        _lib.go_begin.argtypes = [C.POINTER(_Scene), C.POINTER(_Camera), C.POINTER(_Light),
                                  C.POINTER(_Opts)]
        _lib.go_shadow_rows.argtypes = [C.POINTER(_Frame), C.POINTER(_Opts), C.c_int, C.c_int]
        _lib.go_finish.argtypes = [C.POINTER(_Frame), C.POINTER(_Scene), C.POINTER(_Opts)]
        _lib.go_diffuse.restype = C.c_double
        _lib.go_diffuse.argtypes = [C.c_double]
        _lib.go_angular_gaussian.restype = C.c_double
        _lib.go_angular_gaussian.argtypes = [_D, _FP, _D]
        _lib.go_mlp_eval.argtypes = [C.POINTER(_MLP), C.c_int, _D, _D]
        _lib.go_shade.argtypes = [C.POINTER(_Scene), C.c_int, C.POINTER(_Camera),
                                  C.POINTER(_Light), C.POINTER(_Opts), _D]
        _lib.go_key_recipe.restype = C.c_int
        _lib.go_key_recipe.argtypes = [_FP, _FP, _FP, _FP, _FP, C.c_float, C.c_float, C.c_float,
                                       C.c_float, C.c_int, C.c_int, C.POINTER(_Opts), _FP, C.c_float,
                                       _U32, _I32, _FP]
        _lib.go_project.argtypes = [_FP, _FP, _FP, _FP, _FP, C.c_double, C.c_double, C.c_double,
                                    C.c_double, C.c_double, C.c_double, _D, _D]
        _lib.go_light_view_any.restype = C.c_float
        _lib.go_light_view_any.argtypes = [C.POINTER(_Light), _FP, C.c_int, C.c_int, _FP, _FP]
        _lib.go_pos_enc.restype = C.c_int
        _lib.go_pos_enc.argtypes = [_D, _D]
        _lib.go_light_view.argtypes = [_FP, _FP, _FP, _FP]
        _lib.go_max_threads.restype = C.c_int
    return _lib


@dataclass
class Opts:
    """Render options (the paper's constants and the readings of its silent points)."""
    near_z: float = 0.2
    lowpass: float = 0.3
    frustum: float = 1.3
    shadow_bias: float = 0.015
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    t_stop: float = 1e-4
    target: tuple = (0.0, 0.0, 0.0)
    falloff: int = 1
    tile: int = 16
    ablate: int = 0
    threads: int = 0
    margin_alpha: float = 1e-5
    margin_tstop: float = 1e-4
    crop: tuple = (0, 0, 0, 0)
    flip: tuple = ()       # decision codes to take on their other side (testing the bounds)
    record_amb: int = 0    # 1: return the codes of every ambiguous decision as "amb"

    def c(self) -> _Opts:
        o = _Opts()
        for f, _ in _Opts._fields_:
            if f == "nflip":
                continue
            v = getattr(self, f)
            if f == "target":
                o.target = (C.c_float * 3)(*v)
            elif f == "crop":
                o.crop = (C.c_int * 4)(*v)
            elif f == "flip":
                codes = np.unique(np.asarray(v, dtype=np.int64))
                self._flip_keep = np.ascontiguousarray(codes)
                o.flip = self._flip_keep.ctypes.data_as(C.POINTER(C.c_int64)) if codes.size else None
                o.nflip = int(codes.size)
            else:
                setattr(o, f, v)
        return o


def _fp(a: np.ndarray):
    assert a.dtype == np.float32 and a.flags.c_contiguous
    return a.ctypes.data_as(_FP)


def _mlp(m, keep: list) -> _MLP:
    w = np.ascontiguousarray(np.concatenate([x.reshape(-1) for x in m.weights]), dtype=np.float32)
    b = np.ascontiguousarray(np.concatenate([x.reshape(-1) for x in m.biases]), dtype=np.float32)
    keep += [w, b]
    return _MLP(m.in_dim, m.width, m.n_hidden, m.out_dim, m.act, _fp(w), _fp(b))


def c_scene(scene, keep: list) -> _Scene:
    s = _Scene()
    s.n, s.k = scene.n, scene.k
    for a in ("mean_op", "scale", "rot", "shade_rot", "albedo_d", "albedo_s", "latent",
              "lobe_rot", "lobe_sigma", "lobe_amp"):
        arr = np.ascontiguousarray(getattr(scene, a), dtype=np.float32)
        if arr.size == 0:
            arr = np.zeros(4, dtype=np.float32)
        keep.append(arr)
        setattr(s, a, _fp(arr))
    s.phi = _mlp(scene.phi, keep)
    s.psi = _mlp(scene.psi, keep)
    s.lobe_shared = int(getattr(scene, "lobe_shared", False))
    return s


def c_camera(cam) -> _Camera:
    c = _Camera()
    c.R = (C.c_float * 9)(*np.asarray(cam.R, dtype=np.float32).reshape(-1).tolist())
    c.t = (C.c_float * 3)(*np.asarray(cam.t, dtype=np.float32).tolist())
    c.pos = (C.c_float * 3)(*np.asarray(cam.pos, dtype=np.float32).tolist())
    c.fx, c.fy, c.cx, c.cy = cam.fx, cam.fy, cam.cx, cam.cy
    c.width, c.height = cam.width, cam.height
    return c


def c_light(light) -> _Light:
    d = getattr(light, "dir", None)
    d = (0.0, 0.0, 0.0) if d is None else np.asarray(d, dtype=np.float32).tolist()
    return _Light((C.c_float * 3)(*np.asarray(light.pos, dtype=np.float32).tolist()),
                  float(light.intensity), int(getattr(light, "type", 0)), (C.c_float * 3)(*d),
                  float(getattr(light, "extent", 0.0)))


def _arr(ptr, n, dtype):
    if n == 0:
        return np.zeros(0, dtype=dtype)
    return np.ctypeslib.as_array(ptr, shape=(n,)).astype(dtype, copy=True)


def render(scene, cam, light, opts: Opts | None = None) -> dict:
    """Run the whole oracle frame; returns NumPy copies of every stage."""
    opts = opts or Opts()
    keep: list = []
    sc = c_scene(scene, keep)
    cc, lc, oc = c_camera(cam), c_light(light), opts.c()
    fp = lib().go_render(C.byref(sc), C.byref(cc), C.byref(lc), C.byref(oc))
    return _collect(fp)


class StagedFrame:
    """One oracle frame run stage by stage (the arithmetic of render(), for
    timing the stages apart): construction runs O1-O8 (shading, projections,
    lists), shadow_rows(y0, y1) the shadow rays of light-view rows [y0, y1)
    (each row once), finish() the per-Gaussian shadow average, Phi, Psi and
    the camera composite, and returns what render() returns."""

    def __init__(self, scene, cam, light, opts: Opts | None = None):
        self.opts = opts or Opts()
        self.keep: list = []
        self.sc = c_scene(scene, self.keep)
        self.cc, self.lc, self.oc = c_camera(cam), c_light(light), self.opts.c()
        self.fp = lib().go_begin(C.byref(self.sc), C.byref(self.cc), C.byref(self.lc), C.byref(self.oc))
        self.height = cam.height

    def shadow_rows(self, y0: int, y1: int):
        lib().go_shadow_rows(self.fp, C.byref(self.oc), int(y0), int(y1))

    def finish(self) -> dict:
        lib().go_finish(self.fp, C.byref(self.sc), C.byref(self.oc))
        fp, self.fp = self.fp, None
        return _collect(fp)


def _collect(fp) -> dict:
    f = fp.contents
    n, W, H, nt = f.n, f.width, f.height, f.ntiles
    out = {"n": n, "width": W, "height": H, "gx": f.gx, "gy": f.gy, "ntiles": nt,
           "light_R": np.array(f.light_R[:], dtype=np.float32).reshape(3, 3),
           "light_t": np.array(f.light_t[:], dtype=np.float32),
           "light_ortho": float(f.light_ortho)}
    for s, nm in ((0, "cam"), (1, "light")):
        P = int(f.P[s])
        out[f"{nm}_key"] = _arr(f.key[s], n, np.uint32)
        out[f"{nm}_rect"] = _arr(f.rect[s], 4 * n, np.int32).reshape(n, 4)
        out[f"{nm}_uv_f32"] = _arr(f.uv_f32[s], 2 * n, np.float32).reshape(n, 2)
        out[f"{nm}_uv"] = _arr(f.uv[s], 2 * n, np.float64).reshape(n, 2)
        out[f"{nm}_conic"] = _arr(f.conic[s], 3 * n, np.float64).reshape(n, 3)
        out[f"{nm}_P"] = P
        out[f"{nm}_tile_start"] = _arr(f.tile_start[s], nt + 1, np.uint32)
        out[f"{nm}_list"] = _arr(f.list[s], P, np.uint32)
    np_ = W * H
    out.update(
        opacity=_arr(f.opacity, n, np.float64),
        shade=_arr(f.shade, 3 * n, np.float64).reshape(n, 3),
        T=_arr(f.T, n, np.float64), T_bound=_arr(f.T_bound, n, np.float64),
        Tp=_arr(f.Tp, n, np.float64), Tp_bound=_arr(f.Tp_bound, n, np.float64),
        res=_arr(f.res, 3 * n, np.float64).reshape(n, 3),
        img=_arr(f.img, 3 * np_, np.float64).reshape(H, W, 3),
        img_bound=_arr(f.img_bound, 3 * np_, np.float64).reshape(H, W, 3),
        final_T=_arr(f.final_T, np_, np.float64).reshape(H, W),
        n_contrib=_arr(f.n_contrib, np_, np.int32).reshape(H, W),
        S=_arr(f.S, 3 * np_, np.float64).reshape(H, W, 3),
        Sh=_arr(f.Sh, np_, np.float64).reshape(H, W),
        R=_arr(f.Rimg, 3 * np_, np.float64).reshape(H, W, 3),
        shadow_evals=f.shadow_evals, shadow_pass=f.shadow_pass, camera_evals=f.camera_evals,
        amb_shadow=f.amb_shadow, amb_camera=f.amb_camera, camera_pass=f.camera_pass,
        times={"prep": f.t_prep, "bin": f.t_bin, "shadow": f.t_shadow, "mlp": f.t_mlp,
               "camera": f.t_camera},
        amb=np.sort(_arr(f.amb, int(f.namb), np.int64)),
    )
    lib().go_frame_free(fp)
    return out


def max_threads() -> int:
    return int(lib().go_max_threads())


def diffuse(x: float) -> float:
    return lib().go_diffuse(float(x))


def angular_gaussian(h, q, sig) -> float:
    h = np.ascontiguousarray(h, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float32)
    s = np.ascontiguousarray(sig, dtype=np.float64)
    return lib().go_angular_gaussian(h.ctypes.data_as(_D), _fp(q), s.ctypes.data_as(_D))


def mlp_eval(m, x: np.ndarray) -> np.ndarray:
    keep: list = []
    cm = _mlp(m, keep)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros((x.shape[0], m.out_dim), dtype=np.float64)
    lib().go_mlp_eval(C.byref(cm), x.shape[0], x.ctypes.data_as(_D), y.ctypes.data_as(_D))
    return y


def shade(scene, g: int, cam, light, opts: Opts | None = None) -> np.ndarray:
    keep: list = []
    sc = c_scene(scene, keep)
    out = np.zeros(3, dtype=np.float64)
    lib().go_shade(C.byref(sc), g, C.byref(c_camera(cam)), C.byref(c_light(light)),
                   C.byref((opts or Opts()).c()), out.ctypes.data_as(_D))
    return out


def key_recipe(m, s, q, R, t, fx, fy, cx, cy, W, H, opts: Opts | None = None, light_pos=None,
               ortho: float = 0.0):
    """FP32 key recipe of one Gaussian; m = (x, y, z, opacity logit)."""
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    m, s, q, R, t = f32(m), f32(s), f32(q), f32(np.asarray(R).reshape(-1)), f32(t)
    assert m.size == 4, "mean and opacity logit"
    key = C.c_uint32()
    rect = np.zeros(4, dtype=np.int32)
    uv = np.zeros(2, dtype=np.float32)
    pl = _fp(f32(light_pos)) if light_pos is not None else None
    keep = [light_pos]
    vis = lib().go_key_recipe(_fp(m), _fp(s), _fp(q), _fp(R), _fp(t), fx, fy, cx, cy, W, H,
                              C.byref((opts or Opts()).c()), pl, ortho, C.byref(key),
                              rect.ctypes.data_as(_I32), _fp(uv))
    del keep
    return bool(vis), int(key.value), rect, uv


def project(m, s, q, R, t, fx, fy, cx, cy, lowpass=0.3, ortho=0.0):
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    uv = np.zeros(2)
    con = np.zeros(3)
    lib().go_project(_fp(f32(m)), _fp(f32(s)), _fp(f32(q)), _fp(f32(np.asarray(R).reshape(-1))),
                     _fp(f32(t)), fx, fy, cx, cy, lowpass, ortho, uv.ctypes.data_as(_D),
                     con.ctypes.data_as(_D))
    return uv, con


def pos_enc(v) -> np.ndarray:
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.zeros(27)
    lib().go_pos_enc(v.ctypes.data_as(_D), out.ctypes.data_as(_D))
    return out


def environment(scene, cam, lights, weights, opts: Opts | None = None) -> np.ndarray:
    """Sec. 4.5: an environment light as the linear combination
    sum_l w_l render(directional light l) of whole rendered images."""
    out = None
    for L, w in zip(lights, weights):
        img = render(scene, cam, L, opts)["img"]
        out = float(w) * img if out is None else out + float(w) * img
    return out


def light_view_any(light, width, height, target=(0.0, 0.0, 0.0)):
    """(R, t, s) of the light camera: perspective at a point light (s = 0) or
    orthographic along a directional light (s = pixels per world unit)."""
    R = np.zeros(9, dtype=np.float32)
    t = np.zeros(3, dtype=np.float32)
    lc = c_light(light)
    tg = np.ascontiguousarray(target, dtype=np.float32)
    s = lib().go_light_view_any(C.byref(lc), _fp(tg), width, height, _fp(R), _fp(t))
    return R.reshape(3, 3), t, float(s)


def light_view(light_pos, target=(0.0, 0.0, 0.0)):
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    R = np.zeros(9, dtype=np.float32)
    t = np.zeros(3, dtype=np.float32)
    lib().go_light_view(_fp(f32(light_pos)), _fp(f32(target)), _fp(R), _fp(t))
    return R.reshape(3, 3), t


if __name__ == "__main__":
    build(force="--force" in sys.argv)
    print(LIB)
