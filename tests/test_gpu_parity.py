"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Integer work (keys, rectangles, tile lists, sort order, ranges) must match
bit for bit.  Floating-point outputs must satisfy
    |gpu - oracle| <= 1e-4 |oracle| + 1e-6 + bound
per value, where `bound` is the oracle's explicit bound for decisions whose
FP64 operand lies within a relative 1e-5 of a threshold (alpha vs 1/255,
T vs 1e-4); it is zero for every other value.
"""
import json
import os

import numpy as np
import pytest

from paper_2410_11419_gb300 import synth

pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-4, 1e-6


def run_both(gs3, oracle, scene, cam, light, ablate=0, cap=1 << 20, falloff=1, fr=None, mlp_dtype=0):
    """The GPU frame's stages (through the C ABI) and the oracle frame (`fr`
    when given, else rendered here)."""
    import torch
    from paper_2410_11419_gb300 import render as R
    ds = R.DeviceScene(scene, mlp_dtype=mlp_dtype)
    rd = R.Renderer(ds, cam.width, cam.height, cap)
    img = rd.render(cam, light, R.opts_struct(ablate=ablate, falloff=falloff))
    torch.cuda.synchronize()
    hdr = rd.check()
    g = {k: rd.stage(k, s).cpu().numpy() for k, s in
         (("key", 0), ("order", 0), ("tile_start", 0), ("rect", 0), ("shade", 0), ("T", 0),
          ("Tp", 0), ("res", 0), ("final_t", 0), ("n_contrib", 0))}
    for nm, s in (("lkey", 1), ("lorder", 1), ("ltile_start", 1), ("lrect", 1)):
        g[nm] = rd.stage(nm[1:], s).cpu().numpy()
    g["list"] = rd.stage("list", 0)[:hdr.pairs_cam].cpu().numpy()
    g["llist"] = rd.stage("list", 1)[:hdr.pairs_light].cpu().numpy()
    g["img"] = img.cpu().numpy()
    g["light_final"] = rd.stage("light_final").cpu().numpy()
    g["light_stop"] = rd.stage("light_stop").cpu().numpy().view(np.uint32)
    g["hdr"] = hdr
    if fr is None:
        fr = oracle.render(scene, cam, light, oracle.Opts(ablate=ablate, falloff=falloff))
    ds.close()
    return g, fr


def _record(name, err, want, bound):
    """Append error statistics to $GS3_PARITY_STATS (JSON lines) when set."""
    path = os.environ.get("GS3_PARITY_STATS")
    if not path:
        return
    rel = err / np.maximum(np.abs(want), 1e-6)
    amb = np.asarray(bound) > 0 if np.ndim(bound) else np.zeros(err.shape, bool)
    with open(path, "a") as fh:
        fh.write(json.dumps({"test": os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0],
                             "output": name, "count": int(err.size),
                             "max_abs": float(err.max()) if err.size else 0.0,
                             "max_rel": float(rel.max()) if err.size else 0.0,
                             "mean_rel": float(rel.mean()) if err.size else 0.0,
                             "bounded": int(amb.sum())}) + "\n")


def assert_close(name, got, want, bound=0.0):
    err = np.abs(got - want)
    tol = RTOL * np.abs(want) + ATOL + bound
    _record(name, err, want, bound)
    bad = err > tol
    assert not bad.any(), (f"{name}: {bad.sum()} of {bad.size} outside tolerance; worst err "
                           f"{err[bad].max():.3e} at want {want[bad][np.argmax(err[bad])]:.6g}")


def check_integer_stages(g, fr):
    """Keys, rectangles, per-tile lists and ranges: bit-exact."""
    for gs, os_, nm in ((("key", "rect", "tile_start", "list", "order"), "cam", "camera"),
                        (("lkey", "lrect", "ltile_start", "llist", "lorder"), "light", "light")):
        gk, gr, gts, gl, go = (g[x] for x in gs)
        np.testing.assert_array_equal(gk.view(np.uint32), fr[f"{os_}_key"], err_msg=f"{nm} keys")
        vis = fr[f"{os_}_rect"][:, 0] >= 0
        np.testing.assert_array_equal(gr[vis], fr[f"{os_}_rect"][vis], err_msg=f"{nm} rects")
        assert np.all(gr[~vis][:, 0] < 0)
        np.testing.assert_array_equal(gts.view(np.uint32), fr[f"{os_}_tile_start"], err_msg=f"{nm} ranges")
        idx = go.view(np.uint32)[gl.view(np.uint32)]
        np.testing.assert_array_equal(idx, fr[f"{os_}_list"], err_msg=f"{nm} lists")


def check_float_stages(g, fr, expect_shadow=True):
    assert_close("shade", g["shade"][:, :3].astype(np.float64), fr["shade"])
    assert_close("shadow T", g["T"].astype(np.float64), fr["T"], fr["T_bound"])
    assert_close("refined T'", g["Tp"].astype(np.float64), fr["Tp"], fr["Tp_bound"])
    assert_close("residual", g["res"][:, :3].astype(np.float64), fr["res"])
    amb = fr["img_bound"].max(axis=2) > 0
    assert_close("image", g["img"].astype(np.float64), fr["img"], fr["img_bound"])
    ok = ~amb
    assert_close("final T", g["final_t"][ok].astype(np.float64), fr["final_T"][ok])
    np.testing.assert_array_equal(g["n_contrib"][ok], fr["n_contrib"][ok])
    if expect_shadow:
        assert fr["T"].min() < 0.95


CASES = [
    # (name, scene factory, seed, width, height)
    ("tiny_128", lambda: synth.tiny_scene(0), 0, 128, 128),
    ("tiny_ragged", lambda: synth.tiny_scene(0), 3, 120, 88),
    ("ball_3k_k8", lambda: synth.make_scene(5, 3000, 8, "ball"), 5, 200, 152),
    ("shell_20k", lambda: synth.object_scene(2, n=20000), 7, 256, 256),
    ("paper_mlp", lambda: synth.paper_mlp_scene(1, n=2000), 11, 160, 144),
    # 1444 tiles: lists in the second buffer pair
    ("ball_3k_608", lambda: synth.make_scene(6, 3000, 4, "ball"), 13, 608, 608),
    # 16641 tiles, 129 columns: binning chunks of 512 row items (two steps of 256)
    ("tiny_2064", lambda: synth.tiny_scene(0), 17, 2064, 2064),
    # one tile row of 129 columns, and one tile column of 65 rows
    ("strip_wide", lambda: synth.tiny_scene(0), 19, 2064, 16),
    ("strip_tall", lambda: synth.tiny_scene(0), 23, 16, 1040),
]


@pytest.mark.parametrize("name,make,seed,w,h", CASES, ids=[c[0] for c in CASES])
def test_frame_parity(gs3, oracle, name, make, seed, w, h):
    scene = make()
    cam, light = synth.camera_light_pair(seed, w, h)
    g, fr = run_both(gs3, oracle, scene, cam, light)
    assert g["hdr"].pairs_cam == fr["cam_P"] and g["hdr"].pairs_light == fr["light_P"]
    check_integer_stages(g, fr)
    check_float_stages(g, fr)


@pytest.mark.parametrize("seed,w,h", [(30, 16384, 16), (34, 16, 16384)], ids=["wide_16384", "tall_16384"])
def test_maximum_image_sides(gs3, oracle, seed, w, h):
    """The largest image side (16384 pixels, 1024 tiles): one tile row of
    1024 columns (the binning's widest placement and 2048-item chunks), and
    one tile column of 1024 rows (the row pass's widest placement, a plan
    block with every thread a row); 90 degrees along the long side."""
    import math
    fov = 90.0 if h > w else math.degrees(2 * math.atan(h / w))
    cam, light = synth.camera_light_pair(seed, w, h, fov_y_deg=fov)
    g, fr = run_both(gs3, oracle, synth.tiny_scene(0), cam, light)
    assert g["hdr"].pairs_cam == fr["cam_P"] > 0 and g["hdr"].pairs_light == fr["light_P"] > 0
    check_integer_stages(g, fr)
    check_float_stages(g, fr)


@pytest.mark.parametrize("ablate", [1, 2, 4, 7, 8])
def test_ablations(gs3, oracle, ablate):
    scene = synth.tiny_scene(0)
    cam, light = synth.camera_light_pair(1, 96, 96)
    g, fr = run_both(gs3, oracle, scene, cam, light, ablate=ablate)
    check_integer_stages(g, fr) if not (ablate & 1) else None
    check_float_stages(g, fr, expect_shadow=not (ablate & 1))


def test_no_falloff(gs3, oracle):
    scene = synth.tiny_scene(0)
    cam, light = synth.camera_light_pair(2, 64, 64)
    g, fr = run_both(gs3, oracle, scene, cam, light, falloff=0)
    check_float_stages(g, fr)


def test_single_gaussian(gs3, oracle):
    from tests.test_oracle_pins import one_gaussian_scene
    sc = one_gaussian_scene([0.0, 0.0, 0.0], 0.04, logit=1.5, k=2)
    cam = synth.look_at_camera([0.0, 0.0, 3.0], width=64, height=64)
    light = synth.Light(pos=np.array([0.0, 2.5, 1.0], dtype=np.float32), intensity=10.0)
    g, fr = run_both(gs3, oracle, sc, cam, light)
    check_integer_stages(g, fr)
    check_float_stages(g, fr, expect_shadow=False)
    assert g["T"][0] == 1.0


def test_everything_culled(gs3, oracle):
    """Camera looking away from the scene: empty lists, black image, T from the light."""
    scene = synth.tiny_scene(0)
    cam = synth.look_at_camera([0.0, 0.0, 3.0], target=(0.0, 0.0, 6.0), width=64, height=48)
    _, light = synth.camera_light_pair(0, 64, 48)
    g, fr = run_both(gs3, oracle, scene, cam, light)
    assert g["hdr"].pairs_cam == 0
    check_integer_stages(g, fr)
    assert np.all(g["img"] == 0.0)
    assert np.all(g["final_t"] == 1.0)


def test_capacity_overflow_reported(gs3):
    """Too small a key capacity is reported in the workspace status word."""
    import torch
    from paper_2410_11419_gb300 import render as R, _native as N
    scene = synth.tiny_scene(0)
    cam, light = synth.camera_light_pair(0, 128, 128)
    ds = R.DeviceScene(scene)
    rd = R.Renderer(ds, 128, 128, 1000)
    rd.render(cam, light)
    torch.cuda.synchronize()
    h = rd.header()
    assert h.status == N.GS3_ERR_CAPACITY
    assert h.pairs_cam_needed > 1000
    with pytest.raises(N.GS3Error):
        rd.check()
    # a large enough workspace renders the same scene fine afterwards
    rd2 = R.Renderer(ds, 128, 128, h.pairs_cam_needed + h.pairs_light_needed)
    rd2.render(cam, light)
    rd2.check()


@pytest.mark.parametrize("mlp_dtype", [0, 1], ids=["fp32", "bf16"])
def test_moving_camera_fixed_light(gs3, mlp_dtype):
    """The shadow values depend on the scene, the light and the image size,
    not on the camera: after a full frame, the camera-side stages alone render
    another view under the same light bit for bit as its full frame."""
    import torch
    from paper_2410_11419_gb300 import render as R, _native as N
    scene = synth.make_scene(5, 3000, 8, "ball")
    cam_a, light = synth.camera_light_pair(5, 200, 152)
    views = [synth.camera_light_pair(s, 200, 152)[0] for s in (8, 9)]
    ds = R.DeviceScene(scene, mlp_dtype=mlp_dtype)
    moving = R.Renderer(ds, 200, 152, 1 << 20)
    full = R.Renderer(ds, 200, 152, 1 << 20)
    moving.render(cam_a, light)
    cam_side = N.GS3_STAGE_PREP | N.GS3_STAGE_CAMERA_BIN | N.GS3_STAGE_MLP | N.GS3_STAGE_CAMERA
    for cam in views:
        got = moving.render_stages(cam, light, cam_side).clone()
        want = full.render(cam, light).clone()
        torch.cuda.synchronize()
        moving.check()
        full.check()
        assert torch.equal(got, want)
        assert torch.equal(moving.stage("Tp"), full.stage("Tp"))
    # only T carries over: a workspace whose other light-side buffers hold
    # another light's frame gives the same image once T is the right one
    other = R.Renderer(ds, 200, 152, 1 << 20)
    other.render(cam_a, synth.camera_light_pair(6, 200, 152)[1])
    full.render(cam_a, light)
    other.stage("T").copy_(full.stage("T"))
    got = other.render_stages(views[0], light, cam_side).clone()
    want = full.render(views[0], light).clone()
    torch.cuda.synchronize()
    other.check()
    assert torch.equal(got, want)
    ds.close()


def test_bounded_wait_gives_up(gs3):
    """A look-back wait that can never end (its predecessor's words are never
    written) gives up, records GS3_ERR_TIMEOUT, and the context still renders."""
    import time
    import torch
    from paper_2410_11419_gb300 import render as R, _native as N
    t0 = time.perf_counter()
    assert N.gs3_selftest_wait_timeout(3 * 4096) == N.GS3_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 30.0
    with pytest.raises(N.GS3Error):
        N.gs3_selftest_wait_timeout(4096)  # one block: nothing to wait on, rejected
    scene = synth.tiny_scene(0)
    cam, light = synth.camera_light_pair(0, 128, 128)
    rd = R.Renderer(R.DeviceScene(scene), 128, 128, 1 << 20)
    rd.render(cam, light)
    torch.cuda.synchronize()
    rd.check()


def test_invalid_arguments_rejected(gs3):
    from paper_2410_11419_gb300 import render as R, _native as N
    scene = synth.tiny_scene(0)
    ds = R.DeviceScene(scene)
    cam, light = synth.camera_light_pair(0, 64, 64)
    rd = R.Renderer(ds, 64, 64, 1 << 16)
    o = R.opts_struct()
    o.tile = 8
    with pytest.raises(N.GS3Error) as e:
        rd.render(cam, light, o)
    assert e.value.status == N.GS3_ERR_INVALID_ARG
    bad = synth.tiny_scene(0)
    bad.phi.in_dim = 50
    with pytest.raises(N.GS3Error):
        R.DeviceScene(bad)


def test_deterministic_repeat(gs3):
    """Two renders of the same frame are bitwise identical (no atomics in any sum)."""
    import torch
    from paper_2410_11419_gb300 import render as R
    scene = synth.make_scene(4, 5000, 4, "shell")
    cam, light = synth.camera_light_pair(4, 160, 160)
    ds = R.DeviceScene(scene)
    rd = R.Renderer(ds, 160, 160, 1 << 21)
    a = rd.render(cam, light).clone()
    ta = rd.stage("T").clone()
    b = rd.render(cam, light).clone()
    torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(ta, rd.stage("T"))


def test_overlapped_frame_equals_staged(gs3):
    """A whole gs3_render runs the light chain on a side stream beside the
    camera binning; the frame equals the same frame rendered stage by stage
    on one stream, bit for bit (the two chains share no buffer)."""
    import torch
    from paper_2410_11419_gb300 import _native as N, render as R
    scene = synth.object_scene(3, n=20000)
    cam, light = synth.camera_light_pair(9, 256, 256)
    ds = R.DeviceScene(scene)
    rd = R.Renderer(ds, 256, 256, 1 << 22)
    whole = rd.render(cam, light).clone()
    staged = torch.empty_like(whole)
    for st in (N.GS3_STAGE_PREP, N.GS3_STAGE_CAMERA_BIN, N.GS3_STAGE_LIGHT_BIN, N.GS3_STAGE_SHADOW_COMPOSITE,
               N.GS3_STAGE_SHADOW_REDUCE, N.GS3_STAGE_MLP, N.GS3_STAGE_CAMERA):
        rd.render_stages(cam, light, st, out=staged)
    torch.cuda.synchronize()
    rd.check()
    assert torch.equal(whole, staged)
    ds.close()
