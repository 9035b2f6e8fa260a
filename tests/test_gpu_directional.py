"""Directional and environment lighting (Sec. 4.5) on the GPU, through the C ABI.

* A directional light's frame against the FP64 oracle: the orthographic light
  view (rotation, translation, pixel scale) equal bit for bit, keys, lists and
  ranges of both splats bit-exact, and the floating-point stages within
  1e-4 relative + 1e-6 + the oracle's decision bounds.
* gs3_render_environment equals the weighted sum of single renders, and the
  oracle's environment image within the summed tolerances.
* The backward of a directional frame against the FP64 gradient oracle.
"""
import numpy as np
import pytest

from paper_2410_11419_gb300 import synth
from tests.test_gpu_parity import assert_close, check_float_stages, check_integer_stages, run_both

pytestmark = pytest.mark.gpu

CASES = [
    ("tiny_128", lambda: synth.tiny_scene(0), 0, 128, 128),
    ("ball_3k_k8", lambda: synth.make_scene(5, 3000, 8, "ball"), 5, 200, 152),
    ("shell_20k", lambda: synth.object_scene(2, n=20000), 7, 256, 256),
]


@pytest.mark.parametrize("name,make,seed,w,h", CASES, ids=[c[0] for c in CASES])
def test_directional_frame_parity(gs3, oracle, name, make, seed, w, h):
    scene = make()
    cam, _ = synth.camera_light_pair(seed, w, h)
    light = synth.directional_light(seed)
    g, fr = run_both(gs3, oracle, scene, cam, light)
    hdr = g["hdr"]
    assert hdr.light_ortho > 0 and np.float32(hdr.light_ortho) == np.float32(fr["light_ortho"])
    np.testing.assert_array_equal(np.array(hdr.light_R[:], dtype=np.float32), fr["light_R"].reshape(-1))
    np.testing.assert_array_equal(np.array(hdr.light_t[:], dtype=np.float32), fr["light_t"])
    assert hdr.pairs_cam == fr["cam_P"] and hdr.pairs_light == fr["light_P"]
    check_integer_stages(g, fr)
    check_float_stages(g, fr)


def test_point_light_header_is_perspective(gs3, oracle):
    scene = synth.tiny_scene(0)
    cam, light = synth.camera_light_pair(1, 64, 64)
    g, fr = run_both(gs3, oracle, scene, cam, light)
    assert g["hdr"].light_ortho == 0.0 and fr["light_ortho"] == 0.0


def test_environment_render(gs3, oracle):
    import torch
    from paper_2410_11419_gb300 import render as R
    scene = synth.tiny_scene(0)
    cam, _ = synth.camera_light_pair(4, 96, 96)
    lights, w = synth.environment_lights(9, 4)
    ds = R.DeviceScene(scene)
    rd = R.Renderer(ds, 96, 96, 1 << 20)
    env = rd.render_environment(cam, lights, w).clone()
    torch.cuda.synchronize()
    rd.check()
    # the weighted sum of the single renders, accumulated in the same order
    acc = None
    for L, wl in zip(lights, w):
        img = rd.render(cam, L).clone().double()
        acc = float(wl) * img if acc is None else acc + float(wl) * img
    torch.cuda.synchronize()
    np.testing.assert_allclose(env.double().cpu().numpy(), acc.cpu().numpy(), rtol=1e-6, atol=1e-7)
    # against the oracle: sum of per-light tolerances
    want = np.zeros((96, 96, 3))
    tol = np.zeros((96, 96, 3))
    for L, wl in zip(lights, w):
        fr = oracle.render(scene, cam, L)
        want += float(wl) * fr["img"]
        tol += abs(float(wl)) * (1e-4 * np.abs(fr["img"]) + 1e-6 + fr["img_bound"])
    err = np.abs(env.double().cpu().numpy() - want)
    assert np.all(err <= tol + 1e-6), float((err - tol).max())
    ds.close()


def test_environment_rejects_bad_lights(gs3):
    import torch
    from paper_2410_11419_gb300 import _native as N, render as R
    scene = synth.tiny_scene(0)
    cam, _ = synth.camera_light_pair(4, 32, 32)
    ds = R.DeviceScene(scene)
    rd = R.Renderer(ds, 32, 32, 1 << 18)
    bad = synth.directional_light(1)
    bad.extent = 0.0
    with pytest.raises(N.GS3Error):
        rd.render(cam, bad)
    with pytest.raises(N.GS3Error):
        rd.render_environment(cam, [], [])
    ds.close()


def test_directional_backward_matches_gradient_oracle(gs3, oracle):
    from oracle import torch_ref as TR
    from tests.test_gpu_backward import _as_ref_layout, _compare, _gpu_grads
    scene = synth.make_scene(23, 500, 4, "ball")
    cam, _ = synth.camera_light_pair(23, 64, 64)
    light = synth.directional_light(23)
    target = oracle.render(synth.perturbed(scene, 24), cam, light)["img"]
    fr = oracle.render(scene, cam, light)
    dimg, _ = TR.image_grad_of_loss(fr["img"], target)
    ref, _ = TR.grads_given_image_grad(scene, cam, light, dimg)
    gpu = _gpu_grads(scene, cam, light, dimg)
    _compare(gpu, _as_ref_layout(scene, ref))
