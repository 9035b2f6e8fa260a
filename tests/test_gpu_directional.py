"""Directional and environment lighting (Sec. 4.5) on the GPU, through the C ABI.

* A directional light's frame against the FP64 oracle: the orthographic light
  view (rotation, translation, pixel scale) equal bit for bit, keys, lists and
  ranges of both splats bit-exact, and the floating-point stages within
  1e-4 relative + 1e-6 + the oracle's decision bounds.
* gs3_render_environment (one batched frame) equals the weighted sum of
  single renders, and the oracle's environment image within the summed
  tolerances: 9 lights (a group of 8 and one more), FP32 and BF16 MLPs, the
  ablations; its header reports the camera's and the largest light pair
  counts.
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
    eh = rd.env_header()
    assert eh.status == 0
    # the weighted sum of the single renders, accumulated in the same order
    acc = None
    light_pairs = []
    for L, wl in zip(lights, w):
        img = rd.render(cam, L).clone().double()
        h = rd.check()
        light_pairs.append(h.pairs_light)
        acc = float(wl) * img if acc is None else acc + float(wl) * img
    torch.cuda.synchronize()
    np.testing.assert_allclose(env.double().cpu().numpy(), acc.cpu().numpy(), rtol=1e-6, atol=1e-7)
    assert eh.pairs_cam == h.pairs_cam and eh.pairs_light == max(light_pairs)
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


ENV_VARIANTS = [
    ("bf16_3", "bf16", 3, 0),
    ("fp8_8", "fp8", 8, 0),
    ("fp32_no_shadow_splat", "fp32", 5, "shadow"),
    ("bf16_identity_phi_psi", "bf16", 4, "mlps"),
    ("fp32_17", "fp32", 17, 0),
]


@pytest.mark.parametrize("name,dtype,count,ablate", ENV_VARIANTS, ids=[v[0] for v in ENV_VARIANTS])
def test_environment_equals_single_frames(gs3, name, dtype, count, ablate):
    """The batched environment frame against the weighted sum of the same
    lights' single frames, for the tensor-core MLPs, the ablations and more
    than two groups of lights; each light's shadow values T and refined T'
    (batched Phi over the group's lights) equal its single frame's bit for bit."""
    import torch
    from paper_2410_11419_gb300 import _native as N, render as R
    scene = synth.make_scene(3, 3000, 4, "ball")
    cam, _ = synth.camera_light_pair(6, 120, 104)
    lights, w = synth.environment_lights(11, count)
    mlp = {"fp32": N.GS3_MLP_FP32, "bf16": N.GS3_MLP_BF16, "fp8": N.GS3_MLP_FP8_E4M3}[dtype]
    ds = R.DeviceScene(scene, mlp_dtype=mlp)
    rd = R.Renderer(ds, 120, 104, 1 << 20)
    opts = R.opts_struct()
    if ablate == "shadow":
        opts.ablate = N.GS3_ABLATE_SHADOW_SPLAT
    elif ablate == "mlps":
        opts.ablate = N.GS3_ABLATE_PHI | N.GS3_ABLATE_PSI
    env = rd.render_environment(cam, lights, w, opts=opts).clone()
    torch.cuda.synchronize()
    assert rd.env_header().status == 0
    # the last group's lights keep their shadow values in the workspace's
    # per-light frames (8 lights per group), 256-byte aligned frame sizes apart
    n = scene.n
    stride = (N.gs3_workspace_size(n, 120, 104, rd.cap) + 255) // 256 * 256
    g0 = 8 * ((count - 1) // 8)
    kept = {}
    for li in range(g0, count):
        base = (li - g0) * stride
        kept[li] = {nm: rd.env_ws[base + off:base + off + 4 * n].view(torch.float32).clone()
                    for nm, off in (("T", rd.layout.shadow), ("Tp", rd.layout.shadow_refined))}
    acc = None
    for li, (L, wl) in enumerate(zip(lights, w)):
        img = rd.render(cam, L, opts=opts).clone().double()
        rd.check()
        if li in kept:
            for nm in ("T", "Tp"):
                assert torch.equal(kept[li][nm], rd.stage(nm)), (li, nm)
        acc = float(wl) * img if acc is None else acc + float(wl) * img
    torch.cuda.synchronize()
    np.testing.assert_allclose(env.double().cpu().numpy(), acc.cpu().numpy(), rtol=2e-6, atol=1e-7)
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
