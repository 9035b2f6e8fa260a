"""Shared angular-Gaussian basis (Sec. 4.1) on the GPU: frame parity against
the FP64 oracle (lists bit-exact, floats within 1e-4 + bounds) and the
backward, whose shared frame / deviation gradients are sums over every
Gaussian, against the FP64 gradient oracle."""
import pytest

from paper_2410_11419_gb300 import synth
from tests.test_gpu_parity import check_float_stages, check_integer_stages, run_both

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("make,seed,res", [
    (lambda: synth.with_shared_basis(synth.make_scene(14, 2000, 8, "ball"), 15), 14, 160),
    (lambda: synth.with_shared_basis(synth.object_scene(16, n=20000), 17), 16, 256),
], ids=["ball_2k_k8", "shell_20k_k8"])
def test_shared_basis_frame_parity(gs3, oracle, make, seed, res):
    scene = make()
    assert scene.lobe_shared
    cam, light = synth.camera_light_pair(seed, res, res)
    g, fr = run_both(gs3, oracle, scene, cam, light)
    check_integer_stages(g, fr)
    check_float_stages(g, fr)


def test_shared_basis_backward(gs3, oracle):
    from oracle import torch_ref as TR
    from tests.test_gpu_backward import _as_ref_layout, _compare, _gpu_grads
    scene = synth.with_shared_basis(synth.make_scene(25, 400, 3, "ball"), 26)
    cam, light = synth.camera_light_pair(25, 64, 64)
    target = oracle.render(synth.perturbed(scene, 27), cam, light)["img"]
    fr = oracle.render(scene, cam, light)
    dimg, _ = TR.image_grad_of_loss(fr["img"], target)
    ref, _ = TR.grads_given_image_grad(scene, cam, light, dimg)
    gpu = _gpu_grads(scene, cam, light, dimg)
    assert gpu["lobe_rot"].size == 4 * scene.k and gpu["lobe_sigma"].size == 4 * scene.k
    _compare(gpu, _as_ref_layout(scene, ref))
