"""Deep shadow rays on the GPU, through the C ABI.

A stack of 32 nearly opaque layers lit along its axis: a quarter of the
shadow rays have exact occluder products below the smallest FP32 denormal.
The composite stops such a ray once its product is below 2^-40 and the
backward rebuilds every receiver's product from where the ray stopped.
Checked: the frame against the FP64 oracle (exact products, no stop) within
the parity tolerance, the stop records, and the gradients of every
parameter against the FP64 gradient oracle.
"""
import numpy as np
import pytest

from paper_2410_11419_gb300 import synth
from tests.test_gpu_parity import check_float_stages, check_integer_stages, run_both
from tests.test_oracle_deep_shadow import STOP, deep_stack

pytestmark = pytest.mark.gpu


def test_deep_stack_frame_parity(gs3, oracle):
    scene, cam, light = deep_stack(res=64)
    g, fr = run_both(gs3, oracle, scene, cam, light)
    check_integer_stages(g, fr)
    check_float_stages(g, fr)
    A, lim = g["light_final"], g["light_stop"]
    stopped = lim != 0xFFFFFFFF
    assert stopped.mean() > 0.1, stopped.mean()
    # a stopped ray's product froze in [stop (1 - alpha_max), stop); the others stayed >= stop
    assert np.all(A[stopped] < STOP) and np.all(A[stopped] >= STOP * (1 - 0.99) * 0.999)
    assert np.all(A[~stopped] >= STOP)
    # the stopping occluder lies in the ray's tile segment of the light list
    ts = g["ltile_start"].view(np.uint32)
    gx = (cam.width + 15) // 16
    ys, xs = np.nonzero(stopped)
    tiles = (ys // 16) * gx + xs // 16
    assert np.all(lim[stopped] > ts[tiles]) and np.all(lim[stopped] <= ts[tiles + 1])


def test_deep_stack_backward_matches_gradient_oracle(gs3, oracle):
    from oracle import torch_ref as TR
    from tests.test_gpu_backward import _as_ref_layout, _compare, _gpu_grads
    scene, cam, light = deep_stack(res=64)
    target = oracle.render(synth.perturbed(scene, 4), cam, light)["img"]
    fr = oracle.render(scene, cam, light)
    dimg, _ = TR.image_grad_of_loss(fr["img"], target)
    ref, _ = TR.grads_given_image_grad(scene, cam, light, dimg)
    gpu = _gpu_grads(scene, cam, light, dimg)
    rep = _compare(gpu, _as_ref_layout(scene, ref))
    assert len(rep) == 14
