"""Pins of the shared angular-Gaussian basis (Sec. 4.1), CPU.

With a shared basis every spatial Gaussian evaluates the same K lobes
(frames and deviations) with its own weights.  That is exactly the
per-Gaussian form with the basis replicated into every Gaussian, so the two
shadings must agree bit for bit (and the frames to FP64 rounding); and the gradient of a shared parameter is the
sum over the Gaussians, which central finite differences of the C oracle's
loss check.
"""
import numpy as np
import pytest

from paper_2410_11419_gb300 import synth
from tests.test_oracle_grad import H_FD, _loss_of, _same_decisions


def replicated(shared: synth.Scene) -> synth.Scene:
    s = shared.copy()
    s.lobe_rot = np.ascontiguousarray(np.repeat(shared.lobe_rot, shared.n, axis=1))
    s.lobe_sigma = np.ascontiguousarray(np.repeat(shared.lobe_sigma, shared.n, axis=1))
    s.lobe_shared = False
    return s


def test_shared_basis_equals_replicated_lobes(oracle):
    base = synth.make_scene(12, 400, 6, "ball")
    shared = synth.with_shared_basis(base, 13)
    assert shared.lobe_rot.shape == (6, 1, 4) and shared.lobe_amp.shape == (6, 400, 4)
    cam, light = synth.camera_light_pair(12, 64, 64)
    a = oracle.render(shared, cam, light)
    b = oracle.render(replicated(shared), cam, light)
    np.testing.assert_array_equal(a["shade"], b["shade"])  # the shading is where the basis enters
    for k in ("T", "Tp", "res", "img"):  # FP64 sums whose threaded order varies in the last ulp
        np.testing.assert_allclose(a[k], b[k], rtol=1e-13, atol=1e-15, err_msg=k)
    # and it is not the per-Gaussian scene it came from
    c = oracle.render(base, cam, light)
    assert np.abs(a["shade"] - c["shade"]).max() > 1e-3


@pytest.fixture(scope="module")
def shared_case(oracle):
    from oracle import torch_ref as TR
    scene = synth.with_shared_basis(synth.make_scene(25, 400, 3, "ball"), 26)
    cam, light = synth.camera_light_pair(25, 64, 64)
    target = oracle.render(synth.perturbed(scene, 27), cam, light)["img"]
    L, img, grads, fr = TR.render_and_grad(scene, cam, light, target)
    return scene, cam, light, target, L, img, grads, fr


def test_torch_restatement_forward_shared(shared_case):
    scene, cam, light, target, L, img, grads, fr = shared_case
    np.testing.assert_allclose(img, fr["img"], rtol=1e-12, atol=1e-13)
    assert grads["lobe_rot"].shape[1] == 1 and grads["lobe_sigma"].shape[1] == 1


def test_shared_basis_gradients_match_finite_differences(oracle, shared_case):
    scene, cam, light, target, L0, img, grads, fr0 = shared_case
    checked = 0
    for name, comps in (("lobe_rot", range(4)), ("lobe_sigma", range(3))):
        for j in range(scene.k):
            for c in comps:
                idx = (j, 0, c)
                ad = grads[name][idx]
                vals, frames = [], []
                for sgn in (1, -1):
                    sc = scene.copy()
                    arr = getattr(sc, name)
                    arr[idx] = np.float32(float(arr[idx]) + sgn * H_FD)
                    Lv, fr = _loss_of(oracle, sc, cam, light, target)
                    h_eff = float(np.float32(float(getattr(scene, name)[idx]) + sgn * H_FD)) - float(getattr(scene, name)[idx])
                    vals.append((Lv, h_eff))
                    frames.append(fr)
                if not (_same_decisions(frames[0], fr0, target) and _same_decisions(frames[1], fr0, target)):
                    continue
                (Lp, hp), (Lm, hm) = vals
                fd = (Lp - Lm) / (hp - hm)
                assert abs(fd - ad) <= 1e-4 * max(abs(ad), abs(fd)) + 5e-9, (name, idx, fd, ad)
                checked += 1
    assert checked >= 12, checked
