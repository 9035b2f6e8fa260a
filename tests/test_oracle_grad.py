"""Pins of the gradient oracle (oracle/torch_ref.py, FP64 autograd) on CPU.

1. Its forward equals the C oracle's frame (same maths, independent code).
2. Its gradient of L = 0.8 L1 + 0.2 (1 - SSIM) (Sec. 4.4) equals central
   finite differences of the C oracle's loss, h = 1e-5, on coordinates whose
   +-h frames keep the same decision set (tile lists, ray stops, passing pair
   counts, biased occluder prefixes, and the sign of every pixel's L1 term,
   whose kink would break the difference quotient); coordinates whose
   decision set changes are counted and skipped.
"""
import numpy as np
import pytest
import torch

from paper_2410_11419_gb300 import synth

H_FD = 1e-5


@pytest.fixture(scope="module")
def fd_case(oracle):
    from oracle import torch_ref as TR
    scene = synth.make_scene(21, 500, 4, "ball")
    cam, light = synth.camera_light_pair(21, 64, 64)
    target = oracle.render(synth.perturbed(scene, 22), cam, light)["img"]
    L, img, grads, fr = TR.render_and_grad(scene, cam, light, target)
    return scene, cam, light, target, L, img, grads, fr


def test_forward_matches_c_oracle(fd_case):
    scene, cam, light, target, L, img, grads, fr = fd_case
    np.testing.assert_allclose(img, fr["img"], rtol=1e-12, atol=1e-13)


def test_ssim_identities():
    """SSIM(I, I) = 1 and the loss of an image against itself is 0; L1 part of
    two constant images is their difference."""
    from oracle import torch_ref as TR
    a = torch.rand((20, 24, 3), dtype=torch.float64, generator=torch.Generator().manual_seed(1))
    assert float(TR.ssim(a, a)) == pytest.approx(1.0, abs=1e-12)
    assert float(TR.loss(a, a)) == pytest.approx(0.0, abs=1e-12)
    c1 = torch.full((16, 16, 3), 0.3, dtype=torch.float64)
    c2 = torch.full((16, 16, 3), 0.5, dtype=torch.float64)
    l1 = float(TR.loss(c1, c2, lam=0.0))
    assert l1 == pytest.approx(0.2, abs=1e-12)


def _loss_of(oracle, scene, cam, light, target):
    from oracle import torch_ref as TR
    fr = oracle.render(scene, cam, light)
    L = float(TR.loss(torch.as_tensor(fr["img"]), torch.as_tensor(target)))
    return L, fr


def _occluder_bounds(fr):
    """K(j) of every light-list entry: end of its biased occluder prefix."""
    d = fr["light_key"].view(np.float32)
    ts, lst = fr["light_tile_start"], fr["light_list"]
    out = np.zeros(len(lst), dtype=np.int64)
    for t in range(fr["ntiles"]):
        dd = d[lst[ts[t]:ts[t + 1]]]
        out[ts[t]:ts[t + 1]] = np.searchsorted(dd, (dd - np.float32(0.015)).astype(np.float32), side="left")
    return out


def _same_decisions(a, b, target=None):
    if target is not None and not np.array_equal(np.sign(a["img"] - target), np.sign(b["img"] - target)):
        return False
    for k in ("cam_list", "light_list", "cam_tile_start", "light_tile_start", "n_contrib"):
        if not np.array_equal(a[k], b[k]):
            return False
    if not np.array_equal(_occluder_bounds(a), _occluder_bounds(b)):
        return False
    return (a["shadow_pass"] == b["shadow_pass"] and a["camera_evals"] == b["camera_evals"]
            and a["camera_pass"] == b["camera_pass"])


# (parameter group, scene attribute, index builder)
GROUPS = [
    ("mu", "mean_op", lambda g, c: (g, c)),
    ("logit", "mean_op", lambda g, c: (g, 3)),
    ("scale", "scale", lambda g, c: (g, c)),
    ("rot", "rot", lambda g, c: (g, c)),
    ("shade_rot", "shade_rot", lambda g, c: (g, c)),
    ("albedo_d", "albedo_d", lambda g, c: (g, c)),
    ("albedo_s", "albedo_s", lambda g, c: (g, c)),
    ("lobe_rot", "lobe_rot", lambda g, c: (1, g, c)),
    ("lobe_sigma", "lobe_sigma", lambda g, c: (2, g, c)),
    ("lobe_amp", "lobe_amp", lambda g, c: (0, g, c)),
]


def test_gradients_match_finite_differences(oracle, fd_case):
    scene, cam, light, target, L0, img, grads, fr0 = fd_case
    rng = np.random.default_rng(3)
    visible = np.nonzero(fr0["cam_rect"][:, 0] >= 0)[0]
    checked = skipped = 0
    worst = 0.0
    for name, attr, make_idx in GROUPS:
        ncomp = 4 if name in ("rot", "shade_rot", "lobe_rot") else 3
        for _ in range(4):
            g = int(rng.choice(visible))
            c = int(rng.integers(0, ncomp))
            idx = make_idx(g, c)
            if name == "logit":
                ad = grads["logit"][g]
            elif name.startswith("lobe_"):
                ad = grads[name][idx]
            else:
                ad = grads[name][g, c]
            vals = []
            frames = []
            for sgn in (1, -1):
                sc = scene.copy()
                arr = getattr(sc, attr)
                arr[idx] = np.float32(float(arr[idx]) + sgn * H_FD)
                L, fr = _loss_of(oracle, sc, cam, light, target)
                h_eff = float(np.float32(float(getattr(scene, attr)[idx]) + sgn * H_FD)) - float(getattr(scene, attr)[idx])
                vals.append((L, h_eff))
                frames.append(fr)
            if not (_same_decisions(frames[0], fr0, target) and _same_decisions(frames[1], fr0, target)):
                skipped += 1
                continue
            (Lp, hp), (Lm, hm) = vals
            fd = (Lp - Lm) / (hp - hm)
            err = abs(fd - ad)
            tol = 1e-4 * max(abs(ad), abs(fd)) + 5e-9
            worst = max(worst, err / max(abs(ad), 1e-12))
            assert err <= tol, f"{name}{idx}: FD {fd:.6e} AD {ad:.6e}"
            checked += 1
    assert checked >= 30, (checked, skipped)


def test_mlp_weight_gradients_match_finite_differences(oracle, fd_case):
    scene, cam, light, target, L0, img, grads, fr0 = fd_case
    rng = np.random.default_rng(4)
    checked = 0
    for nm in ("phi", "psi"):
        m = getattr(scene, nm)
        for layer in range(len(m.weights)):
            for _ in range(2):
                i = int(rng.integers(0, m.weights[layer].shape[0]))
                j = int(rng.integers(0, m.weights[layer].shape[1]))
                ad = grads[nm + "_w"][layer][i, j]
                vals = []
                for sgn in (1, -1):
                    sc = scene.copy()
                    w = getattr(sc, nm).weights[layer]
                    w0 = float(w[i, j])
                    w[i, j] = np.float32(w0 + sgn * H_FD)
                    h_eff = float(w[i, j]) - w0
                    L, fr = _loss_of(oracle, sc, cam, light, target)
                    assert _same_decisions(fr, fr0, target)
                    vals.append((L, h_eff))
                fd = (vals[0][0] - vals[1][0]) / (vals[0][1] - vals[1][1])
                assert abs(fd - ad) <= 1e-4 * max(abs(ad), abs(fd)) + 5e-9, (nm, layer, i, j, fd, ad)
                checked += 1
    assert checked == 2 * 2 * len(scene.phi.weights)


@pytest.fixture(scope="module")
def fd_case_directional(oracle):
    from oracle import torch_ref as TR
    scene = synth.make_scene(23, 500, 4, "ball")
    cam, _ = synth.camera_light_pair(23, 64, 64)
    light = synth.directional_light(23)
    target = oracle.render(synth.perturbed(scene, 24), cam, light)["img"]
    L, img, grads, fr = TR.render_and_grad(scene, cam, light, target)
    return scene, cam, light, target, L, img, grads, fr


def test_forward_matches_c_oracle_directional(fd_case_directional):
    """Sec. 4.5: the restatement's orthographic shadow splat and directional
    shading equal the C oracle's frame."""
    scene, cam, light, target, L, img, grads, fr = fd_case_directional
    np.testing.assert_allclose(img, fr["img"], rtol=1e-12, atol=1e-13)
    assert fr["light_ortho"] > 0 and fr["T"].min() < 0.9


def test_gradients_match_finite_differences_directional(oracle, fd_case_directional):
    """Central FD of the C oracle's loss under a directional light (same rules
    as the point-light check)."""
    scene, cam, light, target, L0, img, grads, fr0 = fd_case_directional
    rng = np.random.default_rng(7)
    visible = np.nonzero((fr0["cam_rect"][:, 0] >= 0) & (fr0["light_rect"][:, 0] >= 0))[0]
    checked = 0
    for name, attr, make_idx in GROUPS:
        ncomp = 4 if name in ("rot", "shade_rot", "lobe_rot") else 3
        for _ in range(2):
            g = int(rng.choice(visible))
            c = int(rng.integers(0, ncomp))
            idx = make_idx(g, c)
            if name == "logit":
                ad = grads["logit"][g]
            elif name.startswith("lobe_"):
                ad = grads[name][idx]
            else:
                ad = grads[name][g, c]
            vals, frames = [], []
            for sgn in (1, -1):
                sc = scene.copy()
                arr = getattr(sc, attr)
                arr[idx] = np.float32(float(arr[idx]) + sgn * H_FD)
                Lv, fr = _loss_of(oracle, sc, cam, light, target)
                h_eff = float(np.float32(float(getattr(scene, attr)[idx]) + sgn * H_FD)) - float(getattr(scene, attr)[idx])
                vals.append((Lv, h_eff))
                frames.append(fr)
            if not (_same_decisions(frames[0], fr0, target) and _same_decisions(frames[1], fr0, target)):
                continue
            (Lp, hp), (Lm, hm) = vals
            fd = (Lp - Lm) / (hp - hm)
            assert abs(fd - ad) <= 1e-4 * max(abs(ad), abs(fd)) + 5e-9, f"{name}{idx}: FD {fd:.6e} AD {ad:.6e}"
            checked += 1
    assert checked >= 12, checked


H_COARSE = 1e-3


def test_gradients_richardson_fd_coarse_step(oracle, fd_case):
    """Central differences at the step h = 1e-3 (with one Richardson step over
    h and h/2, truncation O(h^4)) on coordinates whose +-h and +-h/2 frames
    keep the decision set.  At this step most position and scale coordinates
    change their tile lists (skipped), and a few kept ones straddle a kink the
    decision set does not name (the alpha clamp at 0.99, the ELU of Eq. 3, a
    lobe at its pole): most agree to 1e-4, all to 5e-2; the tight pin is the
    h = 1e-5 test above.  A difference quotient cannot resolve a gradient
    below its round-off, about eps |L| / h per evaluation (the oracle's
    loss is summed by threads in an order that depends on the partition),
    so the relative error is taken against max(|ad|, |fd|, 1000 eps |L| / h)."""
    scene, cam, light, target, L0, img, grads, fr0 = fd_case
    floor = 1000.0 * np.finfo(np.float64).eps * abs(float(L0)) / H_COARSE
    rng = np.random.default_rng(3)
    visible = np.nonzero(fr0["cam_rect"][:, 0] >= 0)[0]

    def fd_at(attr, idx, h):
        vals, frames = [], []
        for sgn in (1, -1):
            sc = scene.copy()
            arr = getattr(sc, attr)
            arr[idx] = np.float32(float(arr[idx]) + sgn * h)
            L, fr = _loss_of(oracle, sc, cam, light, target)
            h_eff = float(np.float32(float(getattr(scene, attr)[idx]) + sgn * h)) - float(getattr(scene, attr)[idx])
            vals.append((L, h_eff))
            frames.append(fr)
        same = _same_decisions(frames[0], fr0, target) and _same_decisions(frames[1], fr0, target)
        (Lp, hp), (Lm, hm) = vals
        return same, (Lp - Lm) / (hp - hm)

    rel = []
    for name, attr, make_idx in GROUPS:
        ncomp = 4 if name in ("rot", "shade_rot", "lobe_rot") else 3
        for _ in range(4):
            g = int(rng.choice(visible))
            c = int(rng.integers(0, ncomp))
            idx = make_idx(g, c)
            ad = grads["logit"][g] if name == "logit" else (
                grads[name][idx] if name.startswith("lobe_") else grads[name][g, c])
            s1, f1 = fd_at(attr, idx, H_COARSE)
            s2, f2 = fd_at(attr, idx, H_COARSE / 2)
            if not (s1 and s2):
                continue
            fd = (4.0 * f2 - f1) / 3.0
            rel.append(abs(fd - ad) / max(abs(ad), abs(fd), floor))
    rel = np.array(rel)
    assert rel.size >= 20, rel.size
    assert np.mean(rel <= 1e-4) >= 0.75, np.sort(rel)
    assert rel.max() <= 5e-2, np.sort(rel)
