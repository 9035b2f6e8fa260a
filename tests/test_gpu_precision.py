"""Tensor-core MLPs in BF16 and FP8 E4M3 (precision form).

1. The tcgen05 kernels against a plain PyTorch reference of the same
   operation: inputs and hidden weights rounded to BF16 (or scaled and
   rounded to E4M3 with the per-tensor scales), products accumulated in FP32,
   hidden activations rounded between layers, the output layer in FP32.
2. The FP8 scales against their definition recomputed in PyTorch: sw = max|W|/448,
   sx = 2 max|x|/448 over the calibration sample (strided Gaussians x eight
   Fibonacci-sphere directions, T alternating 0 and 1).
3. The whole frame against the FP64 oracle per dtype: integer stages stay
   bit-exact and FP32 stages keep the 1e-4 bound; the MLP outputs and the
   image carry the reduced-precision error, recorded per output (max and
   mean) in $GS3_PARITY_STATS.
"""
import json
import os

import numpy as np
import pytest

from paper_2410_11419_gb300 import synth
from tests.test_gpu_parity import check_float_stages, check_integer_stages

pytestmark = pytest.mark.gpu


def _pe(v):
    import torch
    out = [v]
    for k in range(4):
        out += [torch.sin((2 ** k) * np.pi * v), torch.cos((2 ** k) * np.pi * v)]
    return torch.cat(out, dim=1)


def _act(mlp, h):
    import torch
    return torch.relu(h) if mlp.act == synth.RELU else torch.where(h > 0, h, 0.01 * h)


def torch_reference(scene, mlp, X):
    """Same operation as the BF16 kernel, in plain PyTorch."""
    import torch
    bf = lambda t: t.to(torch.bfloat16).to(torch.float32)
    h = bf(X)
    for li, (w, b) in enumerate(zip(mlp.weights, mlp.biases)):
        w = torch.from_numpy(w).cuda()
        b = torch.from_numpy(b).cuda()
        if li < mlp.n_hidden:
            h = _act(mlp, h @ bf(w).T + b)
            if li + 1 < mlp.n_hidden:
                h = bf(h)
        else:
            h = torch.sigmoid(h @ w.T + b)
    return h


def q8(t, s):
    """Scale by 1/s, saturate to +-448 and round to E4M3; returned in the scaled units."""
    import torch
    return (t * (1.0 / s)).clamp(-448.0, 448.0).to(torch.float8_e4m3fn).to(torch.float32)


def torch_reference_fp8(mlp, X, scales):
    """Same operation as the FP8 kernel, in plain PyTorch, given the scales."""
    import torch
    h = X
    for li, (w, b) in enumerate(zip(mlp.weights, mlp.biases)):
        w = torch.from_numpy(w).cuda()
        b = torch.from_numpy(b).cuda()
        if li < mlp.n_hidden:
            sx, sw = scales[li]
            h = _act(mlp, (q8(h, sx) @ q8(w, sw).T) * np.float32(sx * sw) + b)
        else:
            h = torch.sigmoid(h @ w.T + b)
    return h


def fib_dirs():
    d = np.arange(8, dtype=np.float32)
    z = 1.0 - (2.0 * d + 1.0) / 8.0
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    ph = np.float32(2.39996323) * d
    return np.stack([r * np.cos(ph), r * np.sin(ph), z], 1).astype(np.float32)


def calibration_scales(scene, mlp, which):
    """The FP8 scales by their definition (FP32, PyTorch)."""
    import torch
    n = scene.n
    S = min(n, 16384)
    g = (np.arange(S, dtype=np.int64) * n) // S
    mu = torch.from_numpy(scene.mean_op[g, :3]).cuda()
    lat = torch.cat([torch.from_numpy(scene.latent[0][g]), torch.from_numpy(scene.latent[1][g, :2])], 1).cuda()
    dirs = torch.from_numpy(fib_dirs()).cuda()
    rows = []
    for d in range(8):
        w = dirs[d][None].expand(S, 3)
        parts = [_pe(w), _pe(mu), lat]
        if which == 0:
            parts.insert(0, torch.full((S, 1), float(d & 1), device="cuda"))
        rows.append(torch.cat(parts, 1))
    h = torch.cat(rows, 0)
    out = []
    for li in range(mlp.n_hidden):
        amax = float(h.abs().max())
        w = torch.from_numpy(mlp.weights[li]).cuda()
        out.append((2.0 * amax / 448.0, float(w.abs().max()) / 448.0))
        h = _act(mlp, h @ w.T + torch.from_numpy(mlp.biases[li]).cuda())
    return out


def inputs(scene, cam, light, T):
    import torch
    mu = torch.from_numpy(scene.mean_op[:, :3]).cuda()
    lat = torch.cat([torch.from_numpy(scene.latent[0]), torch.from_numpy(scene.latent[1][:, :2])], 1).cuda()
    wi = torch.from_numpy(light.pos).cuda()[None] - mu
    wi = wi / wi.norm(dim=1, keepdim=True)
    wo = torch.from_numpy(cam.pos).cuda()[None] - mu
    wo = wo / wo.norm(dim=1, keepdim=True)
    xphi = torch.cat([T[:, None], _pe(wi), _pe(mu), lat], 1)
    xpsi = torch.cat([_pe(wo), _pe(mu), lat], 1)
    return xphi, xpsi


@pytest.mark.parametrize("make,res", [
    (lambda: synth.tiny_scene(0), 128),                      # 2x64 ReLU
    (lambda: synth.object_scene(5, n=20_000), 256),          # 3x128 ReLU
    (lambda: synth.paper_mlp_scene(2, n=3000), 160),         # Phi 3x32, Psi 3x128, leaky ReLU
], ids=["tiny_2x64", "shell_3x128", "paper_mlp"])
def test_tc_mlp_matches_torch(gs3, make, res):
    import torch
    from paper_2410_11419_gb300 import _native as N, render as R
    scene = make()
    cam, light = synth.camera_light_pair(4, res, res)
    ds = R.DeviceScene(scene, mlp_dtype=N.GS3_MLP_BF16)
    rd = R.Renderer(ds, res, res, 1 << 22)
    rd.render(cam, light)
    torch.cuda.synchronize()
    rd.check()
    T = rd.stage("T").clone()
    xphi, xpsi = inputs(scene, cam, light, T)
    want_tp = torch_reference(scene, scene.phi, xphi)[:, 0]
    want_res = torch_reference(scene, scene.psi, xpsi)
    got_tp = rd.stage("Tp")
    got_res = rd.stage("res")[:, :3]
    assert torch.isfinite(got_tp).all() and torch.isfinite(got_res).all()
    # accumulation order and BF16 rounding of near-tie hidden values: 2e-3 absolute
    assert (got_tp - want_tp).abs().max().item() < 2e-3
    assert (got_res - want_res).abs().max().item() < 2e-3
    assert (got_tp - want_tp).abs().mean().item() < 2e-4
    ds.close()


FP8_CASES = [
    (lambda: synth.tiny_scene(0), 128),                      # 2x64 ReLU
    (lambda: synth.object_scene(5, n=20_000), 256),          # 3x128 ReLU
    (lambda: synth.paper_mlp_scene(2, n=3000), 160),         # Phi 3x32, Psi 3x128, leaky ReLU
]


@pytest.mark.parametrize("make,res", FP8_CASES, ids=["tiny_2x64", "shell_3x128", "paper_mlp"])
def test_fp8_scales_match_definition(gs3, make, res):
    from paper_2410_11419_gb300 import _native as N, render as R
    scene = make()
    ds = R.DeviceScene(scene, mlp_dtype=N.GS3_MLP_FP8_E4M3)
    for which, mlp in ((0, scene.phi), (1, scene.psi)):
        got = N.gs3_scene_mlp_scales(ds.handle, which, mlp.n_hidden)
        want = calibration_scales(scene, mlp, which)
        for (gx, gw), (wx, ww) in zip(got, want):
            assert gw == pytest.approx(ww, rel=1e-6)     # a max of exact values
            assert gx == pytest.approx(wx, rel=1e-5)     # FP32 forward, summation order
    ds.close()


@pytest.mark.parametrize("make,res", FP8_CASES, ids=["tiny_2x64", "shell_3x128", "paper_mlp"])
def test_fp8_mlp_matches_torch(gs3, make, res):
    import torch
    from paper_2410_11419_gb300 import _native as N, render as R
    scene = make()
    cam, light = synth.camera_light_pair(4, res, res)
    ds = R.DeviceScene(scene, mlp_dtype=N.GS3_MLP_FP8_E4M3)
    rd = R.Renderer(ds, res, res, 1 << 22)
    rd.render(cam, light)
    torch.cuda.synchronize()
    rd.check()
    T = rd.stage("T").clone()
    xphi, xpsi = inputs(scene, cam, light, T)
    want_tp = torch_reference_fp8(scene.phi, xphi, N.gs3_scene_mlp_scales(ds.handle, 0, scene.phi.n_hidden))[:, 0]
    want_res = torch_reference_fp8(scene.psi, xpsi, N.gs3_scene_mlp_scales(ds.handle, 1, scene.psi.n_hidden))
    got_tp = rd.stage("Tp")
    got_res = rd.stage("res")[:, :3]
    assert torch.isfinite(got_tp).all() and torch.isfinite(got_res).all()
    # Same quantised operands; only FP32 accumulation order and E4M3 rounding
    # of hidden values that land within rounding distance of a midpoint differ
    # (one E4M3 step, 1/8 relative, of a single activation each time).
    d_tp, d_res = (got_tp - want_tp).abs(), (got_res - want_res).abs()
    _record(f"fp8_vs_torch[{res}]", {"T'": (float(d_tp.max()), float(d_tp.mean())),
                                     "residual": (float(d_res.max()), float(d_res.mean()))})
    assert d_tp.max().item() < 2e-2 and d_res.max().item() < 2e-2
    assert d_tp.mean().item() < 1e-4 and d_res.mean().item() < 1e-4
    ds.close()


def _record(name, stats):
    path = os.environ.get("GS3_PARITY_STATS")
    if path:
        with open(path, "a") as fh:
            for k, (mx, mn) in stats.items():
                fh.write(json.dumps({"test": name, "output": k, "max_abs": float(mx), "mean_abs": float(mn)}) + "\n")


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_reduced_precision_frame_against_oracle(gs3, oracle, dtype):
    import torch
    from paper_2410_11419_gb300 import _native as N, render as R
    scene = synth.tiny_scene(0)
    cam, light = synth.camera_light_pair(0, 128, 128)
    ds = R.DeviceScene(scene, mlp_dtype=N.GS3_MLP_BF16 if dtype == "bf16" else N.GS3_MLP_FP8_E4M3)
    rd = R.Renderer(ds, 128, 128, 1 << 20)
    img = rd.render(cam, light)
    torch.cuda.synchronize()
    hdr = rd.check()
    fr = oracle.render(scene, cam, light)
    g = {k: rd.stage(k, s).cpu().numpy() for k, s in
         (("key", 0), ("order", 0), ("tile_start", 0), ("rect", 0), ("shade", 0), ("T", 0))}
    for nm, s in (("lkey", 1), ("lorder", 1), ("ltile_start", 1), ("lrect", 1)):
        g[nm] = rd.stage(nm[1:], s).cpu().numpy()
    g["list"] = rd.stage("list", 0)[:hdr.pairs_cam].cpu().numpy()
    g["llist"] = rd.stage("list", 1)[:hdr.pairs_light].cpu().numpy()
    check_integer_stages(g, fr)
    from tests.test_gpu_parity import assert_close
    assert_close("shade", g["shade"][:, :3].astype(np.float64), fr["shade"])
    assert_close("shadow T", g["T"].astype(np.float64), fr["T"], fr["T_bound"])
    tp = rd.stage("Tp").cpu().numpy().astype(np.float64)
    res = rd.stage("res").cpu().numpy()[:, :3].astype(np.float64)
    im = img.cpu().numpy().astype(np.float64)
    stats = {
        "T'": (np.abs(tp - fr["Tp"]).max(), np.abs(tp - fr["Tp"]).mean()),
        "residual": (np.abs(res - fr["res"]).max(), np.abs(res - fr["res"]).mean()),
        "image": (np.abs(im - fr["img"]).max(), np.abs(im - fr["img"]).mean()),
    }
    _record(f"{dtype}_frame", stats)
    if dtype == "bf16":
        # BF16 operands: a few 1e-3 on sigmoid outputs, well under 1e-2
        assert stats["T'"][0] < 1e-2 and stats["residual"][0] < 1e-2
        assert stats["image"][1] < 2e-3 * max(1.0, float(np.abs(fr["img"]).mean()))
    else:
        # E4M3 keeps 3 mantissa bits (relative step 1/8): errors of a few 1e-2
        # on sigmoid outputs are expected; the bound catches a wrong scale or
        # layout, which moves outputs by O(0.1-1)
        assert stats["T'"][0] < 0.1 and stats["residual"][0] < 0.1
        assert stats["T'"][1] < 2e-2 and stats["residual"][1] < 2e-2
        assert stats["image"][1] < 2e-2 * max(1.0, float(np.abs(fr["img"]).mean()))
    ds.close()
