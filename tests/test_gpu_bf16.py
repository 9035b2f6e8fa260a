"""BF16 tensor-core MLPs (precision form).

1. The tcgen05 kernel against a plain PyTorch reference of the same
   operation: inputs and hidden weights rounded to BF16, products accumulated
   in FP32, hidden activations rounded to BF16 between layers, the output
   layer in FP32.
2. The whole BF16 frame against the FP64 oracle: integer stages stay
   bit-exact and FP32 stages keep the 1e-4 bound; the MLP outputs and the
   image carry the BF16 error, recorded per output in $GS3_PARITY_STATS.
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


def torch_reference(scene, mlp, X):
    """Same operation as the kernel, in plain PyTorch."""
    import torch
    bf = lambda t: t.to(torch.bfloat16).to(torch.float32)
    h = bf(X)
    for li, (w, b) in enumerate(zip(mlp.weights, mlp.biases)):
        w = torch.from_numpy(w).cuda()
        b = torch.from_numpy(b).cuda()
        if li < mlp.n_hidden:
            h = h @ bf(w).T + b
            h = torch.relu(h) if mlp.act == synth.RELU else torch.where(h > 0, h, 0.01 * h)
            if li + 1 < mlp.n_hidden:
                h = bf(h)
        else:
            h = torch.sigmoid(h @ w.T + b)
    return h


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


def test_bf16_frame_against_oracle(gs3, oracle):
    import torch
    from paper_2410_11419_gb300 import _native as N, render as R
    scene = synth.tiny_scene(0)
    cam, light = synth.camera_light_pair(0, 128, 128)
    ds = R.DeviceScene(scene, mlp_dtype=N.GS3_MLP_BF16)
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
    path = os.environ.get("GS3_PARITY_STATS")
    if path:
        with open(path, "a") as fh:
            for k, (mx, mn) in stats.items():
                fh.write(json.dumps({"test": "bf16_frame", "output": k, "max_abs": float(mx),
                                     "mean_abs": float(mn)}) + "\n")
    # BF16 operands: a few 1e-3 on sigmoid outputs, well under 1e-2
    assert stats["T'"][0] < 1e-2 and stats["residual"][0] < 1e-2
    assert stats["image"][1] < 2e-3 * max(1.0, float(np.abs(fr["img"]).mean()))
    ds.close()
