"""Differentiable FP64 restatement of the GS^3 frame in plain PyTorch CPU ops.

TEST INFRASTRUCTURE ONLY (gradient oracle): imported by the tests, never by
the library.  It recomputes, in float64 and with autograd, the same frame as
gs3_oracle.c:
  Eq. 1 covariance, Sec. 3 EWA projection, Eq. 2-5 shading, Sec. 4.2 shadow
  splatting with the 0.015 bias and the beta-weighted average, the Phi/Psi
  MLPs with 4-band positional encoding, the camera composite (Eq. 2) and the
  per-pixel combination shading * shadow + residual (Sec. 4), and the loss
  (1 - lambda) L1 + lambda (1 - SSIM), lambda = 0.2 (Sec. 4.4).
The discrete structure -- tile lists and their order, the FP32 light
distances that decide the shadow bias, which (pixel, Gaussian) pairs pass
alpha >= 1/255 and where a camera ray stops -- is taken from the C oracle's
frame (its own integer and decision outputs) and held fixed, so the result
is the gradient of the piecewise-smooth frame on the current decision set.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import oracle as O

DT = torch.float64


def quat_mat(q):
    """(N, 4) -> (N, 3, 3) rotation of the normalised quaternion (w, x, y, z)."""
    q = q / q.norm(dim=1, keepdim=True)
    w, x, y, z = q.unbind(1)
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], 1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], 1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], 1)], 1)


def pos_enc(v):
    out = [v]
    for k in range(4):
        out += [torch.sin((2.0 ** k) * math.pi * v), torch.cos((2.0 ** k) * math.pi * v)]
    return torch.cat(out, 1)


def mlp(params, act, x):
    ws, bs = params
    h = x
    for i, (w, b) in enumerate(zip(ws, bs)):
        h = h @ w.T + b
        if i < len(ws) - 1:
            h = torch.relu(h) if act == 0 else torch.where(h > 0, h, 0.01 * h)
        else:
            h = torch.sigmoid(h)
    return h


def project(mu, scale, rot, R, t, fx, fy, cx, cy, lowpass=0.3, ortho=0.0):
    """Screen position (N, 2) and conic (N, 3) = (A, B, C) of every Gaussian;
    perspective, or orthographic with `ortho` pixels per unit (Sec. 4.5)."""
    p = mu @ R.T + t
    tx, ty, tz = p.unbind(1)
    if ortho > 0:
        u = ortho * tx + cx
        v = ortho * ty + cy
    else:
        u = fx * tx / tz + cx
        v = fy * ty / tz + cy
    Rq = quat_mat(rot)
    M = Rq * scale[:, None, :]
    Sig = M @ M.transpose(1, 2)
    zero = torch.zeros_like(tz)
    if ortho > 0:
        s_ = torch.full_like(tz, ortho)
        J = torch.stack([torch.stack([s_, zero, zero], 1), torch.stack([zero, s_, zero], 1)], 1)
    else:
        J = torch.stack([torch.stack([fx / tz, zero, -fx * tx / (tz * tz)], 1),
                         torch.stack([zero, fy / tz, -fy * ty / (tz * tz)], 1)], 1)
    T = J @ R
    S2 = T @ Sig @ T.transpose(1, 2)
    a = S2[:, 0, 0] + lowpass
    b = S2[:, 0, 1]
    c = S2[:, 1, 1] + lowpass
    det = a * c - b * b
    return torch.stack([u, v], 1), torch.stack([c / det, -b / det, a / det], 1)


def shade(P, cam_pos, light_pos, intensity, falloff=True, light_dir=None, specular=True):
    """Colour (Eq. 2-5), omega_i and omega_o.  A directional light (Sec. 4.5)
    gives omega_i = light_dir for every Gaussian and no fall-off."""
    mu = P["mu"]
    if light_dir is not None:
        tol = light_dir[None].expand_as(mu)
        falloff = False
    else:
        tol = light_pos[None] - mu
    d2 = (tol * tol).sum(1)
    wi = tol / d2.sqrt()[:, None]
    vo = cam_pos[None] - mu
    wo = vo / vo.norm(dim=1, keepdim=True)
    Rs = quat_mat(P["shade_rot"])
    wil = (Rs @ wi[:, :, None])[:, :, 0]
    wol = (Rs @ wo[:, :, None])[:, :, 0]
    x = wil[:, 2]
    off = 0.01 * (1 - math.exp(-1))
    elu = torch.where(x > 0, x, 0.01 * (torch.exp(torch.clamp(x, max=0.0)) - 1))
    fd = (elu + off) / ((1 + off) * math.pi)
    hs = wil + wol
    h = hs / hs.norm(dim=1, keepdim=True)
    fs = torch.zeros_like(mu)
    K = P["lobe_rot"].shape[0] if specular else 0
    for j in range(K):
        Rl = quat_mat(P["lobe_rot"][j])
        hl = (Rl.transpose(1, 2) @ h[:, :, None])[:, :, 0]
        sxy = torch.sqrt(hl[:, 0] ** 2 + hl[:, 1] ** 2)
        theta = torch.atan2(sxy, hl[:, 2])
        sig = P["lobe_sigma"][j]
        sx, sy = hl[:, 0] / sxy, hl[:, 1] / sxy
        q2 = (sx / sig[:, 0]) ** 2 + (sy / sig[:, 1]) ** 2
        e2 = theta * theta * q2 / (sig[:, 2] ** 2)
        G = torch.exp(-0.5 * e2) / sig[:, 2]
        fs = fs + P["lobe_amp"][j] * G[:, None]
    E = intensity / d2 if falloff else intensity * torch.ones_like(d2)
    return E[:, None] * (P["albedo_d"] * fd[:, None] + P["albedo_s"] * fs), wi, wo


def _tile_pixels(tx, ty, W, H, ts):
    xs = torch.arange(tx * ts, min(W, tx * ts + ts), dtype=DT) + 0.5
    ys = torch.arange(ty * ts, min(H, ty * ts + ts), dtype=DT) + 0.5
    yy, xx = torch.meshgrid(ys, xs, indexing="ij")
    return xx.reshape(-1), yy.reshape(-1)


def _power(uv, conic, lst, px, py):
    dx = px[:, None] - uv[lst, 0][None]
    dy = py[:, None] - uv[lst, 1][None]
    A, B, C = conic[lst, 0][None], conic[lst, 1][None], conic[lst, 2][None]
    return -0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy


def frame(P, fr, cam, light, opts, mlps):
    """Image (H, W, 3) of the parameter dict P (tensors, float64) on the
    decision structure of the C-oracle frame fr."""
    n = P["mu"].shape[0]
    W, H, ts = cam.width, cam.height, opts.tile
    # the thresholds are FP32 option values, as in the C oracle
    amin, amax = float(np.float32(opts.alpha_min)), float(np.float32(opts.alpha_max))
    tstop = float(np.float32(opts.t_stop))
    gx = fr["gx"]
    gamma = torch.sigmoid(P["logit"])
    Rc, tc = torch.tensor(cam.R, dtype=DT).reshape(3, 3), torch.tensor(cam.t, dtype=DT)
    Rl, tl = torch.tensor(fr["light_R"], dtype=DT), torch.tensor(fr["light_t"], dtype=DT)
    f = [float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)]
    lp = float(np.float32(opts.lowpass))
    uv_c, con_c = project(P["mu"], P["scale"], P["rot"], Rc, tc, *f, lowpass=lp)
    uv_l, con_l = project(P["mu"], P["scale"], P["rot"], Rl, tl, *f, lowpass=lp,
                          ortho=float(fr.get("light_ortho", 0.0)))
    cam_pos = torch.tensor(cam.pos, dtype=DT)
    light_pos = torch.tensor(light.pos, dtype=DT)
    ldir = None
    if getattr(light, "type", 0) == 1:
        ldir = torch.tensor(np.asarray(light.dir, dtype=np.float32), dtype=DT)
        ldir = ldir / ldir.norm()
    col, wi, wo = shade(P, cam_pos, light_pos, float(light.intensity), bool(opts.falloff), light_dir=ldir,
                        specular=not (opts.ablate & 8))

    # ---- shadow splatting (Sec. 4.2) ----
    num = torch.zeros(n, dtype=DT)
    den = torch.zeros(n, dtype=DT)
    d32 = fr["light_key"].view(np.float32)
    bias = np.float32(opts.shadow_bias)
    ts_l, lst_l = fr["light_tile_start"], fr["light_list"]
    for t in range(fr["ntiles"]):
        b, e = int(ts_l[t]), int(ts_l[t + 1])
        if b == e:
            continue
        lst = torch.from_numpy(lst_l[b:e].astype(np.int64))
        px, py = _tile_pixels(t % gx, t // gx, W, H, ts)
        pw = _power(uv_l, con_l, lst, px, py)
        beta = torch.exp(pw)
        alpha = torch.clamp(gamma[lst][None] * beta, max=amax)
        passing = (alpha >= amin).detach()
        l1a = torch.where(passing, torch.log1p(-alpha), torch.zeros_like(alpha))
        cs = torch.cat([torch.zeros((px.shape[0], 1), dtype=DT), torch.cumsum(l1a, 1)], 1)
        dd = d32[lst_l[b:e]]
        Kj = np.searchsorted(dd, (dd - bias).astype(np.float32), side="left")  # occluder prefix ends
        Tm = torch.exp(cs[:, torch.from_numpy(Kj.astype(np.int64))])
        contrib = torch.where(passing, beta * Tm, torch.zeros_like(beta)).sum(0)
        dsum = torch.where(passing, beta, torch.zeros_like(beta)).sum(0)
        num = num.index_add(0, lst, contrib)
        den = den.index_add(0, lst, dsum)
    if opts.ablate & 1:
        T = torch.ones(n, dtype=DT)
    else:
        T = torch.where(den > 0, num / torch.where(den > 0, den, torch.ones_like(den)), torch.ones_like(den))

    # ---- Phi, Psi (Sec. 4.2, 4.3) ----
    lat = P["latent"]
    if opts.ablate & 2:
        Tp = T
    else:
        Tp = mlp(mlps["phi"], mlps["phi_act"], torch.cat([T[:, None], pos_enc(wi), pos_enc(P["mu"]), lat], 1))[:, 0]
    if opts.ablate & 4:
        res = torch.zeros((n, 3), dtype=DT)
    else:
        res = mlp(mlps["psi"], mlps["psi_act"], torch.cat([pos_enc(wo), pos_enc(P["mu"]), lat], 1))

    # ---- camera composite (Eq. 2) and combination (Sec. 4) ----
    img = torch.zeros((H, W, 3), dtype=DT)
    ts_c, lst_c = fr["cam_tile_start"], fr["cam_list"]
    rows = []
    for t in range(fr["ntiles"]):
        b, e = int(ts_c[t]), int(ts_c[t + 1])
        tx, ty = t % gx, t // gx
        px, py = _tile_pixels(tx, ty, W, H, ts)
        npx = px.shape[0]
        if b == e:
            rows.append((tx, ty, torch.zeros((npx, 3), dtype=DT)))
            continue
        lst = torch.from_numpy(lst_c[b:e].astype(np.int64))
        pw = _power(uv_c, con_c, lst, px, py)
        alpha = torch.clamp(gamma[lst][None] * torch.exp(pw), max=amax)
        passing = (alpha >= amin).detach()
        a = torch.where(passing, alpha, torch.zeros_like(alpha))
        l1a = torch.log1p(-a)
        incl = torch.cumsum(l1a, 1)
        excl = incl - l1a
        # a ray stops before the first passing entry that would bring T below t_stop
        stop = (passing & (torch.exp(incl) < tstop)).detach()
        after = torch.cumsum(stop.to(torch.int64), 1) > 0
        keep = ~after
        w = torch.where(keep, a * torch.exp(excl), torch.zeros_like(a))
        S = w @ col[lst]
        Sh = w @ Tp[lst]
        Rr = w @ res[lst]
        rows.append((tx, ty, S * Sh[:, None] + Rr))
    for tx, ty, vals in rows:
        h = min(H, ty * ts + ts) - ty * ts
        wdt = min(W, tx * ts + ts) - tx * ts
        img = img.index_put((torch.arange(ty * ts, ty * ts + h)[:, None],
                             torch.arange(tx * ts, tx * ts + wdt)[None]), vals.reshape(h, wdt, 3))
    return img, {"T": T, "Tp": Tp, "res": res, "shade": col}


def ssim(a, b):
    """Mean SSIM over pixels and channels: 11x11 Gaussian window, sigma 1.5,
    C1 = 0.01^2, C2 = 0.03^2, zero padding (images (H, W, 3))."""
    g = torch.exp(-((torch.arange(11, dtype=DT) - 5) ** 2) / (2 * 1.5 ** 2))
    g = g / g.sum()
    win = (g[:, None] * g[None, :])[None, None].repeat(3, 1, 1, 1)
    x = a.permute(2, 0, 1)[None]
    y = b.permute(2, 0, 1)[None]
    conv = lambda z: torch.nn.functional.conv2d(z, win, padding=5, groups=3)
    mx, my = conv(x), conv(y)
    sxx = conv(x * x) - mx * mx
    syy = conv(y * y) - my * my
    sxy = conv(x * y) - mx * my
    C1, C2 = 0.01 ** 2, 0.03 ** 2
    m = ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
    return m.mean()


def loss(img, target, lam=0.2):
    return (1 - lam) * (img - target).abs().mean() + lam * (1 - ssim(img, target))


def params_from_scene(scene, requires_grad=True):
    t = lambda a: torch.tensor(np.asarray(a, dtype=np.float64), dtype=DT, requires_grad=requires_grad)
    P = {
        "mu": t(scene.mean_op[:, :3]), "logit": t(scene.mean_op[:, 3]), "scale": t(scene.scale[:, :3]),
        "rot": t(scene.rot), "shade_rot": t(scene.shade_rot), "albedo_d": t(scene.albedo_d[:, :3]),
        "albedo_s": t(scene.albedo_s[:, :3]),
        "latent": t(np.concatenate([scene.latent[0], scene.latent[1][:, :2]], 1)),
        "lobe_rot": t(scene.lobe_rot), "lobe_sigma": t(scene.lobe_sigma[:, :, :3]),
        "lobe_amp": t(scene.lobe_amp[:, :, :3]),
    }
    mlps = {}
    for nm in ("phi", "psi"):
        m = getattr(scene, nm)
        mlps[nm] = ([t(w) for w in m.weights], [t(b) for b in m.biases])
        mlps[nm + "_act"] = m.act
    return P, mlps


def render_and_grad(scene, cam, light, target, opts=None):
    """Loss, image and the gradients of every parameter and weight."""
    opts = opts or O.Opts()
    fr = O.render(scene, cam, light, opts)
    P, mlps = params_from_scene(scene)
    img, aux = frame(P, fr, cam, light, opts, mlps)
    L = loss(img, torch.as_tensor(target, dtype=DT))
    L.backward()
    L = L.detach()
    grads = {k: v.grad.numpy().copy() for k, v in P.items()}
    for nm in ("phi", "psi"):
        grads[nm + "_w"] = [w.grad.numpy().copy() for w in mlps[nm][0]]
        grads[nm + "_b"] = [b.grad.numpy().copy() for b in mlps[nm][1]]
    return float(L), img.detach().numpy(), grads, fr


def grads_given_image_grad(scene, cam, light, dimg, opts=None):
    """Gradients of every parameter for a given dL/d(image) (H, W, 3)."""
    opts = opts or O.Opts()
    fr = O.render(scene, cam, light, opts)
    P, mlps = params_from_scene(scene)
    img, aux = frame(P, fr, cam, light, opts, mlps)
    img.backward(torch.as_tensor(np.asarray(dimg, dtype=np.float64)))
    g = lambda v: np.zeros(tuple(v.shape)) if v.grad is None else v.grad.numpy().copy()
    grads = {k: g(v) for k, v in P.items()}
    for nm in ("phi", "psi"):
        grads[nm + "_w"] = np.concatenate([g(w).reshape(-1) for w in mlps[nm][0]])
        grads[nm + "_b"] = np.concatenate([g(b).reshape(-1) for b in mlps[nm][1]])
    return grads, fr


def image_grad_of_loss(img, target, lam=0.2):
    """dL/d(image) of L = (1 - lam) L1 + lam (1 - SSIM)."""
    x = torch.as_tensor(np.asarray(img, dtype=np.float64)).clone().requires_grad_(True)
    L = loss(x, torch.as_tensor(np.asarray(target, dtype=np.float64)), lam)
    L.backward()
    return x.grad.numpy(), float(L.detach())
