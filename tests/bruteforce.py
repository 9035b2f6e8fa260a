"""Brute-force NumPy restatement of the splat and shadow definitions for tiny
scenes (test helper for the oracle pins).

No tiling data structure: every pixel scans all N Gaussians, keeps those whose
tile rectangle contains the pixel's tile, orders them by (depth bits, index)
and applies Eq. 2 directly.  Shadow values use the direct product definition
T_m(j) = prod over passing k with d_k < d_j - bias of (1 - alpha_k) -- an
O(L^2) product per ray with no prefix or cursor trick.
"""
import numpy as np


def _alpha(uv, conic, opac, px, py, amax):
    dx = px - uv[:, 0]
    dy = py - uv[:, 1]
    power = -0.5 * (conic[:, 0] * dx * dx + conic[:, 2] * dy * dy) - conic[:, 1] * dx * dy
    beta = np.exp(power)
    a = np.minimum(amax, opac * beta)
    return power, beta, a


def _amin(opts):
    """alpha_min as the renderers hold it: an FP32 number."""
    return float(np.float32(opts.alpha_min))


def _amax(opts):
    """alpha_max as the renderers hold it: an FP32 number."""
    return float(np.float32(opts.alpha_max))


def candidates(rect, key, tx, ty):
    inside = (rect[:, 0] >= 0) & (rect[:, 0] <= tx) & (tx <= rect[:, 2]) & \
             (rect[:, 1] <= ty) & (ty <= rect[:, 3])
    idx = np.nonzero(inside)[0]
    order = np.lexsort((idx, key[idx]))  # by key, then index
    return idx[order]


def shadow_values(fr, opts):
    """Per-Gaussian shadow value from the oracle's light-view geometry."""
    n, W, H, ts = fr["n"], fr["width"], fr["height"], opts.tile
    num = np.zeros(n)
    den = np.zeros(n)
    d_all = fr["light_key"].view(np.float32)
    bias = np.float32(opts.shadow_bias)
    for ty in range((H + ts - 1) // ts):
        for tx in range((W + ts - 1) // ts):
            lst = candidates(fr["light_rect"], fr["light_key"], tx, ty)
            if lst.size == 0:
                continue
            uv, con, op = fr["light_uv"][lst], fr["light_conic"][lst], fr["opacity"][lst]
            d = d_all[lst]
            thr = (d - bias).astype(np.float32)
            for py in range(ty * ts, min(H, ty * ts + ts)):
                for px in range(tx * ts, min(W, tx * ts + ts)):
                    power, beta, a = _alpha(uv, con, op, px + 0.5, py + 0.5, _amax(opts))
                    ok = a >= _amin(opts)
                    if not ok.any():
                        continue
                    occ = (d[None, :] < thr[:, None]) & ok[None, :]
                    Tm = np.prod(np.where(occ, 1.0 - a[None, :], 1.0), axis=1)
                    np.add.at(num, lst[ok], (beta * Tm)[ok])
                    np.add.at(den, lst[ok], beta[ok])
    return np.where(den > 0, num / np.where(den > 0, den, 1), 1.0)


def shadow_values_stopped(fr, opts, stop):
    """Shadow values when a ray stops taking occluders once its product is
    below `stop`: walking the ray's entries in depth order, a passing entry
    multiplies the running product only while that product is >= stop, and
    receiver j sees the running product after the entries with
    d_k < d_j - bias.  Also returns, per ray, the exact product over every
    passing entry (log2) and the smallest frozen product."""
    n, W, H, ts = fr["n"], fr["width"], fr["height"], opts.tile
    num = np.zeros(n)
    den = np.zeros(n)
    d_all = fr["light_key"].view(np.float32)
    bias = np.float32(opts.shadow_bias)
    log2_exact, frozen_min = [], []
    for ty in range((H + ts - 1) // ts):
        for tx in range((W + ts - 1) // ts):
            lst = candidates(fr["light_rect"], fr["light_key"], tx, ty)
            if lst.size == 0:
                continue
            uv, con, op = fr["light_uv"][lst], fr["light_conic"][lst], fr["opacity"][lst]
            d = d_all[lst]
            thr = (d - bias).astype(np.float32)
            K = np.searchsorted(d, thr, side="left")  # entries with d_k < thr_j (d is sorted)
            for py in range(ty * ts, min(H, ty * ts + ts)):
                for px in range(tx * ts, min(W, tx * ts + ts)):
                    power, beta, a = _alpha(uv, con, op, px + 0.5, py + 0.5, _amax(opts))
                    ok = a >= _amin(opts)
                    if not ok.any():
                        continue
                    run = np.empty(lst.size + 1)
                    run[0] = 1.0
                    for i in range(lst.size):
                        take = ok[i] and run[i] >= stop
                        run[i + 1] = run[i] * (1.0 - a[i]) if take else run[i]
                    log2_exact.append(np.log2(np.where(ok, 1.0 - a, 1.0)).sum())
                    frozen_min.append(run[-1])
                    Tm = run[K]
                    np.add.at(num, lst[ok], (beta * Tm)[ok])
                    np.add.at(den, lst[ok], beta[ok])
    T = np.where(den > 0, num / np.where(den > 0, den, 1), 1.0)
    return T, np.array(log2_exact), np.array(frozen_min)


def composite(fr, opts, shade, Tp, res):
    """Camera image S * Sh + R and final transmittance, by Eq. 2."""
    W, H, ts = fr["width"], fr["height"], opts.tile
    img = np.zeros((H, W, 3))
    fT = np.ones((H, W))
    wsum = np.zeros((H, W))
    for py in range(H):
        for px in range(W):
            lst = candidates(fr["cam_rect"], fr["cam_key"], px // ts, py // ts)
            T = 1.0
            S = np.zeros(3)
            Sh = 0.0
            R = np.zeros(3)
            ws = 0.0
            for g in lst:
                dx = px + 0.5 - fr["cam_uv"][g, 0]
                dy = py + 0.5 - fr["cam_uv"][g, 1]
                A, B, Cc = fr["cam_conic"][g]
                power = -0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy  # <= 0: positive-definite conic
                a = min(_amax(opts), fr["opacity"][g] * np.exp(power))
                if a < _amin(opts):
                    continue
                Tn = T * (1 - a)
                if Tn < opts.t_stop:
                    break
                w = a * T
                S += w * shade[g]
                Sh += w * Tp[g]
                R += w * res[g]
                ws += w
                T = Tn
            img[py, px] = S * Sh + R
            fT[py, px] = T
            wsum[py, px] = ws
    return img, fT, wsum
