"""Pins of the oracle's directional and environment lighting (Sec. 4.5), CPU.

A directional light replaces the shadow splat's perspective camera with an
orthographic one; its irradiance does not fall off and omega_i is the same
for every Gaussian.  An environment light is a linear combination of
directional renders.  The pins use facts only orthographic projection has
(footprint independent of position and depth, screen offsets proportional to
world offsets, depth = position along the axis) and closed forms.
"""
import math

import numpy as np
import pytest

from paper_2410_11419_gb300 import synth
from tests import bruteforce
from tests.test_oracle_pins import np_mlp, np_pe, one_gaussian_scene


def dlight(d, extent=1.25, intensity=2.0):
    d = np.asarray(d, dtype=np.float64)
    d = (d / np.linalg.norm(d)).astype(np.float32)
    return synth.Light(pos=np.zeros(3, dtype=np.float32), intensity=intensity, type=1, dir=d,
                       extent=float(np.float32(extent)))


def test_orthographic_view_geometry(oracle):
    """The light view looks along -dir, its half-width is `extent` world units
    (s = min(W, H) / (2 extent) pixels per unit), and its depth is the
    position along the axis."""
    W, H = 96, 64
    for d in ([0.3, -0.5, 0.8], [0.0, 0.0, 1.0], [-1.0, 0.2, 0.1]):
        L = dlight(d, extent=1.5)
        R, t, s = oracle.light_view_any(L, W, H)
        R = R.astype(np.float64)
        assert s == pytest.approx(min(W, H) / (2 * 1.5), rel=1e-7)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-6)
        np.testing.assert_allclose(R[2], -L.dir, atol=1e-6)           # forward = -dir
        # a point `extent` to the right of the target lands half the short side right of centre
        p = 1.5 * R[0]
        x = R @ p + t
        assert s * x[0] == pytest.approx(min(W, H) / 2, rel=1e-5)
        # depth grows by delta when the point moves delta away from the light
        z0 = (R @ np.zeros(3) + t)[2]
        z1 = (R @ (-0.25 * L.dir.astype(np.float64)) + t)[2]
        assert z1 - z0 == pytest.approx(0.25, abs=1e-5)
        assert z0 == pytest.approx(4 * 1.5, rel=1e-6)                 # the eye is 4 extents out


def test_orthographic_footprint(oracle):
    """Orthographic EWA: an isotropic Gaussian has Sigma_2D = (s sigma)^2 I + 0.3 I
    wherever it is; an anisotropic one keeps its footprint when moved along
    the axis or sideways, while its screen position moves by s times the
    sideways offset."""
    W, H = 64, 64
    cam = synth.look_at_camera([0.0, 0.0, 3.0], width=W, height=H)
    L = dlight([0.2, 0.4, 0.9])
    R, t, s = oracle.light_view_any(L, W, H)
    sig = 0.05
    for m in ([0, 0, 0], [0.3, -0.2, 0.1], [-0.5, 0.4, -0.3]):
        uv, con = oracle.project(m, [sig] * 3, [1, 0, 0, 0], R, t, cam.fx, cam.fy, cam.cx, cam.cy,
                                 ortho=s)
        var = (float(s) * float(np.float32(sig))) ** 2 + 0.3
        np.testing.assert_allclose(con, [1 / var, 0.0, 1 / var], rtol=1e-6, atol=1e-12)
    q = [0.4, 0.2, -0.6, 0.3]
    sc = [0.02, 0.07, 0.04]
    base_uv, base_con = oracle.project([0, 0, 0], sc, q, R, t, cam.fx, cam.fy, cam.cx, cam.cy, ortho=s)
    np.testing.assert_allclose(base_uv, [cam.cx, cam.cy], atol=1e-5)
    Rd = R.astype(np.float64)
    for off, du in ((0.4 * L.dir.astype(np.float64), 0.0), (0.3 * Rd[0], 0.3 * s), (-0.2 * Rd[1], 0.0)):
        uv, con = oracle.project(off, sc, q, R, t, cam.fx, cam.fy, cam.cx, cam.cy, ortho=s)
        np.testing.assert_allclose(con, base_con, rtol=1e-5)
        assert uv[0] - base_uv[0] == pytest.approx(du, abs=1e-4)


def test_orthographic_keys_are_axial_depths(oracle):
    """The light splat's key is the FP32 depth along the view axis; a
    Gaussian closer to the light sorts first."""
    sc = one_gaussian_scene([[0.0, 0.0, 0.3], [0.0, 0.0, 0.0], [0.0, 0.0, -0.4]], 0.05)
    cam = synth.look_at_camera([3.0, 0.0, 0.0], width=64, height=64)
    L = dlight([0.0, 0.0, 1.0])
    fr = oracle.render(sc, cam, L)
    d = fr["light_key"].view(np.float32).astype(np.float64)
    np.testing.assert_allclose(d, [5.0 - 0.3, 5.0, 5.0 + 0.4], atol=1e-5)  # eye 4 x 1.25 out
    # the three share one screen position (one ray), unlike a perspective light
    np.testing.assert_allclose(fr["light_uv"], np.tile(fr["light_uv"][1], (3, 1)), atol=1e-6)


def test_directional_shading_closed_form(oracle):
    """dir = e_z with identity frames and the camera above: f_d = 1/pi, each lobe
    1/sigma_z, E = the light's irradiance (no fall-off, even with fall-off on),
    and the colour does not depend on the Gaussian's distance to the light."""
    cam = synth.look_at_camera([0.0, 0.0, 3.0], width=32, height=32)
    L = dlight([0.0, 0.0, 1.0], intensity=2.0)
    amp = np.array([0.2, 0.3, 0.4], dtype=np.float32).astype(np.float64)
    rho = np.array([0.8, 0.5, 0.2], dtype=np.float32).astype(np.float64)
    sz = float(np.float32(0.3))
    want = 2.0 * (rho / math.pi + 2 * amp / sz)
    for z in (0.0, -1.0):
        sc = one_gaussian_scene([0.0, 0.0, z], 0.05, k=2)
        np.testing.assert_allclose(oracle.shade(sc, 0, cam, L), want, rtol=1e-12)
        np.testing.assert_allclose(oracle.shade(sc, 0, cam, L, oracle.Opts(falloff=0)), want, rtol=1e-12)


def test_directional_shadow_two_gaussians(oracle):
    """A receiver behind an occluder along the light direction gets
    sum_m beta_m (1 - alpha_front,m) / sum_m beta_m over its light pixels;
    within the 0.015 bias it is unshadowed.  Orthographic, so both splats
    land on the same pixels whatever their separation."""
    L = dlight([0.0, 0.0, 1.0])
    cam = synth.look_at_camera([3.0, 0.0, 0.0], width=64, height=64)
    for sep, shadowed in ((0.6, True), (0.01, False)):
        sc = one_gaussian_scene([[0.0, 0.0, 0.3], [0.0, 0.0, 0.3 - sep]], [0.05, 0.05, 0.05],
                                logit=[1.0, 0.5])
        fr = oracle.render(sc, cam, L)
        assert fr["T"][0] == 1.0
        if not shadowed:
            assert fr["T"][1] == 1.0
            continue
        ys, xs = np.mgrid[0:64, 0:64]

        def ab(g):
            u, v = fr["light_uv"][g]
            A, B, Cc = fr["light_conic"][g]
            dx, dy = xs + 0.5 - u, ys + 0.5 - v
            beta = np.exp(-0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy)
            a = np.minimum(0.99, fr["opacity"][g] * beta)
            rect = fr["light_rect"][g]
            inside = (xs // 16 >= rect[0]) & (xs // 16 <= rect[2]) & (ys // 16 >= rect[1]) & (ys // 16 <= rect[3])
            return beta, a, inside & (a >= 1 / 255)

        b0, a0, ok0 = ab(0)
        b1, a1, ok1 = ab(1)
        # orthographic: identical footprints, so the ratio is the mean of (1 - alpha_front) under beta
        np.testing.assert_allclose(fr["light_conic"][0], fr["light_conic"][1], rtol=1e-6)
        Tm = np.where(ok0, 1 - a0, 1.0)
        want = (b1 * Tm)[ok1].sum() / b1[ok1].sum()
        assert fr["T"][1] == pytest.approx(want, rel=1e-12)
        assert want < 0.8


@pytest.fixture(scope="module")
def directional_frame(oracle):
    sc = synth.make_scene(7, 300, 3, "ball")
    cam, _ = synth.camera_light_pair(7, 48, 40)
    L = synth.directional_light(7)
    opts = oracle.Opts()
    return sc, cam, L, opts, oracle.render(sc, cam, L, opts)


def test_directional_shadow_bruteforce(directional_frame):
    """The tiled two-cursor shadow splat equals the O(L^2) definition under an
    orthographic light view too."""
    sc, cam, L, opts, fr = directional_frame
    T = bruteforce.shadow_values(fr, opts)
    np.testing.assert_allclose(fr["T"], T, rtol=1e-11, atol=1e-14)
    assert fr["T"].min() < 0.9


def test_directional_mlp_inputs(directional_frame):
    """Phi sees the same omega_i = dir for every Gaussian."""
    sc, cam, L, opts, fr = directional_frame
    mu = sc.mean_op[:, :3].astype(np.float64)
    lat = np.concatenate([sc.latent[0], sc.latent[1][:, :2]], 1).astype(np.float64)
    wi = L.dir.astype(np.float64) / np.linalg.norm(L.dir.astype(np.float64))
    xphi = np.stack([np.concatenate([[fr["T"][g]], np_pe(wi), np_pe(mu[g]), lat[g]]) for g in range(sc.n)])
    np.testing.assert_allclose(fr["Tp"], np_mlp(sc.phi, xphi)[:, 0], rtol=1e-12)


def test_environment_is_linear_combination(oracle):
    """Sec. 4.5: the environment render is sum_l w_l render(dir_l); with one
    light of weight w it is w times that light's render, and the weights
    scale it linearly."""
    sc = synth.make_scene(3, 200, 2, "ball")
    cam, _ = synth.camera_light_pair(3, 40, 40)
    lights, w = synth.environment_lights(5, 3)
    frames = [oracle.render(sc, cam, L)["img"] for L in lights]
    env = oracle.environment(sc, cam, lights, w)
    np.testing.assert_allclose(env, sum(float(wi) * f for wi, f in zip(w, frames)), rtol=1e-12)
    np.testing.assert_allclose(oracle.environment(sc, cam, lights[:1], [2.0]), 2.0 * frames[0], rtol=1e-12)
    assert abs(float(np.sum(w)) - 4 * math.pi * 0.5) < 4 * math.pi  # weights are solid-angle sized
