"""Seeded synthetic scenes, cameras and point lights.

This module only draws inputs.  It holds none of the render arithmetic, and
both the CUDA library and the FP64 CPU oracle take their inputs from it.

Random numbers come from NumPy's Philox-4x64 counter-based generator, keyed by
(seed, stream); every parameter field has its own stream, so adding a field
never shifts the draws of another.

Distributions (the paper's Sec. 5 scenes are not available; these stand in
for trained objects of 100k-1M Gaussians at 128^2-1024^2):

* positions: uniform in the unit ball ("ball"), or a noisy sphere shell of
  radius 1 with normal offset N(0, 0.02^2) plus 10 % uniform-ball fluff
  ("shell");
* scale s = exp(U[ln 0.01, ln 0.08]) per axis (the stored parameter is s
  itself, not its logarithm);
* spatial and shading rotations: uniform unit quaternions (w, x, y, z);
* opacity logit ~ N(0, 1)  (opacity = sigmoid(logit));
* diffuse albedo U[0, 1]^3, specular albedo 1;
* latent l ~ N(0, 0.1^2) in 6-D;
* K angular Gaussians per spatial Gaussian: axis uniform on S^2 in the shading
  frame, sharpness lambda log-uniform in [1, 100], RGB amplitude U[0, 0.5]^3.
  The isotropic reduction of Eq. 5 is used: sigma_x = sigma_y = 1,
  sigma_z = lambda^(-1/2), and the lobe frame is the minimal rotation taking
  e_z to the axis;
* MLP weights: Xavier-uniform, zero biases;
* camera and light: on the radius-3 sphere in seeded directions, the camera a
  pinhole with a 40 degree vertical field of view looking at the origin.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# field -> Philox stream id
_STREAMS = {
    "pos": 1, "pos_dir": 2, "pos_r": 3, "scale": 4, "rot": 5, "opacity": 6,
    "albedo": 7, "shade_rot": 8, "latent": 9, "lobe_axis": 10, "lobe_sharp": 11,
    "lobe_amp": 12, "phi": 13, "psi": 14, "camera": 15, "light": 16,
    "shell_noise": 17, "perturb": 18, "environment": 19, "init": 20, "basis": 21,
    "layers": 22,
}

RELU = 0
LEAKY_RELU = 1


def rng(seed: int, stream: str) -> np.random.Generator:
    """Philox generator for one (seed, field) pair."""
    key = np.array([seed & 0xFFFFFFFFFFFFFFFF, _STREAMS[stream]], dtype=np.uint64)
    return np.random.Generator(np.random.Philox(key=key))


def _unit_vectors(g: np.random.Generator, n: int) -> np.ndarray:
    v = g.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v


def _unit_quats(g: np.random.Generator, n: int) -> np.ndarray:
    q = g.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _quat_from_z(axis: np.ndarray) -> np.ndarray:
    """Unit quaternion (w,x,y,z) of the minimal rotation taking e_z to axis."""
    a = axis
    w = 1.0 + a[:, 2]
    q = np.stack([w, -a[:, 1], a[:, 0], np.zeros_like(w)], axis=1)
    bad = w < 1e-9  # axis = -e_z: half turn about x
    q[bad] = np.array([0.0, 1.0, 0.0, 0.0])
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


@dataclass
class MLP:
    """Fully connected net: in_dim -> [width] * n_hidden -> out_dim."""
    in_dim: int
    width: int
    n_hidden: int
    out_dim: int
    act: int
    weights: list = field(default_factory=list)   # float32 (out, in) per layer
    biases: list = field(default_factory=list)    # float32 (out,) per layer

    def dims(self):
        d = [self.in_dim] + [self.width] * self.n_hidden + [self.out_dim]
        return list(zip(d[:-1], d[1:]))

    def packed(self):
        w = np.concatenate([x.reshape(-1) for x in self.weights]).astype(np.float32)
        b = np.concatenate([x.reshape(-1) for x in self.biases]).astype(np.float32)
        return np.ascontiguousarray(w), np.ascontiguousarray(b)


def make_mlp(seed: int, stream: str, in_dim: int, width: int, n_hidden: int,
             out_dim: int, act: int) -> MLP:
    g = rng(seed, stream)
    m = MLP(in_dim, width, n_hidden, out_dim, act)
    for fi, fo in m.dims():
        a = math.sqrt(6.0 / (fi + fo))
        m.weights.append(g.uniform(-a, a, (fo, fi)).astype(np.float32))
        m.biases.append(np.zeros(fo, dtype=np.float32))
    return m


@dataclass
class Scene:
    """Structure-of-arrays float32 parameters, float4-padded.

    mean_op[N,4]   x, y, z, opacity logit
    scale[N,4]     sx, sy, sz, 0           (positive)
    rot[N,4]       w, x, y, z              spatial rotation (unnormalised)
    shade_rot[N,4] w, x, y, z              world -> shading frame
    albedo_d[N,4]  rho_d rgb, 0
    albedo_s[N,4]  rho_s rgb, 0
    latent[2,N,4]  (l0..l3), (l4, l5, 0, 0)
    lobe_rot[K,N,4]   w, x, y, z           lobe frame inside the shading frame
    lobe_sigma[K,N,4] sigma_x, sigma_y, sigma_z, 0
    lobe_amp[K,N,4]   alpha rgb, 0
    """
    n: int
    k: int
    mean_op: np.ndarray
    scale: np.ndarray
    rot: np.ndarray
    shade_rot: np.ndarray
    albedo_d: np.ndarray
    albedo_s: np.ndarray
    latent: np.ndarray
    lobe_rot: np.ndarray
    lobe_sigma: np.ndarray
    lobe_amp: np.ndarray
    phi: MLP
    psi: MLP
    lobe_shared: bool = False  # lobe_rot / lobe_sigma are one shared basis [K, 1, 4]

    ARRAYS = ("mean_op", "scale", "rot", "shade_rot", "albedo_d", "albedo_s",
              "latent", "lobe_rot", "lobe_sigma", "lobe_amp")

    def arrays(self):
        return {a: getattr(self, a) for a in self.ARRAYS}

    def copy(self) -> "Scene":
        s = Scene(self.n, self.k, *[getattr(self, a).copy() for a in self.ARRAYS],
                  phi=MLP(self.phi.in_dim, self.phi.width, self.phi.n_hidden,
                          self.phi.out_dim, self.phi.act,
                          [w.copy() for w in self.phi.weights],
                          [b.copy() for b in self.phi.biases]),
                  psi=MLP(self.psi.in_dim, self.psi.width, self.psi.n_hidden,
                          self.psi.out_dim, self.psi.act,
                          [w.copy() for w in self.psi.weights],
                          [b.copy() for b in self.psi.biases]),
                  lobe_shared=self.lobe_shared)
        return s

    def nbytes(self) -> int:
        return sum(a.nbytes for a in self.arrays().values())


@dataclass
class Camera:
    """Pinhole camera: view rotation rows R (world -> camera, x right, y down,
    z forward), translation t, focal lengths and principal point in pixels,
    centre position pos (world)."""
    R: np.ndarray
    t: np.ndarray
    pos: np.ndarray
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int


@dataclass
class Light:
    """Point light at pos (type 0, Sec. 4.2) or directional light from the scene
    towards dir (type 1, Sec. 4.5) with an orthographic light view of
    half-width extent; intensity is I of the point light's I / d^2, or the
    directional light's irradiance."""
    pos: np.ndarray
    intensity: float
    type: int = 0
    dir: np.ndarray | None = None
    extent: float = 0.0


def _positions(g_dir, g_r, g_noise, n: int, kind: str) -> np.ndarray:
    if kind == "ball":
        d = _unit_vectors(g_dir, n)
        r = g_r.random(n) ** (1.0 / 3.0)
        return d * r[:, None]
    if kind == "shell":
        n_fluff = n // 10
        n_shell = n - n_fluff
        d = _unit_vectors(g_dir, n_shell)
        r = 1.0 + 0.02 * g_noise.standard_normal(n_shell)
        shell = d * r[:, None]
        d2 = _unit_vectors(g_dir, n_fluff)
        r2 = g_r.random(n_fluff) ** (1.0 / 3.0)
        return np.concatenate([shell, d2 * r2[:, None]], axis=0)
    raise ValueError(kind)


def make_scene(seed: int, n: int, k: int, kind: str = "ball", *, mlp_width: int = 64,
               mlp_hidden: int = 2, act: int = RELU, phi_width: int | None = None,
               phi_hidden: int | None = None) -> Scene:
    """Draw one scene; see the module docstring for the distributions."""
    pos = _positions(rng(seed, "pos_dir"), rng(seed, "pos_r"), rng(seed, "shell_noise"), n, kind)
    g = rng(seed, "scale")
    scale = np.exp(g.uniform(math.log(0.01), math.log(0.08), (n, 3)))
    rot = _unit_quats(rng(seed, "rot"), n)
    logit = rng(seed, "opacity").standard_normal(n)
    albedo = rng(seed, "albedo").random((n, 3))
    shade_rot = _unit_quats(rng(seed, "shade_rot"), n)
    latent = 0.1 * rng(seed, "latent").standard_normal((n, 6))
    axis = _unit_vectors(rng(seed, "lobe_axis"), n * k).reshape(k, n, 3) if k else np.zeros((0, n, 3))
    lam = np.exp(rng(seed, "lobe_sharp").uniform(0.0, math.log(100.0), (k, n)))
    amp = rng(seed, "lobe_amp").uniform(0.0, 0.5, (k, n, 3))

    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    z1 = np.zeros((n, 1))
    mean_op = f32(np.concatenate([pos, logit[:, None]], axis=1))
    lobe_rot = np.zeros((k, n, 4))
    lobe_sigma = np.zeros((k, n, 4))
    lobe_amp = np.zeros((k, n, 4))
    for j in range(k):
        lobe_rot[j] = _quat_from_z(axis[j])
        lobe_sigma[j, :, 0] = 1.0
        lobe_sigma[j, :, 1] = 1.0
        lobe_sigma[j, :, 2] = lam[j] ** -0.5
        lobe_amp[j, :, :3] = amp[j]
    lat = np.zeros((2, n, 4))
    lat[0] = latent[:, :4]
    lat[1, :, :2] = latent[:, 4:]
    pw = phi_width if phi_width is not None else mlp_width
    ph = phi_hidden if phi_hidden is not None else mlp_hidden
    return Scene(
        n=n, k=k,
        mean_op=mean_op,
        scale=f32(np.concatenate([scale, z1], axis=1)),
        rot=f32(rot), shade_rot=f32(shade_rot),
        albedo_d=f32(np.concatenate([albedo, z1], axis=1)),
        albedo_s=f32(np.concatenate([np.ones((n, 3)), z1], axis=1)),
        latent=f32(lat), lobe_rot=f32(lobe_rot), lobe_sigma=f32(lobe_sigma),
        lobe_amp=f32(lobe_amp),
        phi=make_mlp(seed, "phi", 61, pw, ph, 1, act),
        psi=make_mlp(seed, "psi", 60, mlp_width, mlp_hidden, 3, act),
    )


def with_shared_basis(scene: Scene, seed: int) -> Scene:
    """The scene with its lobes replaced by one basis of K anisotropic angular
    Gaussians shared by every spatial Gaussian (Sec. 4.1): uniform random lobe
    frames, sigma_x, sigma_y ~ U[0.3, 1], sigma_z = lambda^-1/2 with lambda
    log-uniform in [1, 100]; each spatial Gaussian keeps its RGB weights."""
    s = scene.copy()
    k = s.k
    g = rng(seed, "basis")
    rot = _unit_quats(g, k)
    sig = np.zeros((k, 1, 4))
    sig[:, 0, 0] = g.uniform(0.3, 1.0, k)
    sig[:, 0, 1] = g.uniform(0.3, 1.0, k)
    sig[:, 0, 2] = np.exp(g.uniform(0.0, math.log(100.0), k)) ** -0.5
    s.lobe_rot = np.ascontiguousarray(rot.reshape(k, 1, 4), dtype=np.float32)
    s.lobe_sigma = np.ascontiguousarray(sig, dtype=np.float32)
    s.lobe_shared = True
    return s


def look_at_camera(pos, target=(0.0, 0.0, 0.0), fov_y_deg: float = 40.0,
                   width: int = 128, height: int = 128) -> Camera:
    """Camera at pos looking at target, world +z up (+y when nearly parallel)."""
    pos = np.asarray(pos, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - pos
    f /= np.linalg.norm(f)
    up = np.array([0.0, 0.0, 1.0]) if abs(f[2]) <= 0.999 else np.array([0.0, 1.0, 0.0])
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f], axis=0)
    t = -R @ pos
    foc = 0.5 * height / math.tan(math.radians(fov_y_deg) * 0.5)
    return Camera(R=R.astype(np.float32), t=t.astype(np.float32), pos=pos.astype(np.float32),
                  fx=float(np.float32(foc)), fy=float(np.float32(foc)),
                  cx=float(np.float32(0.5 * width)), cy=float(np.float32(0.5 * height)),
                  width=width, height=height)


def camera_light_pair(seed: int, width: int, height: int, radius: float = 3.0,
                      fov_y_deg: float = 40.0, intensity: float = 10.0):
    """Seeded (camera, point light) pair on the radius-`radius` sphere."""
    cdir = _unit_vectors(rng(seed, "camera"), 1)[0]
    ldir = _unit_vectors(rng(seed, "light"), 1)[0]
    cam = look_at_camera(radius * cdir, fov_y_deg=fov_y_deg, width=width, height=height)
    light = Light(pos=(radius * ldir).astype(np.float32), intensity=float(np.float32(intensity)))
    return cam, light


def directional_light(seed: int, intensity: float = 10.0 / 9.0, extent: float = 1.25) -> Light:
    """Seeded directional light (the point light's direction of the same seed;
    irradiance 10/9 = the point light's I / d^2 at the scene centre)."""
    ldir = _unit_vectors(rng(seed, "light"), 1)[0].astype(np.float32)
    return Light(pos=np.zeros(3, dtype=np.float32), intensity=float(np.float32(intensity)), type=1,
                 dir=ldir, extent=float(np.float32(extent)))


def environment_lights(seed: int, count: int, extent: float = 1.25):
    """`count` seeded directional lights on the sphere with weights summing to
    the solid angle per sample (an environment light sampled uniformly;
    radiance U[0, 1] per direction)."""
    g = rng(seed, "environment")
    dirs = _unit_vectors(g, count).astype(np.float32)
    radiance = g.uniform(0.0, 1.0, count)
    weights = (4.0 * np.pi / count * radiance).astype(np.float32)
    lights = [Light(pos=np.zeros(3, dtype=np.float32), intensity=1.0, type=1, dir=d, extent=float(np.float32(extent)))
              for d in dirs]
    return lights, weights


def paper_initialisation(scene: Scene, seed: int) -> Scene:
    """Copy with the appearance reset to the initial values of Sec. 4.4:
    sigma_x = 0.5, sigma_y = 1, sigma_z ~ U[0.13, 0.69]; rho_d = rho_s = 1;
    every lobe weight 0.5; shading and lobe frames aligned with the world
    axes (identity quaternions).  Geometry, latent and MLPs are kept."""
    s = scene.copy()
    g = rng(seed, "init")
    s.albedo_d[:, :3] = 1.0
    s.albedo_s[:, :3] = 1.0
    s.shade_rot[:] = np.array([1.0, 0.0, 0.0, 0.0], dtype=np.float32)
    if s.k:
        s.lobe_rot[:] = np.array([1.0, 0.0, 0.0, 0.0], dtype=np.float32)
        s.lobe_sigma[..., 0] = 0.5
        s.lobe_sigma[..., 1] = 1.0
        s.lobe_sigma[..., 2] = g.uniform(0.13, 0.69, s.lobe_sigma.shape[:2]).astype(np.float32)
        s.lobe_amp[..., :3] = 0.5
    return s


def perturbed(scene: Scene, seed: int) -> Scene:
    """Copy with mean += N(0, 0.01^2) and diffuse albedo *= U[0.9, 1.1]."""
    s = scene.copy()
    g = rng(seed, "perturb")
    s.mean_op[:, :3] += (0.01 * g.standard_normal((s.n, 3))).astype(np.float32)
    s.albedo_d[:, :3] *= g.uniform(0.9, 1.1, (s.n, 3)).astype(np.float32)
    return s


def layered_scene(seed: int, layers: int = 24, grid: int = 10, k: int = 2, pitch: float = 0.06,
                  gap: float = 0.03) -> Scene:
    """A stack of `layers` planes of grid x grid nearly opaque Gaussians
    (logit N(6, 1), flattened scales U[0.035, 0.05] x U[0.035, 0.05] x 0.01,
    centres on a `pitch` grid jittered by N(0, (pitch / 10)^2)) normal to z, the
    planes `gap` apart from z = +(layers - 1) gap / 2 down.  Seen from a
    light on the +z axis every shadow ray through the stack crosses all
    planes, so its occluder product falls far below the FP32 range."""
    n = layers * grid * grid
    base = make_scene(seed, n, k, "ball", mlp_width=32, mlp_hidden=2)
    g = rng(seed, "layers")
    ij = (np.arange(grid) - (grid - 1) / 2.0) * pitch
    X, Y = np.meshgrid(ij, ij)
    xy = np.tile(np.stack([X.ravel(), Y.ravel()], 1), (layers, 1)) + g.normal(0.0, pitch / 10.0, (n, 2))
    z = np.repeat((layers - 1) / 2.0 * gap - gap * np.arange(layers), grid * grid)
    base.mean_op[:, :3] = np.concatenate([xy, z[:, None]], 1).astype(np.float32)
    base.mean_op[:, 3] = g.normal(6.0, 1.0, n).astype(np.float32)
    base.scale[:, :2] = g.uniform(0.035, 0.05, (n, 2)).astype(np.float32)
    base.scale[:, 2] = np.float32(0.01)
    q = np.concatenate([np.ones((n, 1)), 0.05 * g.standard_normal((n, 3))], 1)
    base.rot = np.ascontiguousarray(q / np.linalg.norm(q, axis=1, keepdims=True), dtype=np.float32)
    return base


# Named workloads -----------------------------------------------------------

def tiny_scene(seed: int = 0) -> Scene:
    """1,000 Gaussians in the unit ball, K = 4, both MLPs 2x64 ReLU."""
    return make_scene(seed, 1000, 4, "ball", mlp_width=64, mlp_hidden=2, act=RELU)


def object_scene(seed: int = 0, n: int = 300_000, k: int = 8) -> Scene:
    """Sphere shell + 10 % fluff, K = 8, both MLPs 3x128 ReLU."""
    return make_scene(seed, n, k, "shell", mlp_width=128, mlp_hidden=3, act=RELU)


def paper_mlp_scene(seed: int = 0, n: int = 1000, k: int = 8) -> Scene:
    """Paper's MLP sizes: Phi {32,32,32}, Psi {128,128,128}, leaky ReLU."""
    return make_scene(seed, n, k, "ball", mlp_width=128, mlp_hidden=3, act=LEAKY_RELU,
                      phi_width=32, phi_hidden=3)
