"""Seeded workloads: frame pairs and sequences with ground truth.

Every workload is a deterministic function of its seed. Frames are rendered on
demand (``Sequence.frame(k)``); per-frame noise uses the generator
``default_rng([seed, k])`` so any frame can be regenerated alone.

Workload recipes (they stand in for the Replica renders the paper used, which
are not available here):

* ``tiny_pair``   64x48, fx=fy=60, cx=32, cy=24; three textured planes, depth
  1-4 m; 8x8-pixel uniform-random block texture; true motion 2 cm + 0.5 deg
  about seeded random directions; Gaussian noise sigma 1/255.
* ``scamp_room``  256x256, fx=fy=128, cx=cy=127.5; camera inside a textured
  box room (0.5-5 m) with a box on the floor; smooth trajectory (sum of three
  sinusoids per axis) scaled to 1 cm and 0.3 deg per frame; noise sigma 2/255.
* ``realistic``   640x480, fx=fy=525, cx=319.5, cy=239.5; ground plane, back
  wall, a near surface patch and a side curtain (the last two sinusoidal
  height fields), depth ~0.7-8 m; per-frame motion U[0, 3 cm] and U[0, 1 deg]
  along smoothly varying directions; noise sigma 2/255, 8-bit quantisation,
  1% dropout pixels set to 0.
* ``batched_family`` 64 sequences (seeds 1000..1063) of the realistic scene
  family at resolutions drawn from {128x96, 256x256, 320x240, 640x480},
  fx=fy=0.8203*W, cx=(W-1)/2, cy=(H-1)/2.
* ``adjoint_family`` 8 sequences of the realistic family at 320x240.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy.spatial.transform import Rotation

from .scenes import (BlockTexture, Camera, HeightField, Plane, Scene,
                     SmoothTexture, render)


def _pose(R, t):
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = t
    return T


def _inv(T):
    R, t = T[:3, :3], T[:3, 3]
    return _pose(R.T, -R.T @ t)


@dataclass
class Sequence:
    """A camera moving through a static scene.

    ``poses[k]`` is the camera-to-world pose of frame k. ``kf_interval``,
    ``sweeps`` and ``sigma_P`` are the tracking schedule and pose-prior strength
    the workload is run with (the prior is the weakest one found not to diverge
    early on that workload family, the selection rule of the paper's App. E.3).
    """
    name: str
    cam: Camera
    scene: Scene
    poses: np.ndarray
    seed: int
    noise_sigma: float
    quantize: bool = False
    dropout: float = 0.0
    sweeps: int = 20
    kf_interval: int = 10
    sigma_P: float = 0.05

    def __post_init__(self):
        self._cache = {}

    @property
    def n_frames(self) -> int:
        return len(self.poses)

    def clean(self, k: int) -> dict:
        if k not in self._cache:
            if len(self._cache) > 8:
                self._cache.clear()
            self._cache[k] = render(self.scene, self.poses[k], self.cam)
        return self._cache[k]

    def frame(self, k: int) -> np.ndarray:
        """Noisy float32 intensity image of frame k (row-major H x W)."""
        img = self.clean(k)["image"].copy()
        rng = np.random.default_rng([self.seed, k])
        if self.noise_sigma > 0:
            img = img + rng.normal(0.0, self.noise_sigma, img.shape)
        if self.quantize:
            img = np.round(255.0 * np.clip(img, 0.0, 1.0)) / 255.0
        if self.dropout > 0:
            img = np.where(rng.random(img.shape) < self.dropout, 0.0, img)
        return img.astype(np.float32)

    def normals(self, k: int) -> np.ndarray:
        """Ground-truth camera-frame unit normals of frame k, float32 (H, W, 3)."""
        return self.clean(k)["normal"].astype(np.float32)

    def depth(self, k: int) -> np.ndarray:
        return self.clean(k)["depth"]

    def relative_pose(self, s: int, t: int) -> np.ndarray:
        """T_{t<-s}: maps frame-s camera coordinates to frame-t camera coordinates."""
        return _inv(self.poses[t]) @ self.poses[s]


# --------------------------------------------------------------------------
# config: tiny frame pair
# --------------------------------------------------------------------------
def _tilted_normal(rng, max_deg):
    """Unit vector within max_deg of -z (facing a camera looking along +z)."""
    ang = np.deg2rad(rng.uniform(0, max_deg))
    phi = rng.uniform(0, 2 * np.pi)
    return np.array([np.sin(ang) * np.cos(phi), np.sin(ang) * np.sin(phi), -np.cos(ang)])


def _plane_facing(rng, center, max_deg, f, texture_seed, extent=None):
    n = _tilted_normal(rng, max_deg)
    a = np.array([1.0, 0.0, 0.0])
    e1 = a - n * (n @ a)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(n, e1)
    block = 8.0 * center[2] / f
    return Plane(center, e1, e2, BlockTexture(block, texture_seed), extent)


def tiny_pair(seed: int = 0) -> Sequence:
    cam = Camera(60.0, 60.0, 32.0, 24.0, 64, 48)
    rng = np.random.default_rng(seed)
    axis = rng.normal(size=3)
    axis /= np.linalg.norm(axis)
    tdir = rng.normal(size=3)
    tdir /= np.linalg.norm(tdir)
    T_ts = _pose(Rotation.from_rotvec(np.deg2rad(0.5) * axis).as_matrix(), 0.02 * tdir)
    poses = np.stack([np.eye(4), _inv(T_ts)])
    for _ in range(1000):
        back = _plane_facing(rng, np.array([0.0, 0.0, rng.uniform(2.8, 3.6)]), 30, cam.fx,
                             int(rng.integers(1 << 30)))
        p1 = _plane_facing(rng, np.array([rng.uniform(-0.6, -0.2), rng.uniform(-0.4, 0.1),
                                          rng.uniform(1.3, 2.0)]), 30, cam.fx,
                           int(rng.integers(1 << 30)), (-0.45, 0.45, -0.35, 0.35))
        p2 = _plane_facing(rng, np.array([rng.uniform(0.2, 0.6), rng.uniform(-0.1, 0.4),
                                          rng.uniform(1.6, 2.4)]), 30, cam.fx,
                           int(rng.integers(1 << 30)), (-0.5, 0.5, -0.4, 0.4))
        scene = Scene([back, p1, p2])
        ok = True
        for T in poses:
            r = render(scene, T, cam)
            z = r["depth"]
            if not (r["hit"].all() and z.min() >= 1.0 and z.max() <= 4.0):
                ok = False
                break
        if ok:
            return Sequence("tiny", cam, scene, poses, seed, noise_sigma=1.0 / 255.0,
                            sweeps=50, kf_interval=1, sigma_P=0.1)
    raise RuntimeError("tiny_pair: rejection sampling failed")


# --------------------------------------------------------------------------
# trajectories
# --------------------------------------------------------------------------
def _sinusoid_path(rng, n, n_terms=3, period_range=(40.0, 160.0)):
    """(n, 3) smooth bounded path: sum of n_terms sinusoids per axis."""
    k = np.arange(n, dtype=np.float64)[:, None]
    out = np.zeros((n, 3))
    for _ in range(n_terms):
        per = rng.uniform(*period_range, size=3)
        ph = rng.uniform(0, 2 * np.pi, size=3)
        amp = rng.uniform(0.5, 1.0, size=3)
        out += amp * np.sin(2 * np.pi * k / per + ph)
    return out


def _smooth_trajectory(rng, n, step_t, step_r_deg):
    """Camera-to-world poses whose mean per-frame translation is step_t (m) and
    mean per-frame rotation is step_r_deg (deg)."""
    pos = _sinusoid_path(rng, n)
    rot = _sinusoid_path(rng, n)
    dp = np.linalg.norm(np.diff(pos, axis=0), axis=1).mean() if n > 1 else 1.0
    dr = np.linalg.norm(np.diff(rot, axis=0), axis=1).mean() if n > 1 else 1.0
    pos = (pos - pos[0]) * (step_t / dp)
    rot = (rot - rot[0]) * (np.deg2rad(step_r_deg) / dr)
    return np.stack([_pose(Rotation.from_rotvec(r).as_matrix(), p) for p, r in zip(pos, rot)])


def _random_speed_trajectory(rng, n, max_t, max_r_deg):
    """Per-frame motion of magnitude U[0, max_t] and U[0, max_r] along smoothly
    varying directions (unit tangents of bounded sinusoid paths), applied in
    the camera frame."""
    dirs_t = np.diff(_sinusoid_path(rng, n + 1), axis=0)
    dirs_r = np.diff(_sinusoid_path(rng, n + 1), axis=0)
    dirs_t /= np.linalg.norm(dirs_t, axis=1, keepdims=True)
    dirs_r /= np.linalg.norm(dirs_r, axis=1, keepdims=True)
    mt = rng.uniform(0.0, max_t, n)
    mr = rng.uniform(0.0, np.deg2rad(max_r_deg), n)
    T = np.eye(4)
    poses = [T]
    for k in range(1, n):
        D = _pose(Rotation.from_rotvec(mr[k] * dirs_r[k]).as_matrix(), mt[k] * dirs_t[k])
        T = T @ D
        poses.append(T)
    return np.stack(poses)


# --------------------------------------------------------------------------
# config: SCAMP-like room
# --------------------------------------------------------------------------
def _box_faces(lo, hi, tex_seed, wl=(0.05, 0.4)):
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    faces = []
    ex, ey, ez = np.eye(3)
    c = 0.5 * (lo + hi)
    h = 0.5 * (hi - lo)
    spec = [  # (center, e1, e2, extent half sizes)
        (c - ez * h[2], ex, ey, (h[0], h[1])), (c + ez * h[2], ex, ey, (h[0], h[1])),
        (c - ex * h[0], ez, ey, (h[2], h[1])), (c + ex * h[0], ez, ey, (h[2], h[1])),
        (c - ey * h[1], ex, ez, (h[0], h[2])), (c + ey * h[1], ex, ez, (h[0], h[2])),
    ]
    for i, (p0, e1, e2, (a, b)) in enumerate(spec):
        faces.append(Plane(p0, e1, e2, SmoothTexture(tex_seed + i, *wl), (-a, a, -b, b)))
    return faces


def scamp_room(seed: int = 1, n_frames: int = 100) -> Sequence:
    cam = Camera(128.0, 128.0, 127.5, 127.5, 256, 256)
    rng = np.random.default_rng(seed)
    room = _box_faces((-2.5, -1.6, -0.6), (2.5, 1.6, 5.0), 1000 * seed + 10)
    box = _box_faces((0.25, 0.7, 0.9), (0.95, 1.6, 1.5), 1000 * seed + 30, (0.03, 0.2))
    scene = Scene(room + box)
    poses = _smooth_trajectory(rng, n_frames, 0.01, 0.3)
    return Sequence("scamp_room", cam, scene, poses, seed, noise_sigma=2.0 / 255.0,
                    sweeps=20, kf_interval=10)


# --------------------------------------------------------------------------
# config: realistic 640x480 (and the batched / adjoint families)
# --------------------------------------------------------------------------
def _realistic_scene(seed: int) -> Scene:
    rng = np.random.default_rng(seed)
    ts = lambda i, wl=(0.04, 0.3): SmoothTexture(1000 * seed + i, *wl)
    ground = Plane((0, 1.0, 0), (1, 0, 0), (0, 0, 1), ts(1))
    back = Plane((0, 0, 7.8), (1, 0, 0), (0, 1, 0), ts(2, (0.1, 0.8)))
    curtain = HeightField((1.3, -0.5, 3.0), (0, 0, 1), (0, 1, 0), amp=rng.uniform(0.1, 0.2),
                          k1=2 * np.pi / rng.uniform(0.5, 1.0), k2=2 * np.pi / rng.uniform(0.5, 1.0),
                          ph1=rng.uniform(0, 6.3), ph2=rng.uniform(0, 6.3), texture=ts(3),
                          extent=(-2.7, 4.7, -2.5, 1.5))
    patch = HeightField((-0.35, 0.35, 1.1), (1, 0, -0.25), (0, 1, 0), amp=rng.uniform(0.04, 0.08),
                        k1=2 * np.pi / rng.uniform(0.5, 0.8), k2=2 * np.pi / rng.uniform(0.5, 0.8),
                        ph1=rng.uniform(0, 6.3), ph2=rng.uniform(0, 6.3), texture=ts(4, (0.02, 0.15)),
                        extent=(-0.3, 0.3, -0.25, 0.25))
    return Scene([ground, back, curtain, patch])


def realistic(seed: int = 2, n_frames: int = 300, width: int = 640, height: int = 480,
              f: float | None = None, sweeps: int = 20) -> Sequence:
    if f is None:
        f = 525.0 / 640.0 * width
    cam = Camera(f, f, (width - 1) / 2.0, (height - 1) / 2.0, width, height)
    rng = np.random.default_rng([seed, 7])
    poses = _random_speed_trajectory(rng, n_frames, 0.03, 1.0)
    return Sequence("realistic", cam, _realistic_scene(seed), poses, seed,
                    noise_sigma=2.0 / 255.0, quantize=True, dropout=0.01,
                    sweeps=sweeps, kf_interval=10)


BATCHED_RESOLUTIONS = ((128, 96), (256, 256), (320, 240), (640, 480))


def batched_family(n_seq: int = 64, n_frames: int = 50, first_seed: int = 1000,
                   sweeps: int = 20) -> list:
    out = []
    for s in range(first_seed, first_seed + n_seq):
        rng = np.random.default_rng([s, 3])
        w, h = BATCHED_RESOLUTIONS[int(rng.integers(len(BATCHED_RESOLUTIONS)))]
        out.append(realistic(s, n_frames, w, h, f=0.8203 * w, sweeps=sweeps))
    return out


def adjoint_family(n_seq: int = 8, n_frames: int = 10, first_seed: int = 2000) -> list:
    return [realistic(s, n_frames, 320, 240, f=262.5, sweeps=30) for s in
            range(first_seed, first_seed + n_seq)]


# --------------------------------------------------------------------------
# construction with an exactly bilinear target image (zero photometric residual)
# --------------------------------------------------------------------------
def affine_pair(seq: Sequence, s: int = 0, t: int = 1, coef=(0.3, 0.004, -0.003, 2e-5)):
    """Source/target pair whose target image is a + b u + c v + d u v sampled at the
    pixel centres, so that bilinear interpolation of it is exact everywhere.

    The source image holds, at each source pixel, the value of that function at the
    pixel's true correspondence in the target view (computed here by ray casting and
    rigid transformation). Returns dict with I_s, I_t, depth (source), normal
    (source), T_ts (4x4), x_t, y_t, Z_t (the true correspondences) and inside
    (correspondence inside [0, W-1] x [0, H-1] with positive depth).
    """
    cam = seq.cam
    a, b, c, d = coef
    src = seq.clean(s)
    T_ts = seq.relative_pose(s, t)
    X_s = cam.ray_grid() * src["depth"][..., None]
    X_t = X_s @ T_ts[:3, :3].T + T_ts[:3, 3]
    Z = X_t[..., 2]
    x = cam.fx * X_t[..., 0] / Z + cam.cx
    y = cam.fy * X_t[..., 1] / Z + cam.cy
    uu, vv = np.meshgrid(np.arange(cam.width, dtype=float), np.arange(cam.height, dtype=float))
    I_t = a + b * uu + c * vv + d * uu * vv
    I_s = a + b * x + c * y + d * x * y
    inside = (Z > 0) & (x >= 0) & (x <= cam.width - 1) & (y >= 0) & (y <= cam.height - 1)
    return {"I_s": I_s, "I_t": I_t, "depth": src["depth"], "normal": src["normal"],
            "T_ts": T_ts, "x_t": x, "y_t": y, "Z_t": Z, "inside": inside}


# --------------------------------------------------------------------------
# PPA-like Poisson-Gaussian degradation (App. D.1)
# theta = (alpha, sigma_r, lambda_d, sigma_p, F, g, b, t_e)
# --------------------------------------------------------------------------
THETA_STRONG = (0.20, 25.0, 1.0, 0.01, 15000.0, 1.5, 10, 0.001)
THETA_MILD = (0.12, 8.0, 0.3, 0.003, 15000.0, 1.5, 10, 0.001)


def ppa_noise(x: np.ndarray, theta, rng: np.random.Generator, prnu: np.ndarray | None = None):
    """Degrade clean linear intensities x in [0, 1] with the paper's sensor model:
    PRNU gain, Poisson shot and dark-current electrons, Gaussian read noise, then
    gain and ADC quantisation to b bits, normalised back to [0, 1].
    ``prnu`` (per-pixel eta) is drawn from rng when not given."""
    alpha, sig_r, lam_d, sig_p, F, g, bits, t_e = theta
    if prnu is None:
        prnu = rng.normal(0.0, sig_p, x.shape)
    xp = np.clip(x * (1.0 + prnu), 0.0, 1.0)
    s = alpha * F * xp
    n_e = rng.poisson(s) + rng.poisson(lam_d * t_e, x.shape) + rng.normal(0.0, sig_r, x.shape)
    full = 2 ** bits - 1
    return (np.clip(np.round(n_e / g), 0, full) / full).astype(np.float32)
