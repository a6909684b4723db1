"""Analytic scenes and a nearest-hit ray caster (FP64, numpy).

Camera frame: x right, y down, z forward. A camera pose is a 4x4
camera-to-world matrix ``T_wc``. The ray through pixel (u, v) (pixel centres
at integer coordinates) has camera-frame direction ((u-cx)/fx, (v-cy)/fy, 1),
so the ray parameter at a hit equals the hit's camera-frame depth z.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Camera:
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int

    def ray_grid(self) -> np.ndarray:
        """(H, W, 3) camera-frame ray directions with unit z component."""
        u = np.arange(self.width, dtype=np.float64)
        v = np.arange(self.height, dtype=np.float64)
        uu, vv = np.meshgrid(u, v)
        return np.stack([(uu - self.cx) / self.fx, (vv - self.cy) / self.fy,
                         np.ones_like(uu)], axis=-1)

    def as_tuple(self):
        return (self.fx, self.fy, self.cx, self.cy, self.width, self.height)


# --------------------------------------------------------------------------
# textures: functions of the surface coordinates (s, t) in metres
# --------------------------------------------------------------------------
@dataclass
class BlockTexture:
    """Piecewise-constant square blocks with values uniform in [0, 1]."""
    block: float
    seed: int
    _table: np.ndarray = field(init=False, repr=False)

    def __post_init__(self):
        self._table = np.random.default_rng(self.seed).random((97, 89))

    def __call__(self, s, t):
        i = np.floor(s / self.block).astype(np.int64) % self._table.shape[0]
        j = np.floor(t / self.block).astype(np.int64) % self._table.shape[1]
        return self._table[i, j]


@dataclass
class SmoothTexture:
    """Sum of seeded plane waves, clipped to [0, 1]; gradients almost everywhere."""
    seed: int
    wavelength_min: float
    wavelength_max: float
    n_waves: int = 8
    _k: np.ndarray = field(init=False, repr=False)
    _phi: np.ndarray = field(init=False, repr=False)
    _amp: np.ndarray = field(init=False, repr=False)

    def __post_init__(self):
        rng = np.random.default_rng(self.seed)
        lam = np.exp(rng.uniform(np.log(self.wavelength_min),
                                 np.log(self.wavelength_max), self.n_waves))
        ang = rng.uniform(0, np.pi, self.n_waves)
        self._k = (2 * np.pi / lam)[:, None] * np.stack([np.cos(ang), np.sin(ang)], 1)
        self._phi = rng.uniform(0, 2 * np.pi, self.n_waves)
        a = rng.uniform(0.5, 1.0, self.n_waves)
        self._amp = 0.42 * a / a.sum() * 2.0

    def __call__(self, s, t):
        val = np.full(np.shape(s), 0.5)
        for k, ph, a in zip(self._k, self._phi, self._amp):
            val = val + 0.5 * a * np.sin(k[0] * s + k[1] * t + ph)
        return np.clip(val, 0.0, 1.0)


# --------------------------------------------------------------------------
# primitives (world frame)
# --------------------------------------------------------------------------
def _unit(x):
    x = np.asarray(x, dtype=np.float64)
    return x / np.linalg.norm(x)


@dataclass
class Plane:
    """Plane through ``p0`` spanned by unit vectors e1, e2; optional finite extent
    (smin, smax, tmin, tmax) in the (s, t) surface coordinates."""
    p0: np.ndarray
    e1: np.ndarray
    e2: np.ndarray
    texture: object
    extent: tuple | None = None

    def __post_init__(self):
        self.p0 = np.asarray(self.p0, dtype=np.float64)
        self.e1 = _unit(self.e1)
        e2 = np.asarray(self.e2, dtype=np.float64)
        self.e2 = _unit(e2 - self.e1 * (self.e1 @ e2))
        self.n = np.cross(self.e1, self.e2)

    def intersect(self, o, d):
        """Ray o + lam*d, d (..., 3). Returns lam (inf where no hit), world normal, (s, t)."""
        denom = d @ self.n
        with np.errstate(divide="ignore", invalid="ignore"):
            lam = ((self.p0 - o) @ self.n) / denom
        X = o + lam[..., None] * d
        rel = X - self.p0
        s, t = rel @ self.e1, rel @ self.e2
        ok = np.isfinite(lam) & (lam > 1e-9)
        if self.extent is not None:
            smin, smax, tmin, tmax = self.extent
            ok &= (s >= smin) & (s <= smax) & (t >= tmin) & (t <= tmax)
        lam = np.where(ok, lam, np.inf)
        nrm = np.broadcast_to(self.n, d.shape)
        return lam, nrm, s, t


@dataclass
class HeightField:
    """Surface X(s, t) = p0 + s e1 + t e2 + h(s, t) n0 with
    h = amp * sin(k1 s + ph1) * sin(k2 t + ph2), over a finite (s, t) extent."""
    p0: np.ndarray
    e1: np.ndarray
    e2: np.ndarray
    amp: float
    k1: float
    k2: float
    ph1: float
    ph2: float
    texture: object
    extent: tuple
    n_march: int = 20
    n_bisect: int = 36

    def __post_init__(self):
        self.p0 = np.asarray(self.p0, dtype=np.float64)
        self.e1 = _unit(self.e1)
        e2 = np.asarray(self.e2, dtype=np.float64)
        self.e2 = _unit(e2 - self.e1 * (self.e1 @ e2))
        self.n0 = np.cross(self.e1, self.e2)

    def _h(self, s, t):
        return self.amp * np.sin(self.k1 * s + self.ph1) * np.sin(self.k2 * t + self.ph2)

    def _g(self, o, d, lam):
        X = o + lam[..., None] * d
        rel = X - self.p0
        return rel @ self.n0 - self._h(rel @ self.e1, rel @ self.e2)

    def intersect(self, o, d):
        shape = d.shape[:-1]
        d = d.reshape(-1, 3)
        n = d.shape[0]
        lam_out = np.full(n, np.inf)
        nrm_out = np.zeros((n, 3))
        s_out = np.zeros(n)
        t_out = np.zeros(n)
        dn = d @ self.n0
        with np.errstate(divide="ignore", invalid="ignore"):
            l_a = ((self.p0 - o) @ self.n0 + self.amp) / dn
            l_b = ((self.p0 - o) @ self.n0 - self.amp) / dn
        lo = np.minimum(l_a, l_b)
        hi = np.maximum(l_a, l_b)
        good = np.isfinite(lo) & np.isfinite(hi) & (hi > 1e-9)
        lo = np.where(good, np.maximum(lo, 1e-9), 1.0)
        hi = np.where(good, hi, 2.0)
        # keep rays whose bracket segment can reach the finite (s, t) extent
        smin, smax, tmin, tmax = self.extent
        rel_lo = o + lo[:, None] * d - self.p0
        rel_hi = o + hi[:, None] * d - self.p0
        s_lo, s_hi = rel_lo @ self.e1, rel_hi @ self.e1
        t_lo, t_hi = rel_lo @ self.e2, rel_hi @ self.e2
        good &= (np.maximum(s_lo, s_hi) >= smin) & (np.minimum(s_lo, s_hi) <= smax)
        good &= (np.maximum(t_lo, t_hi) >= tmin) & (np.minimum(t_lo, t_hi) <= tmax)
        idx = np.nonzero(good)[0]
        if idx.size:
            dd, lo, hi = d[idx], lo[idx], hi[idx]
            # march from the near bracket end to the first sign change, then bisect
            steps = np.linspace(0.0, 1.0, self.n_march + 1)
            g_prev = self._g(o, dd, lo)
            a = lo.copy()
            b = np.full_like(lo, np.nan)
            found = np.zeros(lo.shape, dtype=bool)
            for k in range(1, self.n_march + 1):
                lk = lo + steps[k] * (hi - lo)
                gk = self._g(o, dd, lk)
                cross = (~found) & (np.sign(gk) != np.sign(g_prev))
                a = np.where(cross, lo + steps[k - 1] * (hi - lo), a)
                b = np.where(cross, lk, b)
                found |= cross
                g_prev = gk
            a = np.where(found, a, 1.0)
            b = np.where(found, b, 2.0)
            ga = self._g(o, dd, a)
            for _ in range(self.n_bisect):
                m = 0.5 * (a + b)
                gm = self._g(o, dd, m)
                left = np.sign(gm) == np.sign(ga)
                a = np.where(left, m, a)
                ga = np.where(left, gm, ga)
                b = np.where(left, b, m)
            lam = 0.5 * (a + b)
            rel = o + lam[:, None] * dd - self.p0
            s, t = rel @ self.e1, rel @ self.e2
            ok = found & (s >= smin) & (s <= smax) & (t >= tmin) & (t <= tmax)
            hs = self.amp * self.k1 * np.cos(self.k1 * s + self.ph1) * np.sin(self.k2 * t + self.ph2)
            ht = self.amp * self.k2 * np.sin(self.k1 * s + self.ph1) * np.cos(self.k2 * t + self.ph2)
            dXs = self.e1 + hs[:, None] * self.n0
            dXt = self.e2 + ht[:, None] * self.n0
            nrm = np.cross(dXs, dXt)
            nrm = nrm / np.linalg.norm(nrm, axis=-1, keepdims=True)
            lam_out[idx] = np.where(ok, lam, np.inf)
            nrm_out[idx] = nrm
            s_out[idx] = s
            t_out[idx] = t
        return (lam_out.reshape(shape), nrm_out.reshape(shape + (3,)),
                s_out.reshape(shape), t_out.reshape(shape))


@dataclass
class Scene:
    primitives: list
    background: float = 0.5


def render(scene: Scene, T_wc: np.ndarray, cam: Camera):
    """Nearest-hit ray cast from camera pose ``T_wc`` (camera-to-world).

    Returns a dict with 'image' (H, W) clean intensity, 'depth' (H, W) camera z
    (inf where nothing is hit), 'normal' (H, W, 3) camera-frame unit normals facing
    the camera, and 'hit' (H, W) bool.
    """
    R = T_wc[:3, :3]
    o = T_wc[:3, 3]
    rc = cam.ray_grid()
    d = rc @ R.T
    best = np.full(rc.shape[:2], np.inf)
    img = np.full(rc.shape[:2], scene.background)
    nrm_w = np.zeros(rc.shape)
    nrm_w[..., 2] = -1.0
    for prim in scene.primitives:
        lam, n, s, t = prim.intersect(o, d)
        closer = lam < best
        if not np.any(closer):
            continue
        best = np.where(closer, lam, best)
        img = np.where(closer, prim.texture(s, t), img)
        nrm_w = np.where(closer[..., None], n, nrm_w)
    hit = np.isfinite(best)
    nrm_c = nrm_w @ R  # R^T n for row vectors
    X = rc * np.where(hit, best, 1.0)[..., None]
    flip = np.sum(nrm_c * X, axis=-1) > 0
    nrm_c = np.where(flip[..., None], -nrm_c, nrm_c)
    nrm_c = np.where(hit[..., None], nrm_c, np.array([0.0, 0.0, -1.0]))
    return {"image": img, "depth": best, "normal": nrm_c, "hit": hit}
