"""Factor linearisations of the PixVOD factor graph, FP64 (numpy).

Each pixel i holds the stacked variable mu_i = [xi_i (se(3), 6); d_i (log-depth)]
(Sec. 3.3). Linearisation follows Sec. 3.4 (Eqs. 7-9): a variable is
mu_bar (+) tau with tau in the 7-D tangent space, a residual is
r(mu_bar (+) tau) ~ r_bar + J tau, and the quadratic energy
(1/2)|r_bar + J tau|^2_Lambda has information form
Lambda_f = J^T Lambda J, eta_f = -J^T Lambda r_bar.

Readings of points the paper leaves open (each also listed in the design notes):
* pixel centres are at integer coordinates; a warped point is valid iff Z > 1e-6
  and -1e-3 <= x <= W-1+1e-3, -1e-3 <= y <= H-1+1e-3 (the margin keeps pixels that
  the identity pose maps exactly onto the border valid whatever the rounding; the
  sample point is clamped into the image); an invalid pixel contributes no
  photometric factor (the overlap domain Omega(mu) of Eq. 1), and neither does a
  pixel whose residual or interpolated gradient is not finite (NaN input);
* image gradients are central differences with replicated borders, bilinearly
  interpolated at the warped point like the intensity;
* the Huber threshold t acts on the Mahalanobis residual |r|/sigma_D and the robust
  factor is applied by covariance weighting, w = (2 t M - t^2)/M^2 for M > t;
* prior and identity factors use the identity Jacobian of (-) (the right-Jacobian
  inverse J_r^-1(r_bar) is dropped, r_bar being tiny for these factors); residuals
  themselves are exact;
* the normal-integration measurement uses n_tilde_z = f (n . r(u, v)) with
  r(u, v) = ((u-cx)/fx, (v-cy)/fy, 1); an edge takes the mean of its two pixels'
  n_x/n_tilde_z; |n . r| < 1e-3 gives a zero slope.

Test infrastructure: this package is the CPU oracle. Only tests/, the smoke check
and the bench's CPU-baseline leg may import it.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import lie

Z_MIN = 1e-6
NR_MIN = 1e-3


@dataclass(frozen=True)
class Intrinsics:
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int


# --------------------------------------------------------------------------
# warp (Eq. 2)
# --------------------------------------------------------------------------
def backproject(u, v, d, K: Intrinsics):
    """pi^-1(p, exp(d)) = exp(d) K^-1 [u, v, 1]^T, shape (..., 3)."""
    z = np.exp(d)
    return np.stack([z * (u - K.cx) / K.fx, z * (v - K.cy) / K.fy, z], -1)


def warp(xi, d, u, v, K: Intrinsics):
    """W(p; mu) of Eq. 2: back-project with depth exp(d), apply the rigid motion
    Exp(xi) by left multiplication (X_t = R X_s + t), project with K.
    Returns x, y, Z, X_s, X_t, R."""
    R, t = lie.se3_exp(xi)
    X_s = backproject(u, v, d, K)
    X_t = (R @ X_s[..., None])[..., 0] + t
    Z = X_t[..., 2]
    Zs = np.where(np.abs(Z) > Z_MIN, Z, 1.0)
    x = K.fx * X_t[..., 0] / Zs + K.cx
    y = K.fy * X_t[..., 1] / Zs + K.cy
    return x, y, Z, X_s, X_t, R


BORDER_MARGIN = 1e-3


def warp_valid(x, y, Z, K: Intrinsics):
    """Overlap domain: positive depth and inside the image, with a 1e-3 px margin
    (a pixel warped by the identity pose lands exactly on the border)."""
    m = BORDER_MARGIN
    return (Z > Z_MIN) & (x >= -m) & (x <= K.width - 1 + m) & (y >= -m) & (y <= K.height - 1 + m)


# --------------------------------------------------------------------------
# image sampling
# --------------------------------------------------------------------------
def image_gradient(I):
    """Central differences (I[u+1] - I[u-1])/2 with replicated borders."""
    I = np.asarray(I, dtype=np.float64)
    gx = 0.5 * (np.concatenate([I[:, 1:], I[:, -1:]], 1) - np.concatenate([I[:, :1], I[:, :-1]], 1))
    gy = 0.5 * (np.concatenate([I[1:], I[-1:]], 0) - np.concatenate([I[:1], I[:-1]], 0))
    return gx, gy


def bilinear(I, x, y):
    """Bilinear interpolation at (x, y), pixel centres at integers. Coordinates are
    clamped into the image, so callers mask out-of-image points themselves."""
    H, W = I.shape
    x = np.clip(np.where(np.isfinite(x), x, 0.0), 0.0, W - 1.0)
    y = np.clip(np.where(np.isfinite(y), y, 0.0), 0.0, H - 1.0)
    x0 = np.floor(x).astype(np.int64)
    y0 = np.floor(y).astype(np.int64)
    ax = x - x0
    ay = y - y0
    x1 = np.minimum(x0 + 1, W - 1)
    y1 = np.minimum(y0 + 1, H - 1)
    return ((1 - ay) * ((1 - ax) * I[y0, x0] + ax * I[y0, x1])
            + ay * ((1 - ax) * I[y1, x0] + ax * I[y1, x1]))


# --------------------------------------------------------------------------
# photometric factor (Eq. 3) with Huber covariance weighting (Sec. 4.1)
# --------------------------------------------------------------------------
def huber_weight(M, t):
    """Scale on the factor information so that (1/2) w M^2 equals the Huber cost
    at the Mahalanobis residual M (covariance weighting)."""
    M = np.abs(M)
    safe = np.where(M > t, M, 1.0)
    return np.where(M > t, (2.0 * t * safe - t * t) / (safe * safe), 1.0)


def photometric_residual(xi, d, u, v, I_s_p, I_t, K: Intrinsics):
    """r = I_s[p] - I_t(W(p; mu)); returns r, valid."""
    x, y, Z, _, _, _ = warp(xi, d, u, v, K)
    valid = warp_valid(x, y, Z, K)
    return I_s_p - bilinear(I_t, x, y), valid


def photometric_jacobian(xi, d, u, v, g_x, g_y, K: Intrinsics):
    """dr/dtau (..., 7) for the right perturbation mu_bar (+) tau.

    X_t(tau) = R Exp(theta_tau) X_s + R rho_tau + t (first order) with
    X_s = exp(d + tau_d) K^-1 p, so dX_t/dtau = [-R [X_s]x, R, R X_s];
    dp'/dX_t is the pinhole derivative; dr/dp' = -grad I_t(p')."""
    x, y, Z, X_s, X_t, R = warp(xi, d, u, v, K)
    Zs = np.where(np.abs(Z) > Z_MIN, Z, 1.0)
    gxp = bilinear(g_x, x, y)
    gyp = bilinear(g_y, x, y)
    zero = np.zeros_like(Zs)
    dpi = np.stack([np.stack([K.fx / Zs, zero, -K.fx * X_t[..., 0] / Zs ** 2], -1),
                    np.stack([zero, K.fy / Zs, -K.fy * X_t[..., 1] / Zs ** 2], -1)], -2)
    dr_dp = -np.stack([gxp, gyp], -1)[..., None, :]          # (..., 1, 2)
    dX = np.concatenate([-R @ lie.hat(X_s), R, (R @ X_s[..., None])], -1)  # (..., 3, 7)
    return (dr_dp @ dpi @ dX)[..., 0, :]


def photometric_factor(xi, d, u, v, I_s_p, I_t, g_x, g_y, K: Intrinsics, sigma_D, t_huber):
    """Information form of the linearised photometric factor (Eqs. 3, 8, 9).
    Returns Lambda (..., 7, 7), eta (..., 7), and diagnostics (r, J, w, valid)."""
    r, valid = photometric_residual(xi, d, u, v, I_s_p, I_t, K)
    J = photometric_jacobian(xi, d, u, v, g_x, g_y, K)
    valid = valid & np.isfinite(r) & np.all(np.isfinite(J), axis=-1)
    J = np.where(valid[..., None], J, 0.0)
    r = np.where(valid, r, 0.0)
    w = huber_weight(r / sigma_D, t_huber)
    lam = np.where(valid, w / sigma_D ** 2, 0.0)
    r = np.where(valid, r, 0.0)
    Lam = lam[..., None, None] * (J[..., :, None] * J[..., None, :])
    eta = -(lam * r)[..., None] * J
    return Lam, eta, {"r": r, "J": J, "w": w, "valid": valid}


# --------------------------------------------------------------------------
# prior factors (Eq. 4 and the log-depth prior of Sec. 3.3)
# --------------------------------------------------------------------------
def pose_prior_factor(xi, sigma_P):
    """(1/2)|mu [-] mu_hat|^2 with mu_hat the identity pose; J = I (see header)."""
    r = lie.se3_boxminus(xi, np.zeros_like(xi))
    shape = np.shape(xi)[:-1]
    Lam = np.zeros(shape + (7, 7))
    Lam[..., :6, :6] = np.eye(6) / sigma_P ** 2
    eta = np.zeros(shape + (7,))
    eta[..., :6] = -r / sigma_P ** 2
    return Lam, eta


def depth_prior_factor(d, d_prior, sigma_Z):
    """(1/2)((d - d_prior)/sigma_Z)^2 on the log-depth."""
    shape = np.shape(d)
    Lam = np.zeros(shape + (7, 7))
    Lam[..., 6, 6] = 1.0 / sigma_Z ** 2
    eta = np.zeros(shape + (7,))
    eta[..., 6] = -(d - d_prior) / sigma_Z ** 2
    return Lam, eta


# --------------------------------------------------------------------------
# pairwise factors over (x_a, x_b), 14-D joint tangent space
# --------------------------------------------------------------------------
def _pair_info(J, r, lam):
    """J (..., m, 14), r (..., m) -> Lambda (..., 14, 14), eta (..., 14)."""
    Jt = np.swapaxes(J, -1, -2)
    return lam * (Jt @ J), -lam * (Jt @ r[..., None])[..., 0]


def identity_factor(xi_a, xi_b, sigma_R):
    """Camera-motion identity factor, Eq. 5: r = xi_a [-] xi_b, J = [I 0 | -I 0]."""
    r = lie.se3_boxminus(xi_a, xi_b)
    shape = np.shape(r)[:-1]
    J = np.zeros(shape + (6, 14))
    J[..., :, 0:6] = np.eye(6)
    J[..., :, 7:13] = -np.eye(6)
    return _pair_info(J, r, 1.0 / sigma_R ** 2)


def normal_factor(d_a, d_b, m, sigma_N):
    """Normal-integration factor, Eq. 6, for a pixel pair where b is the right
    (or lower) neighbour of a: r = (d_b - d_a) + m."""
    r = (d_b - d_a + m)[..., None]
    shape = np.shape(d_a)
    J = np.zeros(shape + (1, 14))
    J[..., 0, 6] = -1.0
    J[..., 0, 13] = 1.0
    return _pair_info(J, r, 1.0 / sigma_N ** 2)


def normal_log_slopes(normals, K: Intrinsics, u0: int = 0, v0: int = 0):
    """Per-pixel n_x/n_tilde_z and n_y/n_tilde_z for camera-frame normals (H, W, 3).

    For a surface point X = z r(u, v) on the tangent plane n . X = c, ln z =
    ln c - ln(n . r), so d ln z / du = -(n_x/fx)/(n . r) = -n_x/n_tilde_z with
    n_tilde_z = fx (n . r) (and fy for the vertical direction)."""
    n = np.asarray(normals, dtype=np.float64)
    h, w = n.shape[:2]
    uu, vv = np.meshgrid(np.arange(w, dtype=np.float64) + u0, np.arange(h, dtype=np.float64) + v0)
    nr = n[..., 0] * (uu - K.cx) / K.fx + n[..., 1] * (vv - K.cy) / K.fy + n[..., 2]
    ok = np.abs(nr) >= NR_MIN
    nrs = np.where(ok, nr, 1.0)
    ax = np.where(ok, n[..., 0] / (K.fx * nrs), 0.0)
    ay = np.where(ok, n[..., 1] / (K.fy * nrs), 0.0)
    return ax, ay


def normal_edge_measurements(normals, K: Intrinsics, u0: int = 0, v0: int = 0):
    """Edge measurements of Eq. 6: m_x (H, W-1) between (u, v) and (u+1, v), m_y
    (H-1, W) between (u, v) and (u, v+1); each the mean of its two pixels' slopes."""
    ax, ay = normal_log_slopes(normals, K, u0, v0)
    return 0.5 * (ax[:, :-1] + ax[:, 1:]), 0.5 * (ay[:-1, :] + ay[1:, :])
