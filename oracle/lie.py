"""SO(3) / SE(3) exponential and logarithm in FP64 (numpy, vectorised over
leading dimensions).

Conventions (paper, App. C.2 equation for Exp): a tangent vector is
xi = [theta; rho] (rotation first). Exp(xi) = [Exp(theta), V(theta) rho; 0, 1]
with V(theta) = I + B(th) [theta]x + C(th) [theta]x^2. The right-plus of Sec. 3.4
(Sola's notation) is X (+) tau = X Exp(tau); X (-) Y = Log(Y^-1 X).

Test infrastructure: this package is the CPU oracle. Only tests/, the smoke check
and the bench's CPU-baseline leg may import it.
"""
from __future__ import annotations

import numpy as np


def hat(w: np.ndarray) -> np.ndarray:
    """(..., 3) -> (..., 3, 3) skew-symmetric matrix with hat(w) x = w x x."""
    w = np.asarray(w, dtype=np.float64)
    z = np.zeros(w.shape[:-1])
    return np.stack([
        np.stack([z, -w[..., 2], w[..., 1]], -1),
        np.stack([w[..., 2], z, -w[..., 0]], -1),
        np.stack([-w[..., 1], w[..., 0], z], -1),
    ], -2)


def _coef_A(th):
    """sin(th)/th."""
    th2 = th * th
    small = th < 1e-3
    safe = np.where(small, 1.0, th)
    return np.where(small, 1.0 - th2 / 6.0 + th2 * th2 / 120.0, np.sin(safe) / safe)


def _coef_B(th):
    """(1 - cos th)/th^2, written as (1/2) (sin(th/2)/(th/2))^2 (no cancellation)."""
    a = _coef_A(0.5 * th)
    return 0.5 * a * a


_C_SERIES = [(-1.0) ** k / float(np.prod(np.arange(1, 2 * k + 4))) for k in range(13)]


def _coef_C(th):
    """(th - sin th)/th^3 = sum_k (-1)^k th^(2k)/(2k+3)!; the series below 1 rad
    (13 terms), the closed form above."""
    th2 = th * th
    small = th < 1.0
    safe = np.where(small, 1.0, th)
    series = np.zeros_like(th2)
    for c in reversed(_C_SERIES):
        series = series * th2 + c
    return np.where(small, series, (safe - np.sin(safe)) / safe ** 3)


def so3_exp(theta: np.ndarray) -> np.ndarray:
    """Rodrigues' formula, (..., 3) -> (..., 3, 3)."""
    theta = np.asarray(theta, dtype=np.float64)
    th = np.linalg.norm(theta, axis=-1)[..., None, None]
    W = hat(theta)
    return np.eye(3) + _coef_A(th) * W + _coef_B(th) * (W @ W)


def so3_log(R: np.ndarray) -> np.ndarray:
    """(..., 3, 3) -> (..., 3); valid for rotation angles below pi.

    The angle is atan2(|w|, (tr R - 1)/2) with w = vee(R - R^T)/2 = sin(th) axis,
    which stays accurate for small angles."""
    R = np.asarray(R, dtype=np.float64)
    w = 0.5 * np.stack([R[..., 2, 1] - R[..., 1, 2], R[..., 0, 2] - R[..., 2, 0],
                        R[..., 1, 0] - R[..., 0, 1]], -1)
    s = np.linalg.norm(w, axis=-1)
    c = 0.5 * (np.trace(R, axis1=-2, axis2=-1) - 1.0)
    th = np.arctan2(s, c)
    return w / _coef_A(th)[..., None]


def se3_V(theta: np.ndarray) -> np.ndarray:
    """Left Jacobian of SO(3): V(theta) = I + B W + C W^2."""
    th = np.linalg.norm(theta, axis=-1)[..., None, None]
    W = hat(theta)
    return np.eye(3) + _coef_B(th) * W + _coef_C(th) * (W @ W)


def se3_exp(xi: np.ndarray):
    """xi (..., 6) = [theta; rho] -> (R (..., 3, 3), t (..., 3))."""
    xi = np.asarray(xi, dtype=np.float64)
    theta, rho = xi[..., :3], xi[..., 3:]
    R = so3_exp(theta)
    t = (se3_V(theta) @ rho[..., None])[..., 0]
    return R, t


def se3_log(R: np.ndarray, t: np.ndarray) -> np.ndarray:
    """Inverse of se3_exp; rho solves V(theta) rho = t."""
    theta = so3_log(R)
    rho = np.linalg.solve(se3_V(theta), np.asarray(t, dtype=np.float64)[..., None])[..., 0]
    return np.concatenate([theta, rho], -1)


def se3_compose(a, b):
    """(R_a, t_a) * (R_b, t_b)."""
    Ra, ta = a
    Rb, tb = b
    return Ra @ Rb, (Ra @ tb[..., None])[..., 0] + ta


def se3_inverse(a):
    R, t = a
    Rt = np.swapaxes(R, -1, -2)
    return Rt, -(Rt @ t[..., None])[..., 0]


def se3_boxplus(xi: np.ndarray, tau: np.ndarray) -> np.ndarray:
    """Log(Exp(xi) Exp(tau)) (right-plus, Sec. 3.4)."""
    return se3_log(*se3_compose(se3_exp(xi), se3_exp(tau)))


def se3_boxminus(xi_a: np.ndarray, xi_b: np.ndarray) -> np.ndarray:
    """Log(Exp(xi_b)^-1 Exp(xi_a)), the residual of Eq. 5 (mu_a [-] mu_b)."""
    return se3_log(*se3_compose(se3_inverse(se3_exp(xi_b)), se3_exp(xi_a)))


def se3_matrix(xi: np.ndarray) -> np.ndarray:
    R, t = se3_exp(xi)
    T = np.zeros(np.shape(xi)[:-1] + (4, 4))
    T[..., :3, :3] = R
    T[..., :3, 3] = t
    T[..., 3, 3] = 1.0
    return T
