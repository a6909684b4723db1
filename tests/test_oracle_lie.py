"""Pins for oracle.lie: library routines (scipy Rotation, expm, logm), identities,
and high-precision closed forms of the series coefficients (sympy)."""
import numpy as np
import pytest
import scipy.linalg
from scipy.spatial.transform import Rotation

from oracle import lie

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _thetas(rng):
    dirs = rng.normal(size=(40, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    mags = np.concatenate([[0.0, 1e-12, 1e-8, 1e-5, 9.99e-4, 1.001e-3, 0.0999, 0.1001],
                           rng.uniform(0, 2.5, 32)])
    return dirs * mags[:, None]


def test_so3_exp_matches_scipy():
    th = _thetas(np.random.default_rng(0))
    R = lie.so3_exp(th)
    np.testing.assert_allclose(R, Rotation.from_rotvec(th).as_matrix(), atol=1e-14)


def test_so3_log_matches_scipy():
    th = _thetas(np.random.default_rng(1))
    R = Rotation.from_rotvec(th).as_matrix()
    np.testing.assert_allclose(lie.so3_log(R), Rotation.from_matrix(R).as_rotvec(), atol=1e-13)


def _twist(xi):
    T = np.zeros((4, 4))
    T[:3, :3] = lie.hat(xi[:3])
    T[:3, 3] = xi[3:]
    return T


def test_se3_exp_matches_matrix_exponential():
    rng = np.random.default_rng(2)
    th = _thetas(rng)
    rho = rng.normal(size=th.shape) * 0.5
    for t, r in zip(th, rho):
        xi = np.concatenate([t, r])
        np.testing.assert_allclose(lie.se3_matrix(xi), scipy.linalg.expm(_twist(xi)), atol=1e-13)


def test_se3_log_matches_matrix_logarithm_and_round_trips():
    rng = np.random.default_rng(3)
    th = _thetas(rng)
    rho = rng.normal(size=th.shape)
    xi = np.concatenate([th, rho], 1)
    R, t = lie.se3_exp(xi)
    back = lie.se3_log(R, t)
    np.testing.assert_allclose(back, xi, atol=1e-12)
    for x in xi[8:16]:
        L = scipy.linalg.logm(lie.se3_matrix(x)).real
        np.testing.assert_allclose(lie.se3_log(*lie.se3_exp(x)), np.concatenate(
            [[L[2, 1], L[0, 2], L[1, 0]], L[:3, 3]]), atol=1e-10)


def test_series_coefficients_against_high_precision():
    sympy = pytest.importorskip("sympy")
    x = sympy.Symbol("x")
    exprs = {
        "A": sympy.sin(x) / x,
        "B": (1 - sympy.cos(x)) / x ** 2,
        "C": (x - sympy.sin(x)) / x ** 3,
    }
    fns = {"A": lie._coef_A, "B": lie._coef_B, "C": lie._coef_C}
    for th in [1e-7, 1e-4, 9.99e-4, 1.001e-3, 0.0999, 0.1001, 0.5, 0.999, 1.001, 2.0]:
        for k, e in exprs.items():
            exact = float(e.subs(x, sympy.Rational(repr(th))).evalf(40))
            got = float(fns[k](np.array(th)))
            assert abs(got - exact) <= 4e-15 * abs(exact), (k, th, got, exact)


def test_boxminus_antisymmetric_and_boxplus_inverse():
    rng = np.random.default_rng(4)
    a = rng.normal(size=(20, 6)) * 0.3
    b = rng.normal(size=(20, 6)) * 0.3
    np.testing.assert_allclose(lie.se3_boxminus(a, b), -lie.se3_boxminus(b, a), atol=1e-12)
    tau = lie.se3_boxminus(a, b)
    np.testing.assert_allclose(lie.se3_boxplus(b, tau), a, atol=1e-12)
