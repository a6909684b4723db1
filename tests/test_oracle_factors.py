"""Pins for oracle.factors against geometry computed independently by the
ray caster in ``synth`` (zero residual at ground truth, exact warps, exact
log-depth differences), finite differences, and closed forms."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import synth
from oracle import factors as fac
from oracle import lie
from oracle.factors import Intrinsics

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _K(seq):
    return Intrinsics(*seq.cam.as_tuple())


def _gt_xi(T):
    # ground-truth twist from the 4x4 relative pose via scipy (not the oracle's Log)
    import scipy.linalg
    L = scipy.linalg.logm(T).real
    return np.array([L[2, 1], L[0, 2], L[1, 0], L[0, 3], L[1, 3], L[2, 3]])


@pytest.fixture(scope="module")
def affine(tiny_seq):
    return synth.affine_pair(tiny_seq)


def test_warp_matches_ray_caster(tiny_seq, affine):
    K = _K(tiny_seq)
    xi = _gt_xi(affine["T_ts"])
    uu, vv = tiny_seq.cam.ray_grid()[..., 0] * K.fx + K.cx, tiny_seq.cam.ray_grid()[..., 1] * K.fy + K.cy
    x, y, Z, *_ = fac.warp(xi, np.log(affine["depth"]), uu, vv, K)
    np.testing.assert_allclose(x, affine["x_t"], atol=1e-10)
    np.testing.assert_allclose(y, affine["y_t"], atol=1e-10)
    np.testing.assert_allclose(Z, affine["Z_t"], atol=1e-12)
    valid = fac.warp_valid(x, y, Z, K)
    far = (np.minimum(np.abs(affine["x_t"]), np.abs(affine["x_t"] - (K.width - 1))) > 1e-6) & \
          (np.minimum(np.abs(affine["y_t"]), np.abs(affine["y_t"] - (K.height - 1))) > 1e-6)
    assert np.array_equal(valid[far], affine["inside"][far])


def test_zero_photometric_residual_at_ground_truth(tiny_seq, affine):
    K = _K(tiny_seq)
    xi = _gt_xi(affine["T_ts"])
    uu, vv = np.meshgrid(np.arange(K.width, dtype=float), np.arange(K.height, dtype=float))
    r, valid = fac.photometric_residual(xi, np.log(affine["depth"]), uu, vv, affine["I_s"],
                                        affine["I_t"], K)
    assert valid.sum() > 0.8 * valid.size
    assert np.abs(r[valid]).max() < 1e-12


def test_gradient_and_bilinear_exact_on_bilinear_image():
    a, b, c, d = 0.2, 0.01, -0.02, 3e-4
    H, W = 9, 13
    uu, vv = np.meshgrid(np.arange(W, dtype=float), np.arange(H, dtype=float))
    I = a + b * uu + c * vv + d * uu * vv
    gx, gy = fac.image_gradient(I)
    np.testing.assert_allclose(gx[:, 1:-1], (b + d * vv)[:, 1:-1], atol=1e-15)
    np.testing.assert_allclose(gy[1:-1], (c + d * uu)[1:-1], atol=1e-15)
    # replicated border: (I[1] - I[0]) / 2
    np.testing.assert_allclose(gx[:, 0], 0.5 * (b + d * vv[:, 0]), atol=1e-15)
    rng = np.random.default_rng(0)
    x = rng.uniform(0, W - 1, 200)
    y = rng.uniform(0, H - 1, 200)
    np.testing.assert_allclose(fac.bilinear(I, x, y), a + b * x + c * y + d * x * y, atol=1e-14)
    np.testing.assert_allclose(fac.bilinear(I, uu, vv), I, atol=0)
    np.testing.assert_allclose(fac.bilinear(I, np.array([W - 1.0]), np.array([H - 1.0])), I[-1, -1])


def test_photometric_jacobian_matches_finite_differences(tiny_seq, affine):
    K = _K(tiny_seq)
    gx, gy = fac.image_gradient(affine["I_t"])
    rng = np.random.default_rng(5)
    xi0 = _gt_xi(affine["T_ts"])
    checked = 0
    for _ in range(60):
        u, v = float(rng.integers(4, K.width - 4)), float(rng.integers(4, K.height - 4))
        xi = xi0 + rng.normal(size=6) * 2e-3
        d = np.log(affine["depth"][int(v), int(u)]) + rng.normal() * 0.05
        x, y, Z, *_ = fac.warp(xi, d, u, v, K)
        # the bilinear image is smooth inside a cell; keep away from its edges and the border
        if not (2 <= x <= K.width - 3 and 2 <= y <= K.height - 3):
            continue
        if min(x % 1, 1 - x % 1, y % 1, 1 - y % 1) < 1e-3:
            continue
        J = fac.photometric_jacobian(xi, d, u, v, gx, gy, K)

        def r(tau):
            return fac.photometric_residual(lie.se3_boxplus(xi, tau[:6]), d + tau[6], u, v, 0.0,
                                            affine["I_t"], K)[0]

        h = 1e-6
        Jfd = np.array([(r(h * e) - r(-h * e)) / (2 * h) for e in np.eye(7)])
        np.testing.assert_allclose(J, Jfd, rtol=1e-6, atol=1e-6 * np.abs(Jfd).max())
        checked += 1
    assert checked > 30


def test_photometric_factor_information_form():
    rng = np.random.default_rng(6)
    K = Intrinsics(50.0, 55.0, 20.0, 15.0, 40, 30)
    It = rng.random((30, 40))
    gx, gy = fac.image_gradient(It)
    xi = rng.normal(size=6) * 1e-3
    L, e, dg = fac.photometric_factor(xi, 0.3, 12.0, 9.0, 0.4, It, gx, gy, K, 5e-3, 400.0)
    J, r = dg["J"], dg["r"]
    np.testing.assert_allclose(L, np.outer(J, J) / 25e-6, rtol=1e-14)
    np.testing.assert_allclose(e, -J * r / 25e-6, rtol=1e-14)
    # an invalid warp contributes nothing
    behind = xi + np.array([0, 0, 0, 0, 0, -10.0])    # moves the point behind the camera
    L, e, dg = fac.photometric_factor(behind, 0.3, 12.0, 9.0, 0.4, It, gx, gy, K, 5e-3, 400.0)
    assert not dg["valid"] and np.all(L == 0) and np.all(e == 0)


def test_huber_weight_reproduces_huber_cost():
    t = 2.0
    M = np.array([0.0, 0.5, 1.9999, 2.0, 2.0001, 3.0, 10.0, 400.0])
    w = fac.huber_weight(M, t)
    huber = np.where(M <= t, 0.5 * M ** 2, t * M - 0.5 * t ** 2)
    np.testing.assert_allclose(0.5 * w * M ** 2, huber, rtol=1e-14, atol=1e-300)
    assert np.all(w <= 1.0) and np.all(w[M <= t] == 1.0)
    np.testing.assert_allclose(fac.huber_weight(-M, t), w)


def test_priors():
    rng = np.random.default_rng(7)
    xi = rng.normal(size=(5, 6)) * 0.1
    L, e = fac.pose_prior_factor(xi, 0.5)
    np.testing.assert_allclose(e[:, :6], -xi / 0.25, atol=1e-12)
    np.testing.assert_allclose(L[0], np.diag([4.0] * 6 + [0.0]))
    L, e = fac.depth_prior_factor(np.array([0.3]), 0.1, 2.0)
    assert L[0, 6, 6] == 0.25 and np.isclose(e[0, 6], -0.05) and np.all(e[0, :6] == 0)


def test_identity_factor_jacobian_at_zero_residual():
    rng = np.random.default_rng(8)
    xi = rng.normal(size=6) * 0.1
    L, e = fac.identity_factor(xi, xi, 0.5)
    assert np.abs(e).max() < 1e-12

    def r(tau):
        return lie.se3_boxminus(lie.se3_boxplus(xi, tau[:6]), lie.se3_boxplus(xi, tau[7:13]))

    h = 1e-6
    Jfd = np.array([(r(h * e_) - r(-h * e_)) / (2 * h) for e_ in np.eye(14)]).T
    # at zero residual the identity Jacobian [I 0 | -I 0] is exact; the factor's
    # information must equal J^T J / sigma^2 with that Jacobian
    np.testing.assert_allclose(L, Jfd.T @ Jfd / 0.25, atol=1e-8)
    # eta = -J^T Lambda r for a non-zero residual
    other = xi + rng.normal(size=6) * 1e-3
    L, e = fac.identity_factor(xi, other, 0.5)
    rr = lie.se3_boxminus(xi, other)
    np.testing.assert_allclose(e[:6], -rr / 0.25, atol=1e-12)
    np.testing.assert_allclose(e[7:13], rr / 0.25, atol=1e-12)


def test_normal_measurement_matches_exact_log_depth_difference():
    """On a plane the exact log-depth step between neighbours, ln(z_a/z_b) =
    ln(1 + a), comes from the ray caster's depths; the normal factor's residual
    at the true log-depths must vanish to third order in a."""
    rng = np.random.default_rng(9)
    cam = synth.Camera(70.0, 64.0, 30.5, 20.5, 62, 42)
    K = Intrinsics(*cam.as_tuple())
    worst = 0.0
    for k in range(6):
        n = np.array([rng.uniform(-0.6, 0.6), rng.uniform(-0.6, 0.6), -1.0])
        e1 = np.cross(n, [0, 1.0, 0])
        e2 = np.cross(n, e1)
        scene = synth.Scene([synth.Plane((0, 0, rng.uniform(1.5, 3)), e1, e2,
                                         synth.SmoothTexture(k, 0.1, 0.3))])
        out = synth.render(scene, np.eye(4), cam)
        assert out["hit"].all()
        z, nrm = out["depth"], out["normal"]
        m_x, m_y = fac.normal_edge_measurements(nrm, K)
        d = np.log(z)
        for (da, db, m, za, zb) in ((d[:, :-1], d[:, 1:], m_x, z[:, :-1], z[:, 1:]),
                                    (d[:-1], d[1:], m_y, z[:-1], z[1:])):
            a = za / zb - 1.0
            L, e = fac.normal_factor(da, db, m, 1.0)
            res = -e[..., 13]          # eta_b = -J_b r with J_b = +1, sigma 1
            assert np.all(np.abs(res) <= 0.2 * np.abs(a) ** 3 + 1e-12)
            worst = max(worst, np.abs(a).max())
    assert worst > 5e-3    # the planes are tilted enough for the bound to matter
