"""Pins for oracle.gbp and oracle.tracker: exactness of Gaussian BP means at a
fixed point against a dense Gauss-Newton solve, tree exactness of marginals,
brute-force marginalisation, SPD invariants, a linear least-squares special
case, crop-window equivalence, and keyframe pose composition."""
import numpy as np
import pytest
import scipy.linalg
import scipy.sparse
import scipy.sparse.linalg

import synth
from oracle import factors as fac
from oracle import gbp, lie
from oracle.factors import Intrinsics
from oracle.gbp import Params

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

# Weaker couplings than the paper's leaf values: exactness of the GBP fixed point does
# not depend on the strengths, and with these the 8x8 loopy grid converges in ~1500
# damped sweeps (with the paper's sigma_R it has not converged after 20000).
MILD = Params(sigma_D=0.05, sigma_P=1.0, sigma_R=0.3, sigma_N=0.2, sigma_Z=1.0,
              t_huber=400.0, damping=0.5)


def _crop_window(seq, v0, u0, h, w, d_prior=0.0):
    K = Intrinsics(*seq.cam.as_tuple())
    full = gbp.make_window(K, seq.frame(0), seq.normals(0), seq.frame(1), d_prior)
    m_x, m_y = fac.normal_edge_measurements(seq.normals(0), K)
    return gbp.Window(K, full.I_s[v0:v0 + h, u0:u0 + w], m_x[v0:v0 + h, u0:u0 + w - 1],
                      m_y[v0:v0 + h - 1, u0:u0 + w], full.I_t, full.g_x, full.g_y, u0, v0, d_prior)


def _perturbed_mu(rng, h, w, d0):
    mu = np.zeros((h, w, 7))
    mu[..., :6] = 0.004 * rng.normal(size=(h, w, 6))
    mu[..., 6] = d0 + 0.05 * rng.normal(size=(h, w))
    return mu


def test_factor_to_variable_matches_covariance_marginal():
    rng = np.random.default_rng(0)
    for to in (0, 1):
        A = rng.normal(size=(3, 9, 14))
        Lf = np.swapaxes(A, -1, -2) @ A
        ef = rng.normal(size=(3, 14))
        B = rng.normal(size=(3, 9, 7))
        Lin = np.swapaxes(B, -1, -2) @ B + np.eye(7)
        ein = rng.normal(size=(3, 7))
        Lm, em = gbp.factor_to_variable(Lf, ef, Lin, ein, to)
        keep = slice(7, 14) if to == 1 else slice(0, 7)
        other = slice(0, 7) if to == 1 else slice(7, 14)
        for k in range(3):
            J = Lf[k].copy()
            e = ef[k].copy()
            J[other, other] += Lin[k]
            e[other] += ein[k]
            J[keep, keep] += np.eye(7)        # makes the joint invertible; removed below
            S = np.linalg.inv(J)
            mean = S @ e
            Lmarg = np.linalg.inv(S[keep, keep])
            np.testing.assert_allclose(Lm[k], Lmarg - np.eye(7), rtol=1e-9, atol=1e-9)
            np.testing.assert_allclose(em[k], Lmarg @ mean[keep], rtol=1e-9, atol=1e-9)


def test_fixed_point_equals_dense_gauss_newton(tiny_seq):
    """Gaussian BP means at convergence are exact (loopy or not): the 8x8 grid's
    belief means equal the solve of the dense linearised system (448 unknowns)."""
    win = _crop_window(tiny_seq, 20, 28, 8, 8)
    mu0 = _perturbed_mu(np.random.default_rng(1), 8, 8, 0.4)
    tau, bel_L, it = gbp.frozen_gbp(win, mu0, MILD, max_iter=5000, tol=1e-14)
    Lam, eta = gbp.dense_system(win, mu0, MILD)
    ref = np.linalg.solve(Lam, eta).reshape(8, 8, 7)
    assert it < 5000
    scale = np.abs(ref).max()
    np.testing.assert_allclose(tau, ref, atol=1e-8 * scale, rtol=0)


def test_damping_does_not_move_fixed_point(tiny_seq):
    win = _crop_window(tiny_seq, 10, 10, 6, 7)
    mu0 = _perturbed_mu(np.random.default_rng(2), 6, 7, 0.3)
    t0, _, _ = gbp.frozen_gbp(win, mu0, gbp.with_params(MILD, damping=0.3), tol=1e-14)
    t1, _, _ = gbp.frozen_gbp(win, mu0, gbp.with_params(MILD, damping=0.7), tol=1e-14)
    np.testing.assert_allclose(t0, t1, atol=1e-9 * np.abs(t0).max())


@pytest.mark.parametrize("off", ["sigma_N", "sigma_R"])
def test_chain_is_exact_in_means_and_marginal_covariances(tiny_seq, off):
    """A 1xN window with one pairwise factor type is a tree (with both types, the
    identity and normal factors of one pixel pair close a loop through the pixels'
    photometric coupling): undamped GBP gives exact marginals after N sweeps."""
    n = 9
    win = _crop_window(tiny_seq, 30, 20, 1, n)
    mu0 = _perturbed_mu(np.random.default_rng(3), 1, n, 0.2)
    p = gbp.with_params(Params(sigma_P=0.1), damping=0.0, **{off: 1e150})
    tau, bel_L, it = gbp.frozen_gbp(win, mu0, p, max_iter=n + 1, tol=0.0)
    Lam, eta = gbp.dense_system(win, mu0, p)
    ref = np.linalg.solve(Lam, eta).reshape(1, n, 7)
    np.testing.assert_allclose(tau, ref, atol=1e-9 * np.abs(ref).max())
    cov = np.linalg.inv(Lam)
    for c in range(n):
        blk = slice(7 * c, 7 * c + 7)
        np.testing.assert_allclose(np.linalg.inv(bel_L[0, c]), cov[blk, blk],
                                   rtol=1e-7, atol=1e-12 * np.abs(cov[blk, blk]).max())


def test_relinearised_sweeps_converge_to_gauss_newton_stationary_point(tiny_seq):
    """With relinearisation every sweep, at convergence one dense Gauss-Newton step
    from the GBP means (same linearisation) is zero. Uses the exactly-bilinear image
    pair (smooth photometric model); on the block texture the relinearised
    iteration settles into a limit cycle instead."""
    K = Intrinsics(*tiny_seq.cam.as_tuple())
    aff = synth.affine_pair(tiny_seq)
    m_x, m_y = fac.normal_edge_measurements(aff["normal"], K)
    g_x, g_y = fac.image_gradient(aff["I_t"])
    v0, u0, h, w = 16, 24, 5, 6
    win = gbp.Window(K, aff["I_s"][v0:v0 + h, u0:u0 + w], m_x[v0:v0 + h, u0:u0 + w - 1],
                     m_y[v0:v0 + h - 1, u0:u0 + w], aff["I_t"], g_x, g_y, u0, v0, 0.3)
    st = gbp.reset_state((h, w), 0.3, MILD)
    for _ in range(1000):
        st = gbp.sweep(win, st, MILD)
    assert st.diag["valid"].all()
    Lam, eta = gbp.dense_system(win, st.mu, MILD)
    step = np.linalg.solve(Lam, eta)
    assert np.abs(step).max() < 1e-9
    assert np.abs(st.diag["tau"]).max() < 1e-9


def test_beliefs_and_messages_stay_positive_definite(tiny_seq):
    K = Intrinsics(*tiny_seq.cam.as_tuple())
    p = Params(sigma_P=0.1)
    win = gbp.make_window(K, tiny_seq.frame(0), tiny_seq.normals(0), tiny_seq.frame(1))
    st = gbp.reset_state(win.shape, 0.0, p)
    floor = np.diag([1 / p.sigma_P ** 2] * 6 + [1 / p.sigma_Z ** 2])
    for _ in range(12):
        st = gbp.sweep(win, st, p)
        ev = np.linalg.eigvalsh(st.bel_L - floor)
        assert ev.min() > -1e-9 * np.abs(st.bel_L).max()
        em = np.linalg.eigvalsh(st.msg_L)
        assert em.min() > -1e-9 * np.abs(st.msg_L).max()
        np.testing.assert_allclose(st.bel_L, np.swapaxes(st.bel_L, -1, -2), rtol=0,
                                   atol=1e-12 * np.abs(st.bel_L).max())
        assert np.abs(st.bel_eta).max() < 1e-9 * (1 + np.abs(st.bel_L).max())


def test_no_photometric_term_gives_least_squares_normal_integration(tiny_seq):
    """sigma_D -> infinity: poses stay at the prior mean and the log-depths are the
    linear least-squares integration of the normal measurements plus the prior."""
    h, w = 7, 9
    win = _crop_window(tiny_seq, 12, 30, h, w, d_prior=0.25)
    p = gbp.with_params(MILD, sigma_D=1e150)
    mu0 = np.zeros((h, w, 7))
    mu0[..., 6] = 0.25
    tau, _, _ = gbp.frozen_gbp(win, mu0, p, tol=1e-15)
    # rows: sqrt(lam_N) (d_b - d_a + m) and sqrt(lam_Z) (d - d_prior)
    idx = np.arange(h * w).reshape(h, w)
    rows, cols, vals, rhs = [], [], [], []
    r = 0
    for (a, b, m) in ((idx[:, :-1], idx[:, 1:], win.m_x), (idx[:-1], idx[1:], win.m_y)):
        for ia, ib, mm in zip(a.ravel(), b.ravel(), m.ravel()):
            rows += [r, r]
            cols += [ia, ib]
            vals += [-1.0 / p.sigma_N, 1.0 / p.sigma_N]
            rhs.append(-mm / p.sigma_N)
            r += 1
    for i in range(h * w):
        rows.append(r)
        cols.append(i)
        vals.append(1.0 / p.sigma_Z)
        rhs.append(0.25 / p.sigma_Z)
        r += 1
    A = scipy.sparse.csr_matrix((vals, (rows, cols)), shape=(r, h * w))
    d = scipy.sparse.linalg.lsqr(A, np.array(rhs), atol=1e-15, btol=1e-15, iter_lim=100000)[0]
    np.testing.assert_allclose(0.25 + tau[..., 6], d.reshape(h, w), atol=1e-9)
    assert np.abs(tau[..., :6]).max() < 1e-12


def test_crop_window_sweep_matches_full_sweep_at_centre(tiny_seq):
    """A pixel's new state after one sweep depends only on its 4-neighbourhood, so
    a sweep over a 3x3 crop reproduces the full-image sweep at the crop centre."""
    K = Intrinsics(*tiny_seq.cam.as_tuple())
    p = Params(sigma_P=0.1)
    win = gbp.make_window(K, tiny_seq.frame(0), tiny_seq.normals(0), tiny_seq.frame(1))
    st = gbp.reset_state(win.shape, 0.0, p)
    for _ in range(3):
        st = gbp.sweep(win, st, p)
    nxt = gbp.sweep(win, st, p)
    for (v, u) in ((5, 7), (20, 33), (47, 63), (0, 10)):
        v0, u0 = max(v - 1, 0), max(u - 1, 0)
        v1, u1 = min(v + 2, K.height), min(u + 2, K.width)
        sub = gbp.Window(K, win.I_s[v0:v1, u0:u1], win.m_x[v0:v1, u0:u1 - 1], win.m_y[v0:v1 - 1, u0:u1],
                         win.I_t, win.g_x, win.g_y, u0, v0, win.d_prior)
        cs = gbp.State(st.mu[v0:v1, u0:u1], st.bel_L[v0:v1, u0:u1], st.bel_eta[v0:v1, u0:u1],
                       st.msg_L[v0:v1, u0:u1], st.msg_eta[v0:v1, u0:u1])
        out = gbp.sweep(sub, cs, p)
        np.testing.assert_allclose(out.mu[v - v0, u - u0], nxt.mu[v, u], rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(out.msg_L[v - v0, u - u0], nxt.msg_L[v, u], rtol=1e-10, atol=1e-6)


def test_tracker_composes_keyframe_poses():
    """T_cam<-world after several keyframe segments equals the product of the
    segments' Exp(xi_est), composed here with scipy's matrix exponential."""
    from oracle.tracker import Tracker
    seq = synth.realistic(5, 7, 32, 24, sweeps=2)
    K = Intrinsics(*seq.cam.as_tuple())
    tr = Tracker(K, Params(sigma_P=0.05), kf_interval=3)
    segs = []
    T = np.eye(4)
    for k in range(7):
        xi = tr.track(seq.frame(k), seq.normals(k), n_iters=2)
        if k > 0:
            twist = np.zeros((4, 4))
            twist[:3, :3] = lie.hat(xi[:3])
            twist[:3, 3] = xi[3:]
            E = scipy.linalg.expm(twist)
            np.testing.assert_allclose(tr.pose_global(), E @ T, atol=1e-12)
            if k % 3 == 0:
                T = E @ T
                segs.append(k)
    assert segs == [3, 6]
    assert np.isfinite(tr.depth()).all()
