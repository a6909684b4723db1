"""Synchronous Gaussian Belief Propagation over the pixel grid, FP64 (numpy).

Textbook form: every variable belief and every factor-to-variable message is a
full 7-D information pair (Lambda 7x7, eta 7). A factor-to-variable message is
the marginal, by Schur complement, of the factor's 14-D joint plus the incoming
variable-to-factor message (belief minus that factor's last message) of the
other variable (Sec. 3.4 and the GBP steps it cites).

Schedule of one synchronous sweep (Sec. 4.1, Sec. 3.4):
  1. relinearise every factor at the current means mu_bar (Eq. 7-9);
  2. compute every pairwise factor-to-variable message from the previous
     sweep's beliefs and messages (all at once, synchronously);
  3. damp: m <- (1 - beta) m_new + beta m_old (pairwise messages only);
  4. beliefs b = unary + sum of incoming messages; tau = Lambda_b^-1 eta_b;
  5. mu_bar <- mu_bar (+) tau (right-plus on the pose, plus on log-depth);
  6. project stored messages and beliefs onto the tangent space at the new
     linearisation point, first order: eta <- eta - Lambda tau (Sec. 4.1).
The pose estimate of a frame is the pixel average of the pose components
(App. C.2, estimator equation).

Message slots per pixel: 0..3 identity factor shared with the left, right,
upper, lower neighbour; 4..7 normal-integration factor, same order. Slots whose
neighbour lies outside the window hold zero.

Test infrastructure: this package is the CPU oracle. Only tests/, the smoke check
and the bench's CPU-baseline leg may import it.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

from . import factors as fac
from . import lie
from .factors import Intrinsics

LEFT, RIGHT, UP, DOWN = 0, 1, 2, 3
NORMAL = 4          # offset of the normal-integration slots
N_SLOTS = 8


@dataclass(frozen=True)
class Params:
    """Factor strengths (Sec. 4.2: sigma_D, sigma_P, sigma_R, sigma_N, t_huber at
    their paper values), the log-depth prior sigma_Z (not given by the paper) and
    the message damping beta (not in the paper)."""
    sigma_D: float = 5e-3
    sigma_P: float = 1.0
    sigma_R: float = 4e-4
    sigma_N: float = 1e-3
    sigma_Z: float = 1.0
    t_huber: float = 400.0
    damping: float = 0.5


@dataclass
class Window:
    """A rectangular window [v0, v0+h) x [u0, u0+w) of the keyframe with the data
    its pixels need. I_t, g_x, g_y are the whole target image (warps may land
    anywhere); I_s, m_x, m_y cover the window only."""
    K: Intrinsics
    I_s: np.ndarray
    m_x: np.ndarray
    m_y: np.ndarray
    I_t: np.ndarray
    g_x: np.ndarray
    g_y: np.ndarray
    u0: int = 0
    v0: int = 0
    d_prior: float = 0.0

    @property
    def shape(self):
        return self.I_s.shape

    def coords(self):
        h, w = self.shape
        uu, vv = np.meshgrid(np.arange(w, dtype=np.float64) + self.u0,
                             np.arange(h, dtype=np.float64) + self.v0)
        return uu, vv


def make_window(K: Intrinsics, I_s, normals, I_t, d_prior=0.0) -> Window:
    """Whole-image window from a keyframe, its normals and a target frame."""
    m_x, m_y = fac.normal_edge_measurements(normals, K)
    g_x, g_y = fac.image_gradient(I_t)
    return Window(K, np.asarray(I_s, np.float64), m_x, m_y, np.asarray(I_t, np.float64),
                  g_x, g_y, 0, 0, float(d_prior))


@dataclass
class State:
    mu: np.ndarray        # (h, w, 7)
    bel_L: np.ndarray     # (h, w, 7, 7)
    bel_eta: np.ndarray   # (h, w, 7)
    msg_L: np.ndarray     # (h, w, 8, 7, 7)
    msg_eta: np.ndarray   # (h, w, 8, 7)
    diag: dict = field(default_factory=dict)


def reset_state(shape, d0: float, params: Params, d_prior: float | None = None) -> State:
    """Keyframe initial state: identity pose, log-depth d0, no messages, and the
    belief equal to the prior factors at that point."""
    h, w = shape
    mu = np.zeros((h, w, 7))
    mu[..., 6] = d0
    Lp, ep = fac.pose_prior_factor(mu[..., :6], params.sigma_P)
    Lz, ez = fac.depth_prior_factor(mu[..., 6], d0 if d_prior is None else d_prior, params.sigma_Z)
    return State(mu, Lp + Lz, ep + ez, np.zeros((h, w, N_SLOTS, 7, 7)),
                 np.zeros((h, w, N_SLOTS, 7)))


# --------------------------------------------------------------------------
# factors at the current linearisation point
# --------------------------------------------------------------------------
def unary(win: Window, mu, params: Params):
    """Photometric (Eq. 3), pose prior (Eq. 4) and log-depth prior factors."""
    uu, vv = win.coords()
    xi, d = mu[..., :6], mu[..., 6]
    Lph, eph, diag = fac.photometric_factor(xi, d, uu, vv, win.I_s, win.I_t, win.g_x, win.g_y,
                                            win.K, params.sigma_D, params.t_huber)
    Lp, ep = fac.pose_prior_factor(xi, params.sigma_P)
    Lz, ez = fac.depth_prior_factor(d, win.d_prior, params.sigma_Z)
    return Lph + Lp + Lz, eph + ep + ez, diag


def edge_factors(win: Window, mu, params: Params):
    """Linearised identity (Eq. 5) and normal-integration (Eq. 6) factors on the
    horizontal edges (a = (v, u), b = (v, u+1)) and vertical edges (a = (v, u),
    b = (v+1, u)). Each is (Lambda 14x14, eta 14) over (x_a, x_b)."""
    xi, d = mu[..., :6], mu[..., 6]
    return {
        "id_h": fac.identity_factor(xi[:, :-1], xi[:, 1:], params.sigma_R),
        "id_v": fac.identity_factor(xi[:-1, :], xi[1:, :], params.sigma_R),
        "nm_h": fac.normal_factor(d[:, :-1], d[:, 1:], win.m_x, params.sigma_N),
        "nm_v": fac.normal_factor(d[:-1, :], d[1:, :], win.m_y, params.sigma_N),
    }


# --------------------------------------------------------------------------
# messages
# --------------------------------------------------------------------------
def factor_to_variable(Lam_f, eta_f, Lam_in, eta_in, to: int):
    """Message from a pairwise factor to its variable ``to`` (0 = a, 1 = b): add the
    other variable's incoming message to the factor, then marginalise the other
    variable out (Schur complement)."""
    keep = slice(7, 14) if to == 1 else slice(0, 7)
    other = slice(0, 7) if to == 1 else slice(7, 14)
    Lam = Lam_f.copy()
    eta = eta_f.copy()
    Lam[..., other, other] += Lam_in
    eta[..., other] += eta_in
    A = Lam[..., keep, keep]
    B = Lam[..., keep, other]
    C = Lam[..., other, other]
    rhs = np.concatenate([Lam[..., other, keep], eta[..., other, None]], -1)
    X = np.linalg.solve(C, rhs)
    return A - B @ X[..., :7], eta[..., keep] - (B @ X[..., 7:])[..., 0]


def pairwise_messages(F: dict, st: State):
    """All new factor-to-variable messages of one synchronous step."""
    new_L = np.zeros_like(st.msg_L)
    new_eta = np.zeros_like(st.msg_eta)

    def v2f(sl, slot):
        return st.bel_L[sl] - st.msg_L[sl][..., slot, :, :], st.bel_eta[sl] - st.msg_eta[sl][..., slot, :]

    A_h, B_h = (slice(None), slice(None, -1)), (slice(None), slice(1, None))
    A_v, B_v = (slice(None, -1), slice(None)), (slice(1, None), slice(None))
    for kind, off in (("id", 0), ("nm", NORMAL)):
        for (A, B, slot_a, slot_b, key) in ((A_h, B_h, RIGHT, LEFT, kind + "_h"),
                                            (A_v, B_v, DOWN, UP, kind + "_v")):
            Lf, ef = F[key]
            La, ea = v2f(A, off + slot_a)
            Lb, eb = v2f(B, off + slot_b)
            Lm, em = factor_to_variable(Lf, ef, La, ea, to=1)
            new_L[B][..., off + slot_b, :, :] = Lm
            new_eta[B][..., off + slot_b, :] = em
            Lm, em = factor_to_variable(Lf, ef, Lb, eb, to=0)
            new_L[A][..., off + slot_a, :, :] = Lm
            new_eta[A][..., off + slot_a, :] = em
    return new_L, new_eta


# --------------------------------------------------------------------------
# one synchronous sweep with relinearisation
# --------------------------------------------------------------------------
def sweep(win: Window, st: State, params: Params) -> State:
    Lu, eu, diag = unary(win, st.mu, params)
    F = edge_factors(win, st.mu, params)
    nL, ne = pairwise_messages(F, st)
    beta = params.damping
    mL = (1.0 - beta) * nL + beta * st.msg_L
    me = (1.0 - beta) * ne + beta * st.msg_eta
    bL = Lu + mL.sum(axis=2)
    be = eu + me.sum(axis=2)
    tau = np.linalg.solve(bL, be[..., None])[..., 0]
    mu = np.empty_like(st.mu)
    mu[..., :6] = lie.se3_boxplus(st.mu[..., :6], tau[..., :6])
    mu[..., 6] = st.mu[..., 6] + tau[..., 6]
    me = me - (mL @ tau[:, :, None, :, None])[..., 0]
    be = be - (bL @ tau[..., None])[..., 0]
    return State(mu, bL, be, mL, me, {"tau": tau, **diag})


def pose_estimate(mu) -> np.ndarray:
    """xi_est = (1/N) sum_i mu_i[0:6] (App. C.2, estimator equation)."""
    return mu[..., :6].reshape(-1, 6).mean(axis=0)


# --------------------------------------------------------------------------
# frozen linearisation and the dense system (used to pin the message passing)
# --------------------------------------------------------------------------
def frozen_gbp(win: Window, mu0, params: Params, max_iter=20000, tol=1e-13):
    """GBP on the linear Gaussian system obtained by linearising every factor once
    at mu0. Returns the belief means tau (in the tangent space at mu0), the belief
    information matrices and the number of sweeps run."""
    Lu, eu, _ = unary(win, mu0, params)
    F = edge_factors(win, mu0, params)
    h, w = mu0.shape[:2]
    st = State(mu0, Lu.copy(), eu.copy(), np.zeros((h, w, N_SLOTS, 7, 7)),
               np.zeros((h, w, N_SLOTS, 7)))
    beta = params.damping
    it = 0
    for it in range(1, max_iter + 1):
        nL, ne = pairwise_messages(F, st)
        mL = (1.0 - beta) * nL + beta * st.msg_L
        me = (1.0 - beta) * ne + beta * st.msg_eta
        change = max(np.abs(mL - st.msg_L).max() / (1.0 + np.abs(mL).max()),
                     np.abs(me - st.msg_eta).max() / (1.0 + np.abs(me).max()))
        st = State(mu0, Lu + mL.sum(axis=2), eu + me.sum(axis=2), mL, me)
        if change < tol:
            break
    tau = np.linalg.solve(st.bel_L, st.bel_eta[..., None])[..., 0]
    return tau, st.bel_L, it


def dense_system(win: Window, mu, params: Params):
    """Sum every linearised factor into one (7N x 7N) information matrix and 7N
    vector (pixel-major, 7 unknowns per pixel)."""
    h, w = mu.shape[:2]
    n = h * w * 7
    Lam = np.zeros((n, n))
    eta = np.zeros(n)
    Lu, eu, _ = unary(win, mu, params)
    F = edge_factors(win, mu, params)

    def blk(r, c):
        return slice((r * w + c) * 7, (r * w + c) * 7 + 7)

    for r in range(h):
        for c in range(w):
            Lam[blk(r, c), blk(r, c)] += Lu[r, c]
            eta[blk(r, c)] += eu[r, c]
    edges = [("id_h", r, c, r, c + 1) for r in range(h) for c in range(w - 1)]
    edges += [("nm_h", r, c, r, c + 1) for r in range(h) for c in range(w - 1)]
    edges += [("id_v", r, c, r + 1, c) for r in range(h - 1) for c in range(w)]
    edges += [("nm_v", r, c, r + 1, c) for r in range(h - 1) for c in range(w)]
    for key, ra, ca, rb, cb in edges:
        Lf, ef = F[key]
        Lf, ef = Lf[ra, ca], ef[ra, ca]
        ia, ib = blk(ra, ca), blk(rb, cb)
        Lam[ia, ia] += Lf[:7, :7]
        Lam[ia, ib] += Lf[:7, 7:]
        Lam[ib, ia] += Lf[7:, :7]
        Lam[ib, ib] += Lf[7:, 7:]
        eta[ia] += ef[:7]
        eta[ib] += ef[7:]
    return Lam, eta


def with_params(p: Params, **kw) -> Params:
    return replace(p, **kw)
