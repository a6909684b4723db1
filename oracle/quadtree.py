"""GBP with the hierarchical identity topology, FP64 (numpy).

The camera-motion identity factors (Eq. 5) do not join grid neighbours here:
each pixel's pose is joined to a pose node of level 1, which covers a 2x2 block
of pixels; each node of level l is joined to the node of level l + 1 covering
its 2x2 block of level-l nodes, up to a single root (Sec. 3.3 and its factor
graph figure: the hierarchical quadtree pattern of the main experiments). The
factor between levels l - 1 and l uses sigma_R / 2^(l-1) and a node of level l
carries a pose prior with sigma_P / 2^l (Sec. 4.2: both halved at each higher
level than the leaf). The normal-integration factors (Eq. 6) keep the grid.

Readings: nodes of a ragged image cover the blocks that exist (ceil(h / 2^l) x
ceil(w / 2^l) nodes at level l; an edge node has fewer than four children); the
levels stop at the first level of one node; the pose estimate stays the pixel
average (App. C.2). A node is a 7-D variable like a pixel, whose seventh
component is a dummy held by a unit-information prior at zero: the identity
factors do not touch it, so it decouples exactly and the textbook 14-D factor
and message code of gbp.py is used unchanged.

Message slots: a pixel uses slot 0 for the factor to its level-1 node and slots
4..7 for its normal-integration factors (as in gbp.py); slots 1..3 stay zero. A
node uses slots 0..3 for its children (index 2 (row % 2) + (col % 2) of the
child) and slot 4 for its parent.

Test infrastructure: this package is the CPU oracle. Only tests/, the smoke check
and the bench's CPU-baseline leg may import it.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import factors as fac
from . import gbp, lie
from .gbp import NORMAL, N_SLOTS, Params, State, Window

PARENT = 0          # pixel slot of the factor to the level-1 node
NODE_SLOTS = 5      # node slots: 0..3 children, 4 parent
NODE_PARENT = 4


def level_shapes(h: int, w: int) -> list:
    """Node grid shapes of levels 1..L (L: the first level with one node)."""
    shapes = []
    while h > 1 or w > 1:
        h, w = (h + 1) // 2, (w + 1) // 2
        shapes.append((h, w))
    return shapes


def sigma_R_between(params: Params, level: int) -> float:
    """Identity factor between levels level - 1 and level (level >= 1)."""
    return params.sigma_R / 2.0 ** (level - 1)


def sigma_P_at(params: Params, level: int) -> float:
    return params.sigma_P / 2.0 ** level


@dataclass
class TreeState:
    pixels: State          # as gbp.State (slot 0 = parent)
    nodes: list            # per level >= 1: gbp.State with NODE_SLOTS slots


def node_unary(mu, level: int, params: Params):
    """Pose prior of a level-`level` node and the unit prior on its dummy component."""
    Lp, ep = fac.pose_prior_factor(mu[..., :6], sigma_P_at(params, level))
    Ld, ed = fac.depth_prior_factor(mu[..., 6], 0.0, 1.0)
    return Lp + Ld, ep + ed


def reset_tree(shape, d0: float, params: Params, d_prior: float | None = None) -> TreeState:
    """Keyframe initial state: identity poses, log-depth d0, no messages, beliefs
    equal to the unary priors."""
    px = gbp.reset_state(shape, d0, params, d_prior)
    nodes = []
    for lvl, (h, w) in enumerate(level_shapes(*shape), start=1):
        mu = np.zeros((h, w, 7))
        L, e = node_unary(mu, lvl, params)
        nodes.append(State(mu, L, e, np.zeros((h, w, NODE_SLOTS, 7, 7)), np.zeros((h, w, NODE_SLOTS, 7))))
    return TreeState(px, nodes)


def _children(level_mu_child, h_par: int, w_par: int):
    """For each child slot k = 2 dr + dc: (index arrays of the children that exist,
    index arrays of their parents)."""
    hc, wc = level_mu_child.shape[:2]
    out = []
    for dr in (0, 1):
        for dc in (0, 1):
            rp, cp = np.meshgrid(np.arange(h_par), np.arange(w_par), indexing="ij")
            rc, cc = 2 * rp + dr, 2 * cp + dc
            ok = (rc < hc) & (cc < wc)
            out.append((2 * dr + dc, (rc[ok], cc[ok]), (rp[ok], cp[ok])))
    return out


def _levels(st: TreeState):
    """[(state, parent slot, level)] for pixels (level 0) and nodes."""
    return [(st.pixels, PARENT, 0)] + [(n, NODE_PARENT, l) for l, n in enumerate(st.nodes, start=1)]


def tree_messages(st: TreeState, params: Params, mus=None):
    """New identity messages of one synchronous step, linearised at `mus` (per
    level means; the current means by default): (pixel msg arrays, node msg arrays)."""
    levels = _levels(st)
    mus = [s.mu for s, _, _ in levels] if mus is None else mus
    new = [(np.zeros_like(s.msg_L), np.zeros_like(s.msg_eta)) for s, _, _ in levels]
    for lvl in range(1, len(levels)):
        child, cslot, _ = levels[lvl - 1]
        par = levels[lvl][0]
        hp, wp = par.mu.shape[:2]
        for k, ci, pi in _children(mus[lvl - 1], hp, wp):
            if len(ci[0]) == 0:
                continue
            Lf, ef = fac.identity_factor(mus[lvl - 1][ci][..., :6], mus[lvl][pi][..., :6],
                                         sigma_R_between(params, lvl))
            # a = child, b = parent
            La = child.bel_L[ci] - child.msg_L[ci][:, cslot]
            ea = child.bel_eta[ci] - child.msg_eta[ci][:, cslot]
            Lb = par.bel_L[pi] - par.msg_L[pi][:, k]
            eb = par.bel_eta[pi] - par.msg_eta[pi][:, k]
            Lm, em = gbp.factor_to_variable(Lf, ef, La, ea, to=1)
            new[lvl][0][pi[0], pi[1], k] = Lm
            new[lvl][1][pi[0], pi[1], k] = em
            Lm, em = gbp.factor_to_variable(Lf, ef, Lb, eb, to=0)
            new[lvl - 1][0][ci[0], ci[1], cslot] = Lm
            new[lvl - 1][1][ci[0], ci[1], cslot] = em
    return new


def normal_messages(win: Window, st: State, params: Params, mu=None):
    """New normal-integration messages (pixel slots 4..7), factors linearised at
    `mu` (the current means by default), as in gbp.pairwise_messages."""
    mu = st.mu if mu is None else mu
    d = mu[..., 6]
    F = {"nm_h": fac.normal_factor(d[:, :-1], d[:, 1:], win.m_x, params.sigma_N),
         "nm_v": fac.normal_factor(d[:-1, :], d[1:, :], win.m_y, params.sigma_N)}
    new_L = np.zeros_like(st.msg_L)
    new_eta = np.zeros_like(st.msg_eta)

    def v2f(sl, slot):
        return st.bel_L[sl] - st.msg_L[sl][..., slot, :, :], st.bel_eta[sl] - st.msg_eta[sl][..., slot, :]

    A_h, B_h = (slice(None), slice(None, -1)), (slice(None), slice(1, None))
    A_v, B_v = (slice(None, -1), slice(None)), (slice(1, None), slice(None))
    for (A, B, slot_a, slot_b, key) in ((A_h, B_h, gbp.RIGHT, gbp.LEFT, "nm_h"),
                                        (A_v, B_v, gbp.DOWN, gbp.UP, "nm_v")):
        Lf, ef = F[key]
        La, ea = v2f(A, NORMAL + slot_a)
        Lb, eb = v2f(B, NORMAL + slot_b)
        Lm, em = gbp.factor_to_variable(Lf, ef, La, ea, to=1)
        new_L[B][..., NORMAL + slot_b, :, :] = Lm
        new_eta[B][..., NORMAL + slot_b, :] = em
        Lm, em = gbp.factor_to_variable(Lf, ef, Lb, eb, to=0)
        new_L[A][..., NORMAL + slot_a, :, :] = Lm
        new_eta[A][..., NORMAL + slot_a, :] = em
    return new_L, new_eta


def _unaries(win: Window, mus, params: Params):
    Lu, eu, diag = gbp.unary(win, mus[0], params)
    return [(Lu, eu)] + [node_unary(m, l, params) for l, m in enumerate(mus[1:], start=1)], diag


def _new_messages(win: Window, st: TreeState, params: Params, mus):
    new = tree_messages(st, params, mus)
    nL, ne = normal_messages(win, st.pixels, params, mus[0])
    new[0] = (new[0][0] + nL, new[0][1] + ne)   # disjoint slots
    return new


def sweep_tree(win: Window, st: TreeState, params: Params) -> TreeState:
    """One synchronous sweep (same steps as gbp.sweep) over pixels and nodes."""
    levels = _levels(st)
    mus = [s.mu for s, _, _ in levels]
    un, diag = _unaries(win, mus, params)
    new = _new_messages(win, st, params, mus)
    beta = params.damping
    out = []
    for (s, _, _), (Lu, eu), (nL, ne) in zip(levels, un, new):
        mL = (1.0 - beta) * nL + beta * s.msg_L
        me = (1.0 - beta) * ne + beta * s.msg_eta
        bL = Lu + mL.sum(axis=2)
        be = eu + me.sum(axis=2)
        tau = np.linalg.solve(bL, be[..., None])[..., 0]
        mu = np.empty_like(s.mu)
        mu[..., :6] = lie.se3_boxplus(s.mu[..., :6], tau[..., :6])
        mu[..., 6] = s.mu[..., 6] + tau[..., 6]
        me = me - (mL @ tau[..., None, :, None])[..., 0]
        be = be - (bL @ tau[..., None])[..., 0]
        out.append(State(mu, bL, be, mL, me, {"tau": tau}))
    out[0].diag.update(diag)
    return TreeState(out[0], out[1:])


def frozen_tree(win: Window, mus0, params: Params, n_iter: int, tol: float = 0.0):
    """GBP on the system linearised once at the means mus0 (per level): beliefs =
    unary + incoming messages, no relinearisation or projection. Returns the belief
    means (tangent offsets at mus0), belief informations and the sweeps run."""
    un, _ = _unaries(win, mus0, params)
    st = TreeState(State(mus0[0], un[0][0].copy(), un[0][1].copy(),
                         np.zeros(mus0[0].shape[:2] + (N_SLOTS, 7, 7)), np.zeros(mus0[0].shape[:2] + (N_SLOTS, 7))),
                   [State(m, u[0].copy(), u[1].copy(), np.zeros(m.shape[:2] + (NODE_SLOTS, 7, 7)),
                          np.zeros(m.shape[:2] + (NODE_SLOTS, 7))) for m, u in zip(mus0[1:], un[1:])])
    beta = params.damping
    it = 0
    for it in range(1, n_iter + 1):
        new = _new_messages(win, st, params, mus0)
        levels, change = [], 0.0
        for s, (Lu, eu), (nL, ne) in zip([st.pixels] + st.nodes, un, new):
            mL = (1.0 - beta) * nL + beta * s.msg_L
            me = (1.0 - beta) * ne + beta * s.msg_eta
            change = max(change, np.abs(mL - s.msg_L).max() / (1.0 + np.abs(mL).max()),
                         np.abs(me - s.msg_eta).max() / (1.0 + np.abs(me).max()))
            levels.append(State(s.mu, Lu + mL.sum(axis=2), eu + me.sum(axis=2), mL, me))
        st = TreeState(levels[0], levels[1:])
        if change < tol:
            break
    taus = [np.linalg.solve(s.bel_L, s.bel_eta[..., None])[..., 0] for s in [st.pixels] + st.nodes]
    return taus, [s.bel_L for s in [st.pixels] + st.nodes], it


def dense_tree(win: Window, mus, params: Params):
    """Every linearised factor summed into one information matrix and vector over
    all variables (pixels row-major, then each level's nodes row-major, 7 each)."""
    shapes = [m.shape[:2] for m in mus]
    offs = np.cumsum([0] + [h * w for h, w in shapes])
    n = int(offs[-1]) * 7
    Lam, eta = np.zeros((n, n)), np.zeros(n)

    def blk(lvl, r, c):
        i = (int(offs[lvl]) + r * shapes[lvl][1] + c) * 7
        return slice(i, i + 7)

    def add(ia, ib, Lf, ef):
        Lam[ia, ia] += Lf[:7, :7]
        Lam[ia, ib] += Lf[:7, 7:]
        Lam[ib, ia] += Lf[7:, :7]
        Lam[ib, ib] += Lf[7:, 7:]
        eta[ia] += ef[:7]
        eta[ib] += ef[7:]

    un, _ = _unaries(win, mus, params)
    for lvl, (Lu, eu) in enumerate(un):
        for r in range(shapes[lvl][0]):
            for c in range(shapes[lvl][1]):
                Lam[blk(lvl, r, c), blk(lvl, r, c)] += Lu[r, c]
                eta[blk(lvl, r, c)] += eu[r, c]
    for lvl in range(1, len(mus)):
        hc, wc = shapes[lvl - 1]
        for r in range(hc):
            for c in range(wc):
                Lf, ef = fac.identity_factor(mus[lvl - 1][r, c, :6], mus[lvl][r // 2, c // 2, :6],
                                             sigma_R_between(params, lvl))
                add(blk(lvl - 1, r, c), blk(lvl, r // 2, c // 2), Lf, ef)
    d = mus[0][..., 6]
    h, w = shapes[0]
    for r in range(h):
        for c in range(w):
            if c + 1 < w:
                Lf, ef = fac.normal_factor(d[r, c], d[r, c + 1], win.m_x[r, c], params.sigma_N)
                add(blk(0, r, c), blk(0, r, c + 1), Lf, ef)
            if r + 1 < h:
                Lf, ef = fac.normal_factor(d[r, c], d[r + 1, c], win.m_y[r, c], params.sigma_N)
                add(blk(0, r, c), blk(0, r + 1, c), Lf, ef)
    return Lam, eta
