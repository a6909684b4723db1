"""Pins of the hierarchical (quadtree) identity topology in the oracle
(oracle/quadtree.py), against the dense linear algebra of the same factors:

* with the normal-integration factors off the factor graph is a tree, so
  undamped GBP with frozen linearisation is exact after as many sweeps as the
  tree is deep: means and marginal covariances equal the dense inverse;
* with them on (loops through the pixel grid) the damped GBP fixed point has the
  dense solve's means (exactness of GBP means at a fixed point);
* relinearised sweeps converge to a point where one dense Gauss-Newton step of
  the same factors is zero;
* level shapes and the slot layout.
"""
import numpy as np
import pytest

import synth
from oracle import factors as fac
from oracle import gbp
from oracle import quadtree as qt
from oracle.factors import Intrinsics


# couplings weak enough for loopy GBP to converge on an 8x8 window (as in the
# grid's fixed-point pin)
MILD = gbp.Params(sigma_D=0.05, sigma_P=1.0, sigma_R=0.3, sigma_N=0.2, sigma_Z=1.0)


def window(h=8, w=8, seed=0):
    """A crop of the tiny pair with its camera re-centred on the crop."""
    seq = synth.tiny_pair(seed)
    fx, fy, cx, cy, W, H = seq.cam.as_tuple()
    v0, u0 = (H - h) // 2, (W - w) // 2
    K = Intrinsics(fx, fy, cx - u0, cy - v0, w, h)
    crop = (slice(v0, v0 + h), slice(u0, u0 + w))
    I_s = seq.frame(0).astype(np.float64)[crop]
    I_t = seq.frame(1).astype(np.float64)[crop]
    return gbp.make_window(K, I_s, seq.normals(0).astype(np.float64)[crop], I_t, 0.0)


def start_means(win, seed=1):
    rng = np.random.default_rng(seed)
    h, w = win.shape
    mus = [np.concatenate([0.01 * rng.normal(size=(h, w, 6)), 0.3 + 0.1 * rng.normal(size=(h, w, 1))], -1)]
    for (hl, wl) in qt.level_shapes(h, w):
        mus.append(np.concatenate([0.01 * rng.normal(size=(hl, wl, 6)), np.zeros((hl, wl, 1))], -1))
    return mus


def dense_blocks(Lam, eta, mus):
    x = np.linalg.solve(Lam, eta)
    cov = np.linalg.inv(Lam)
    out, i = [], 0
    for m in mus:
        n = m.shape[0] * m.shape[1]
        xs = x[7 * i:7 * (i + n)].reshape(m.shape[0], m.shape[1], 7)
        cs = np.stack([cov[7 * (i + j):7 * (i + j + 1), 7 * (i + j):7 * (i + j + 1)] for j in range(n)])
        out.append((xs, cs.reshape(m.shape[0], m.shape[1], 7, 7)))
        i += n
    return out


def test_level_shapes():
    assert qt.level_shapes(48, 64) == [(24, 32), (12, 16), (6, 8), (3, 4), (2, 2), (1, 1)]
    assert qt.level_shapes(17, 33) == [(9, 17), (5, 9), (3, 5), (2, 3), (1, 2), (1, 1)]
    assert qt.level_shapes(1, 1) == []


def test_level_strengths_match_the_printed_geometric_means():
    """App. E.2 prints the geometric means of the per-layer strengths of the
    hierarchy the paper runs on its 128 x 128 images (sigma_R = 3.536e-5,
    sigma_P = 8.839e-2 from the Sec. 4.2 leaf values). A 128 x 128 tree has eight
    layers (the pixels and seven node levels). Layer l's sigma_P is that of its
    own prior; its sigma_R is that of the factor joining it to its parent, and
    the root's is the value the halving rule gives the layer above the last
    factor (it has no parent, the mean still counts it). A schedule that halves
    from the wrong layer (sigma_R / 2^l between levels l - 1 and l) or at another
    rate misses the printed values by a factor of 1.4 or more."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")) as fh:
        gold = json.load(fh)
    leaf = gold["sec4_2_leaf"]
    p = gbp.Params(sigma_P=leaf["sigma_P"], sigma_R=leaf["sigma_R"])
    layers = len(qt.level_shapes(128, 128)) + 1
    assert layers == 8
    s_P = [qt.sigma_P_at(p, l) for l in range(layers)]
    s_R = [qt.sigma_R_between(p, l + 1) for l in range(layers)]
    gmean = lambda xs: float(np.exp(np.mean(np.log(xs))))  # noqa: E731
    # the paper prints four significant digits
    assert gmean(s_P) == pytest.approx(gold["appE2_geometric_mean"]["sigma_P"], rel=6e-4)
    assert gmean(s_R) == pytest.approx(gold["appE2_geometric_mean"]["sigma_R"], rel=6e-4)
    # consecutive layers differ by the Sec. 4.2 factor
    for a, b in zip(s_P[1:], s_P[:-1]):
        assert a / b == pytest.approx(gold["sec4_2_level_factor"])
    # only the seven factors below the root exist in the oracle's tree
    assert len(s_R[:-1]) == len(qt.level_shapes(128, 128))


@pytest.mark.parametrize("shape", [(8, 8), (6, 7)])
def test_tree_is_exact_after_its_depth(shape):
    win = window(*shape)
    p = gbp.Params(sigma_P=0.1, sigma_N=np.inf, damping=0.0)
    mus = start_means(win)
    depth = len(mus)
    taus, bels, _ = qt.frozen_tree(win, mus, p, n_iter=2 * depth + 2)
    ref = dense_blocks(*qt.dense_tree(win, mus, p), mus)
    for tau, bel, (x, cov) in zip(taus, bels, ref):
        scale = np.abs(x).max()
        assert np.abs(tau - x).max() <= 1e-9 * scale
        marg = np.linalg.inv(bel)
        assert np.abs(marg - cov).max() <= 1e-9 * np.abs(cov).max()


def test_fewer_sweeps_than_the_depth_are_not_exact():
    """The previous pin is not vacuous: one sweep short of the leaf-root-leaf path
    the root's information has not reached every pixel."""
    win = window(8, 8)
    p = gbp.Params(sigma_P=0.1, sigma_N=np.inf, damping=0.0)
    mus = start_means(win)
    taus, _, _ = qt.frozen_tree(win, mus, p, n_iter=2)
    x = dense_blocks(*qt.dense_tree(win, mus, p), mus)[0][0]
    assert np.abs(taus[0] - x).max() > 1e-6 * np.abs(x).max()


def test_loopy_fixed_point_has_the_dense_means():
    win = window(8, 8)
    p = MILD
    mus = start_means(win)
    taus, _, it = qt.frozen_tree(win, mus, p, n_iter=5000, tol=1e-14)
    assert it < 5000
    ref = dense_blocks(*qt.dense_tree(win, mus, p), mus)
    for tau, (x, _) in zip(taus, ref):
        assert np.abs(tau - x).max() <= 1e-8 * np.abs(x).max()


def test_relinearised_sweeps_reach_a_gauss_newton_stationary_point():
    """As the grid's pin: on the exactly-bilinear image pair (a smooth photometric
    model; the block texture makes the relinearised iteration cycle), one dense
    Gauss-Newton step from the converged means is zero."""
    seq = synth.tiny_pair(0)
    K = Intrinsics(*seq.cam.as_tuple())
    aff = synth.affine_pair(seq)
    m_x, m_y = fac.normal_edge_measurements(aff["normal"], K)
    g_x, g_y = fac.image_gradient(aff["I_t"])
    v0, u0, h, w = 16, 24, 5, 6
    win = gbp.Window(K, aff["I_s"][v0:v0 + h, u0:u0 + w], m_x[v0:v0 + h, u0:u0 + w - 1],
                     m_y[v0:v0 + h - 1, u0:u0 + w], aff["I_t"], g_x, g_y, u0, v0, 0.3)
    st = qt.reset_tree((h, w), 0.3, MILD)
    for _ in range(1000):
        st = qt.sweep_tree(win, st, MILD)
    assert st.pixels.diag["valid"].all()
    mus = [st.pixels.mu] + [n.mu for n in st.nodes]
    Lam, eta = qt.dense_tree(win, mus, MILD)
    step = np.linalg.solve(Lam, eta)
    assert np.abs(step).max() < 1e-9
    assert np.abs(st.pixels.diag["tau"]).max() < 1e-9


def test_slot_layout():
    win = window(6, 7)
    p = gbp.Params(sigma_P=0.1)
    st = qt.reset_tree(win.shape, 0.0, p)
    st = qt.sweep_tree(win, st, p)
    assert np.all(st.pixels.msg_L[..., 1:4, :, :] == 0.0)
    assert np.any(st.pixels.msg_L[..., 0, :6, :6] != 0.0)
    # every node has its parent message except the root, and messages only from
    # the children that exist
    for lvl, n in enumerate(st.nodes, start=1):
        has_parent = lvl < len(st.nodes)
        assert np.any(n.msg_L[..., qt.NODE_PARENT, :6, :6] != 0.0) == has_parent
    last = st.nodes[0]     # level 1 over 6x7 pixels: 3x4 nodes, the last column has one child column
    assert np.all(last.msg_L[:, -1, 1, :, :] == 0.0) and np.all(last.msg_L[:, -1, 3, :, :] == 0.0)
