"""CPU checks of the test glue used by the GPU parity tests: the compressed
(library-layout) state reproduces the oracle's sweep exactly, and checkpoint
blobs written from oracle states decode to the same fields."""
import numpy as np
import pytest

from oracle import gbp
from helpers import (blob_from_compressed, compressed_from_oracle, oracle_intrinsics, oracle_params,
                     oracle_state_from_compressed, oracle_window, rounded, run_oracle_pair,
                     synthetic_state)

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def test_surrogate_belief_gives_the_same_sweep(tiny_seq):
    """One oracle sweep from the block-diagonal surrogate diag(P, s) equals one
    oracle sweep from the full 7x7 belief (the messages depend only on the
    marginals P and s, and the new belief only on unary factors and messages)."""
    K = oracle_intrinsics(tiny_seq.cam)
    p = oracle_params(sigma_P=tiny_seq.sigma_P)
    st, rec, win = run_oracle_pair(tiny_seq, K, p, 4, record=(2, 4))
    for k, s in rec.items():
        ref = gbp.sweep(win, s, p)
        c = compressed_from_oracle(s, 1 / p.sigma_P ** 2)
        # u u^T reproduces the rank-one part P - M_p
        np.testing.assert_allclose(c["M_p"] + np.stack(
            [c["u"][..., r] * c["u"][..., q] for r in range(6) for q in range(r + 1)], -1), c["P"],
            rtol=1e-9, atol=1e-9 * np.abs(c["P"]).max())
        sur = gbp.sweep(win, oracle_state_from_compressed(c), p)
        np.testing.assert_allclose(sur.mu, ref.mu, rtol=1e-9, atol=1e-10)
        np.testing.assert_allclose(sur.msg_L, ref.msg_L, rtol=1e-9, atol=1e-9 * np.abs(ref.msg_L).max())
        np.testing.assert_allclose(sur.msg_eta, ref.msg_eta, rtol=1e-8, atol=1e-8 * np.abs(ref.msg_eta).max())


def test_checkpoint_blob_decodes_to_the_same_fields(tiny_seq):
    pv = pytest.importorskip("paper_2606_03989_gb300")
    from paper_2606_03989_gb300 import build
    build.build()
    K = oracle_intrinsics(tiny_seq.cam)
    p = oracle_params(sigma_P=tiny_seq.sigma_P)
    win = oracle_window(tiny_seq, K)
    c = synthetic_state(48, 64, p, seed=1)
    for prec in (64, 32):
        cr = rounded(c, prec)
        view = pv.parse_state(blob_from_compressed(cr, win, prec, frame_index=5, d_prior=0.25))
        assert view.frame_index == 5 and view.has_target and view.d_prior == 0.25
        np.testing.assert_array_equal(view.mu, cr["mu"])
        np.testing.assert_array_equal(view.M_p, cr["M_p"])
        np.testing.assert_array_equal(view.u, cr["u"])
        np.testing.assert_array_equal(view.identity_messages, cr["id"])
        np.testing.assert_array_equal(view.normal_messages, cr["nm"])
        np.testing.assert_allclose(view.P, cr["P"], rtol=1e-15, atol=0)
        np.testing.assert_array_equal(view.inputs[1], np.asarray(win.I_t, np.float32 if prec == 32 else np.float64))


def test_quadtree_checkpoint_node_section_decodes(tiny_seq):
    """Header words 12..14 (node count, node planes, byte offset) locate the node
    section a quadtree handle appends after the scalars; grid blobs have none."""
    pv = pytest.importorskip("paper_2606_03989_gb300")
    from paper_2606_03989_gb300 import build
    build.build()
    K = oracle_intrinsics(tiny_seq.cam)
    p = oracle_params(sigma_P=tiny_seq.sigma_P)
    win = oracle_window(tiny_seq, K)
    c = synthetic_state(48, 64, p, seed=3)
    from oracle import quadtree as qt
    n = sum(h * w for h, w in qt.level_shapes(48, 64))
    rng = np.random.default_rng(5)
    for prec in (64, 32):
        dt = np.float64 if prec == 64 else np.float32
        grid = blob_from_compressed(rounded(c, prec), win, prec)
        assert pv.parse_state(grid).nodes is None
        nodes = rng.normal(size=(162, n)).astype(dt)
        hd = np.frombuffer(grid, "<i8", count=32).copy()
        hd[12:15] = [n, 162, len(grid)]
        blob = hd.tobytes() + grid[256:] + nodes.tobytes()
        view = pv.parse_state(blob)
        np.testing.assert_array_equal(view.nodes, nodes.astype(np.float64))
        np.testing.assert_array_equal(view.node_pose, nodes[0:6].T.astype(np.float64))
        np.testing.assert_array_equal(view.mu, rounded(c, prec)["mu"])
