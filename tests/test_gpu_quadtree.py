"""Quadtree identity topology on the GPU (topology = PIXVOD_TOPOLOGY_QUADTREE)
against the quadtree oracle (oracle/quadtree.py, pinned in
test_oracle_quadtree.py): the pixel state after 1 and 3 synchronous sweeps from
the keyframe reset, on 16x12, a ragged 33x17 and 64x48 (six node levels), on
degenerate trees (one level; one node column or row), and after 2 sweeps at
640x480; the node states of every level; checkpoints of quadtree handles."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import synth  # noqa: E402
import paper_2606_03989_gb300 as pv  # noqa: E402
from oracle import gbp  # noqa: E402
from oracle import quadtree as qt  # noqa: E402
from helpers import (compressed_from_oracle, compressed_from_view, field_errors, oracle_intrinsics,  # noqa: E402
                     oracle_params, pack6)

DEV = torch.device("cuda:0")
SIZES = [(16, 12), (33, 17), (64, 48)]


def sequence(w, h):
    return synth.tiny_pair(0) if (w, h) == (64, 48) else synth.realistic(7, 2, w, h)


def run_pair(seq, precision, sweeps):
    p = pv.params(precision=precision, kf_interval=0, sigma_P=seq.sigma_P, topology=pv.TOPOLOGY_QUADTREE)
    trk = pv.Tracker(seq.cam.as_tuple(), p, DEV)
    trk.track(torch.from_numpy(seq.frame(0)).to(DEV), torch.from_numpy(seq.normals(0)).to(DEV))
    trk.track(torch.from_numpy(seq.frame(1)).to(DEV), n_iters=sweeps)
    return trk


def oracle_pair(seq, sweeps):
    p = oracle_params(sigma_P=seq.sigma_P)
    win = gbp.make_window(oracle_intrinsics(seq.cam), seq.frame(0).astype(np.float64),
                          seq.normals(0).astype(np.float64), seq.frame(1).astype(np.float64), 0.0)
    st = qt.reset_tree(win.shape, 0.0, p)
    for _ in range(sweeps):
        st = qt.sweep_tree(win, st, p)
    return st, p


@pytest.mark.parametrize("size", SIZES)
@pytest.mark.parametrize("sweeps", [1, 3])
def test_fp64_matches_the_quadtree_oracle(size, sweeps):
    seq = sequence(*size)
    st, p = oracle_pair(seq, sweeps)
    trk = run_pair(seq, 64, sweeps)
    assert trk.status() == 0
    err = field_errors(compressed_from_view(trk.state()), compressed_from_oracle(st.pixels, 1 / p.sigma_P ** 2))
    # one sweep from the same state agrees to rounding; the iteration then
    # amplifies rounding-order differences (measured 1.3e-9 on the means after 3)
    tol = 1e-9 if sweeps == 1 else 1e-8
    assert max(err["P"], err["M_p"], err["s"], err["id"], err["nm"]) < tol, err
    assert err["mu_abs"] < tol, err
    assert np.abs(trk.pose() - gbp.pose_estimate(st.pixels.mu)).max() < 1e-10


def oracle_nodes(st) -> dict:
    """The oracle's node states of all levels (level 1 first, row-major), in the
    checkpoint's node-plane order: pose, belief information (6x6 pose block,
    packed) and the messages of slots 0..4 (21 packed Lambda then 6 eta)."""
    mu = np.concatenate([n.mu[..., :6].reshape(-1, 6) for n in st.nodes])
    M = np.concatenate([pack6(n.bel_L[..., :6, :6]).reshape(-1, 21) for n in st.nodes])
    msg = np.concatenate([np.concatenate([pack6(n.msg_L[..., :, :6, :6]), n.msg_eta[..., :, :6]], -1)
                          .reshape(-1, qt.NODE_SLOTS, 27) for n in st.nodes])
    return {"mu": mu, "M": M, "msg": msg}


@pytest.mark.parametrize("size", SIZES)
def test_fp64_node_states_match_the_quadtree_oracle(size):
    """The checkpoint's node planes against the oracle's nodes after 3 sweeps:
    pose, belief information and the five message slots of every level."""
    seq = sequence(*size)
    st, p = oracle_pair(seq, 3)
    view = run_pair(seq, 64, 3).state()
    ora = oracle_nodes(st)
    n = ora["mu"].shape[0]
    assert view.nodes.shape == (162, n)
    nd = view.nodes.T
    got = {"mu": nd[:, 0:6], "M": nd[:, 6:27], "msg": nd[:, 27:162].reshape(n, qt.NODE_SLOTS, 27)}
    assert np.abs(got["mu"] - ora["mu"]).max() < 1e-8
    for k in ("M", "msg"):
        err = np.abs(got[k] - ora[k]).max() / np.abs(ora[k]).max()
        assert err < 1e-8, (k, err)
    # the root has no parent
    assert np.all(got["msg"][-1, qt.NODE_PARENT] == 0.0)


@pytest.mark.parametrize("size", [(2, 2), (2, 9), (9, 2), (5, 3)])
def test_degenerate_trees_fp64(size):
    """Trees of one level (2x2: the level-1 node is the root), one node column or
    row, and odd sides at every level: one FP64 sweep from the reset against the
    oracle, pixels and nodes."""
    seq = synth.realistic(7, 2, *size)
    st, p = oracle_pair(seq, 1)
    trk = run_pair(seq, 64, 1)
    assert trk.status() == 0
    view = trk.state()
    err = field_errors(compressed_from_view(view), compressed_from_oracle(st.pixels, 1 / p.sigma_P ** 2))
    assert max(err["P"], err["M_p"], err["s"], err["id"], err["nm"]) < 1e-9, err
    assert err["mu_abs"] < 1e-9, err
    ora = oracle_nodes(st)
    n = ora["mu"].shape[0]
    nd = view.nodes.T
    assert np.abs(nd[:, 0:6] - ora["mu"]).max() < 1e-9
    for got, ref in ((nd[:, 6:27], ora["M"]), (nd[:, 27:162].reshape(n, qt.NODE_SLOTS, 27), ora["msg"])):
        assert np.abs(got - ref).max() <= 1e-9 * max(np.abs(ref).max(), 1.0)


def test_full_size_two_sweeps_fp64():
    """640x480, the benchmark size: 10 node levels, 102,409 nodes, and every
    thread range of the node-message launch many blocks deep. Two FP64 sweeps
    from the keyframe reset against the oracle at every pixel and every node."""
    seq = synth.realistic(2, 2)
    st, p = oracle_pair(seq, 2)
    trk = run_pair(seq, 64, 2)
    assert trk.status() == 0
    view = trk.state()
    err = field_errors(compressed_from_view(view), compressed_from_oracle(st.pixels, 1 / p.sigma_P ** 2))
    assert max(err["P"], err["M_p"], err["s"], err["id"], err["nm"]) < 1e-8, err
    assert err["mu_abs"] < 1e-8, err
    ora = oracle_nodes(st)
    n = ora["mu"].shape[0]
    assert n == 102409 and view.nodes.shape == (162, n)
    nd = view.nodes.T
    assert np.abs(nd[:, 0:6] - ora["mu"]).max() < 1e-8
    assert np.abs(nd[:, 6:27] - ora["M"]).max() / np.abs(ora["M"]).max() < 1e-8
    msg = nd[:, 27:162].reshape(n, qt.NODE_SLOTS, 27)
    assert np.abs(msg - ora["msg"]).max() / np.abs(ora["msg"]).max() < 1e-8
    assert np.abs(trk.pose() - gbp.pose_estimate(st.pixels.mu)).max() < 1e-10


@pytest.mark.parametrize("precision", [32, 64])
def test_checkpoint_round_trip_continues_bit_identically(precision):
    """save after 2 sweeps, load into a fresh quadtree handle, 3 more sweeps on
    both: the pixel and node states agree bit for bit (the node states are in the
    checkpoint)."""
    seq = sequence(33, 17)
    a = run_pair(seq, precision, 2)
    blob = a.save_state()
    p = pv.params(precision=precision, kf_interval=0, sigma_P=seq.sigma_P, topology=pv.TOPOLOGY_QUADTREE)
    b = pv.Tracker(seq.cam.as_tuple(), p, DEV)
    b.load_state(blob)
    assert b.save_state() == blob
    for t in (a, b):
        t.sweep(3)
    va, vb = a.state(), b.state()
    assert a.status() == 0 and b.status() == 0
    assert np.array_equal(va.planes, vb.planes) and np.array_equal(va.nodes, vb.nodes)
    assert np.abs(va.nodes).max() > 0


def test_grid_checkpoint_holds_no_nodes():
    seq = sequence(16, 12)
    trk = pv.Tracker(seq.cam.as_tuple(), pv.params(kf_interval=0, sigma_P=seq.sigma_P), DEV)
    trk.track(torch.from_numpy(seq.frame(0)).to(DEV), torch.from_numpy(seq.normals(0)).to(DEV))
    assert trk.state().nodes is None


@pytest.mark.parametrize("size", SIZES)
def test_fp32_pose_matches_the_quadtree_oracle(size):
    seq = sequence(*size)
    st, _ = oracle_pair(seq, 3)
    trk = run_pair(seq, 32, 3)
    assert trk.status() == 0
    assert np.abs(trk.pose() - gbp.pose_estimate(st.pixels.mu)).max() < 1e-4


def test_grid_and_quadtree_differ():
    """The topology switch changes the computation (the identity slots 1..3 of a
    quadtree pixel stay empty, those of a grid pixel do not)."""
    seq = sequence(16, 12)
    q = run_pair(seq, 64, 2).state()
    p = pv.params(precision=64, kf_interval=0, sigma_P=seq.sigma_P)
    trk = pv.Tracker(seq.cam.as_tuple(), p, DEV)
    trk.track(torch.from_numpy(seq.frame(0)).to(DEV), torch.from_numpy(seq.normals(0)).to(DEV))
    trk.track(torch.from_numpy(seq.frame(1)).to(DEV), n_iters=2)
    g = trk.state()
    idq, idg = q.identity_messages, g.identity_messages
    assert np.all(idq[..., 1:4, :] == 0.0)
    assert np.any(idg[..., 1:4, :] != 0.0)
    assert np.abs(q.mu - g.mu).max() > 1e-8


def test_quadtree_refusals():
    seq = sequence(16, 12)
    trk = run_pair(seq, 32, 1)
    blob = trk.save_state()
    import ctypes
    # a grid handle of the same image takes no quadtree checkpoint, nor the reverse
    g = pv.Tracker(seq.cam.as_tuple(), pv.params(kf_interval=0), DEV)
    buf = ctypes.create_string_buffer(blob, len(blob))
    assert pv.lib.pixvod_load_state(g._h, buf, len(blob)) == pv.EINVAL
    gb = g.save_state()
    assert pv.lib.pixvod_load_state(trk._h, ctypes.create_string_buffer(gb, len(gb)), len(gb)) == pv.EINVAL
    bad = bytearray(blob)
    bad[12 * 8] ^= 1    # node count
    assert pv.lib.pixvod_load_state(trk._h, ctypes.create_string_buffer(bytes(bad), len(bad)), len(bad)) == pv.EINVAL
    z = torch.zeros(1 << 20, dtype=torch.uint8, device=DEV)
    assert pv.lib.pixvod_set_recording(trk._h, (z.data_ptr() + 255) // 256 * 256, 1 << 19, 5, 1) == pv.ESTATE
    K = pv.intrinsics(*seq.cam.as_tuple())
    arr = (pv.pixvod_intrinsics * 1)(K)
    need = ctypes.c_size_t(0)
    p = pv.params(topology=pv.TOPOLOGY_QUADTREE)
    assert pv.lib.pixvod_batch_workspace_bytes(1, ctypes.cast(arr, ctypes.c_void_p), ctypes.byref(p),
                                               ctypes.byref(need)) == pv.OK  # batches take quadtree sequences
    bad = pv.params(topology=2)
    assert pv.lib.pixvod_workspace_bytes(ctypes.byref(K), ctypes.byref(bad), ctypes.byref(need)) == pv.EINVAL


# Batches of quadtree sequences (different image sizes, keyframes): the plain
# schedule and the batched one (one launch of each quadtree kernel per sweep for
# all sequences) reproduce every sequence tracked alone bit for bit; the single
# quadtree handle is checked against the oracle above. The persistent schedule
# is refused (a quadtree sweep is three dependent launches).
QT_SIZES = [(70, 45), (64, 48), (33, 17), (96, 64)]
QT_FRAMES, QT_SWEEPS, QT_KF = 4, 3, 3


def qt_batch_params(prec):
    return pv.params(precision=prec, kf_interval=QT_KF, sigma_P=0.05, topology=pv.TOPOLOGY_QUADTREE)


@pytest.fixture(scope="module")
def qt_seqs():
    out = []
    for i, (w, h) in enumerate(QT_SIZES):
        s = synth.realistic(60 + i, QT_FRAMES, w, h)
        out.append((s, [torch.from_numpy(s.frame(k)).to(DEV) for k in range(QT_FRAMES)],
                    [torch.from_numpy(s.normals(k)).to(DEV) for k in range(QT_FRAMES)]))
    return out


@pytest.mark.parametrize("prec", [32, 64])
def test_quadtree_batch_matches_sequences_tracked_alone_bitwise(qt_seqs, prec):
    ref_blobs, ref_poses = [], []
    for s, frames, normals in qt_seqs:
        trk = pv.Tracker(s.cam.as_tuple(), qt_batch_params(prec), DEV)
        for k in range(QT_FRAMES):
            trk.track(frames[k], normals[k] if k % QT_KF == 0 else None, n_iters=QT_SWEEPS)
        ref_blobs.append(trk.save_state())
        ref_poses.append(trk.pose())
    for sched in (pv.SCHED_PLAIN, pv.SCHED_BATCHED):
        b = pv.Batch([s.cam.as_tuple() for s, _, _ in qt_seqs], qt_batch_params(prec), DEV)
        assert b.schedule()[0] == pv.SCHED_BATCHED  # the default for quadtree sequences
        b.set_schedule(sched)
        with pytest.raises(pv.PixvodError):
            b.set_schedule(pv.SCHED_PERSISTENT, 2)
        for k in range(QT_FRAMES):
            b.set_inputs([f[k] for _, f, _ in qt_seqs], [n[k] for _, _, n in qt_seqs])
            b.track(QT_SWEEPS)
        assert b.status() == 0
        for i in range(len(qt_seqs)):
            assert b.save_state(i) == ref_blobs[i], (pv.SCHED_NAMES[sched], i)
        assert np.array_equal(b.poses(), np.stack(ref_poses))


def test_quadtree_batch_autotune_keeps_results(qt_seqs):
    ref = pv.Batch([s.cam.as_tuple() for s, _, _ in qt_seqs], qt_batch_params(32), DEV)
    tuned = pv.Batch([s.cam.as_tuple() for s, _, _ in qt_seqs], qt_batch_params(32), DEV)
    for k in range(QT_FRAMES):
        for b in (ref, tuned):
            b.set_inputs([f[k] for _, f, _ in qt_seqs], [n[k] for _, _, n in qt_seqs])
            b.track(QT_SWEEPS)
        if k == 0:
            times, (sched, _) = tuned.autotune(QT_SWEEPS, 1)
            assert times["plain"] > 0 and times["batched"] > 0
            assert times["persistent2"] < 0 and times["persistent4"] < 0  # not candidates
            assert sched in (pv.SCHED_PLAIN, pv.SCHED_BATCHED)
    for i in range(len(qt_seqs)):
        assert tuned.save_state(i) == ref.save_state(i), i
