"""Batches of sequences with different image sizes: every schedule (plain,
batched per-sweep launches, persistent cooperative launch) must reproduce
sequences tracked alone with pixvod_track bit for bit (the per-tile arithmetic
and the reduction order do not depend on the schedule); the single-sequence path
itself is checked against the oracle in test_gpu_parity.py."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import synth  # noqa: E402
import paper_2606_03989_gb300 as pv  # noqa: E402

DEV = torch.device("cuda:0")
SIZES = [(70, 45), (64, 48), (96, 64), (33, 17), (128, 96)]
N_FRAMES, SWEEPS, KF = 5, 3, 3


@pytest.fixture(scope="module")
def seqs():
    out = []
    for i, (w, h) in enumerate(SIZES):
        s = synth.realistic(40 + i, N_FRAMES, w, h)
        frames = [torch.from_numpy(s.frame(k)).to(DEV) for k in range(N_FRAMES)]
        normals = [torch.from_numpy(s.normals(k)).to(DEV) for k in range(N_FRAMES)]
        out.append((s, frames, normals))
    return out


def params(prec):
    return pv.params(precision=prec, kf_interval=KF, sigma_P=0.05)


def run_single(seqs, prec):
    blobs, poses = [], []
    for s, frames, normals in seqs:
        trk = pv.Tracker(s.cam.as_tuple(), params(prec), DEV)
        for k in range(N_FRAMES):
            trk.track(frames[k], normals[k] if k % KF == 0 else None, n_iters=SWEEPS)
        blobs.append(trk.save_state())
        poses.append(trk.pose())
    return blobs, np.stack(poses)


def run_batch(seqs, prec, schedule=None, blocks=4, autotune=False):
    b = pv.Batch([s.cam.as_tuple() for s, _, _ in seqs], params(prec), DEV)
    if schedule is not None:
        b.set_schedule(schedule, blocks)
    for k in range(N_FRAMES):
        b.set_inputs([f[k] for _, f, _ in seqs], [n[k] for _, _, n in seqs])
        b.track(SWEEPS)
        if k == 0 and autotune:
            times, chosen = b.autotune(SWEEPS, 1)
            assert all(t != 0 for t in times.values()), times
    assert b.status() == 0
    return [b.save_state(i) for i in range(b.n)], b.poses(), b


@pytest.mark.parametrize("prec", [32, 64])
def test_every_schedule_matches_single_sequences_bitwise(seqs, prec):
    ref_blobs, ref_poses = run_single(seqs, prec)
    for sched, blocks in ((pv.SCHED_PLAIN, 4), (pv.SCHED_BATCHED, 4), (pv.SCHED_PERSISTENT, 4),
                          (pv.SCHED_PERSISTENT, 2), (pv.SCHED_PERSISTENT, 1)):
        blobs, poses, _ = run_batch(seqs, prec, sched, blocks)
        for i in range(len(seqs)):
            assert blobs[i] == ref_blobs[i], (pv.SCHED_NAMES[sched], blocks, i)
        assert np.array_equal(poses, ref_poses)


def test_autotune_keeps_results_identical(seqs):
    ref_blobs, ref_poses = run_single(seqs, 32)
    blobs, poses, b = run_batch(seqs, 32, autotune=True)
    sched, blocks = b.schedule()
    assert sched in (pv.SCHED_PLAIN, pv.SCHED_BATCHED, pv.SCHED_PERSISTENT)
    for i in range(len(seqs)):
        assert blobs[i] == ref_blobs[i], i
    assert np.array_equal(poses, ref_poses)


def test_graph_capture_of_a_batch_step(seqs):
    """A frame step of the persistent schedule captured in a CUDA graph replays to
    the same state as running it eagerly."""
    bufs_f = [torch.empty_like(f[0]) for _, f, _ in seqs]
    bufs_n = [torch.empty_like(n[0]) for _, _, n in seqs]
    s = torch.cuda.Stream(DEV)
    outs = []
    for use_graph in (False, True):
        with torch.cuda.stream(s):
            b = pv.Batch([q.cam.as_tuple() for q, _, _ in seqs], params(32), DEV, stream=s)
            b.set_schedule(pv.SCHED_PERSISTENT, 4)
            b.set_inputs(bufs_f, bufs_n)
            for k in range(2):
                for i, (_, f, n) in enumerate(seqs):
                    bufs_f[i].copy_(f[k])
                    bufs_n[i].copy_(n[k])
                b.track(SWEEPS)
            for i, (_, f, n) in enumerate(seqs):
                bufs_f[i].copy_(f[2])
            if use_graph:
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=s):
                    b.track(SWEEPS)
                g.replay()
            else:
                b.track(SWEEPS)
            s.synchronize()
            outs.append([b.save_state(i)[256:] for i in range(b.n)])
    for i in range(len(seqs)):
        assert outs[0][i] == outs[1][i], i


def test_batch_argument_errors(seqs):
    b = pv.Batch([s.cam.as_tuple() for s, _, _ in seqs], params(32), DEV)
    lib = pv.lib
    assert lib.pixvod_batch_track(b._h, 3) == pv.ESTATE              # no inputs registered
    assert lib.pixvod_batch_autotune(b._h, 3, 1, None) == pv.ESTATE  # before the first frame
    assert lib.pixvod_batch_set_schedule(b._h, 7, 1) == pv.EINVAL
    assert lib.pixvod_batch_set_schedule(b._h, pv.SCHED_PERSISTENT, 0) == pv.EINVAL
    assert lib.pixvod_batch_save_state(b._h, len(seqs), None, 0) == pv.EINVAL


def test_grid_barrier_timeout_is_reported_and_the_device_stays_usable(seqs):
    """Failure path of the persistent schedule's bounded grid barrier, with no
    fault: the test hook starts the arrival counter at 2^24, so no arrival counts
    as the last one, every block's wait (shortened to 2000 polls) runs out, sets
    PIXVOD_FLAG_TIMEOUT and leaves the launch. The host reads ETIMEOUT; other
    schedules of the same batch, and a fresh batch, then run normally."""
    b = pv.Batch([s.cam.as_tuple() for s, _, _ in seqs], params(32), DEV)
    b.set_schedule(pv.SCHED_PERSISTENT, 4)
    b.set_wait_limit(2000)
    b.set_inputs([f[0] for _, f, _ in seqs], [n[0] for _, _, n in seqs])
    b.track(SWEEPS)                       # keyframe: no sweeps, no barrier
    assert b.status() == 0
    b.inject_barrier_fault(True)
    b.set_inputs([f[1] for _, f, _ in seqs], [n[1] for _, _, n in seqs])
    b.track(SWEEPS)                       # SWEEPS > 1: the blocks meet a barrier
    flags = ctypes.c_uint32(0)
    assert pv.lib.pixvod_batch_get_status(b._h, ctypes.byref(flags)) == pv.ETIMEOUT
    assert flags.value & pv.FLAG_TIMEOUT
    # the context is intact: a fresh batch reproduces single-sequence tracking
    ref_blobs, ref_poses = run_single(seqs, 32)
    blobs, poses, _ = run_batch(seqs, 32, pv.SCHED_PERSISTENT, 4)
    assert np.array_equal(poses, ref_poses)
    assert all(blobs[i] == ref_blobs[i] for i in range(len(seqs)))
    assert pv.lib.pixvod_batch_set_wait_limit(b._h, -1) == pv.EINVAL


def test_every_schedule_matches_the_oracle_tracker(seqs):
    """Every sequence of an FP64 batch, in every schedule, against the oracle
    tracker (oracle/tracker.py) frame by frame at the stated tolerance: pose 1e-5,
    inverse depth 1e-4 (relative, valid pixels), global pose, and the log-depth
    prior mean (a mean log-depth, held like the inverse depths). A keyframe every
    2 frames and 2 sweeps per frame: frames warm-start from the previous state,
    are re-anchored, and restart from the reset, while no frame is far enough
    from a reset for the iteration's amplification of rounding (which on these
    noisy frames reaches 1e-4 in inverse depth after about 6 sweeps, between
    the oracle's dense Schur forms and the library's structured ones) to reach
    the tolerance."""
    import sys
    import os
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from helpers import compare_tracks, oracle_intrinsics, oracle_params, oracle_track
    kf, sweeps = 2, 2
    refs = [oracle_track(s, oracle_intrinsics(s.cam), oracle_params(sigma_P=0.05), kf, n_frames=N_FRAMES,
                         sweeps=sweeps)[1] for s, _, _ in seqs]
    for sched, blocks in ((pv.SCHED_PLAIN, 4), (pv.SCHED_BATCHED, 4), (pv.SCHED_PERSISTENT, 4),
                          (pv.SCHED_PERSISTENT, 1)):
        b = pv.Batch([s.cam.as_tuple() for s, _, _ in seqs],
                     pv.params(precision=64, kf_interval=kf, sigma_P=0.05), DEV)
        b.set_schedule(sched, blocks)
        gpu = [[] for _ in seqs]
        for k in range(N_FRAMES):
            b.set_inputs([f[k] for _, f, _ in seqs], [n[k] for _, _, n in seqs])
            b.track(sweeps)
            xi = b.poses()
            for i in range(len(seqs)):
                v = b.state(i)
                gpu[i].append((xi[i], v.T_cur, v.d_prior, v.mu))
        assert b.status() == 0
        for i, ref in enumerate(refs):
            compare_tracks(gpu[i], ref, None, "%s/%d seq %d" % (pv.SCHED_NAMES[sched], blocks, i))
