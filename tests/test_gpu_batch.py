"""Batches of sequences with different image sizes: every schedule (plain,
batched per-sweep launches, persistent cooperative launch) must reproduce
sequences tracked alone with pixvod_track bit for bit (the per-tile arithmetic
and the reduction order do not depend on the schedule); the single-sequence path
itself is checked against the oracle in test_gpu_parity.py."""
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
