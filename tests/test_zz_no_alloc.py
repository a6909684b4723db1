"""pixvod_pose_mean_static: the allocation-free pose average, for callers that
cannot allocate device memory (for example code running under stream capture,
or a real-time loop that forbids allocation after start-up).

Its output must equal what the existing entry points report for the same state:
the pose average from pixvod_get_pose and the mean log-depth stored in the
checkpoint by pixvod_save_state, on two calls in a row. This file is collected
last so that a run stopping at the first failure has run every other test; it
must pass alone in a fresh process as well as after the other tests.
"""
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


def _mu_planes_on_device(blob):
    """The 7 pose/log-depth planes of a checkpoint, uploaded with the checkpoint's
    own pitch and plane stride."""
    hd = np.frombuffer(blob, dtype="<i8", count=12)
    prec, W, H, pitch = (int(x) for x in hd[2:6])
    assert prec == 32
    planes = np.frombuffer(blob, dtype=np.float32, count=7 * H * pitch, offset=int(hd[8]))
    return torch.from_numpy(planes.copy()).to(DEV), W, H, pitch, H * pitch


def _call(d_mu, W, H, pitch, plane, out, stream):
    return pv.lib.pixvod_pose_mean_static(d_mu.data_ptr(), W, H, pitch, plane, out.data_ptr(),
                                          stream.cuda_stream)


def test_static_pose_mean_matches_the_tracker_reduction():
    seq = synth.realistic(3, 3, 160, 120)
    trk = pv.Tracker(seq.cam.as_tuple(), pv.params(kf_interval=0, sigma_P=seq.sigma_P), DEV)
    trk.track(torch.from_numpy(seq.frame(0)).to(DEV), torch.from_numpy(seq.normals(0)).to(DEV))
    trk.track(torch.from_numpy(seq.frame(1)).to(DEV), n_iters=4)
    xi = trk.pose()                                  # existing entry point
    blob = trk.save_state()
    d_mean = np.frombuffer(blob, dtype=np.float64, count=40, offset=int(np.frombuffer(
        blob, dtype="<i8", count=12)[9]))[39]          # mean log-depth of the last reduction
    d_mu, W, H, pitch, plane = _mu_planes_on_device(blob)
    stream = torch.cuda.current_stream(DEV)
    # the first call on a device resolves the scratch address (and may load the
    # library's module); memory is compared around the two calls that follow
    first = torch.full((7,), float("nan"), dtype=torch.float64, device=DEV)
    assert _call(d_mu, W, H, pitch, plane, first, stream) == pv.OK
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info(DEV)[0]
    outs = [first.cpu().numpy()]
    for _ in range(2):
        out = torch.full((7,), float("nan"), dtype=torch.float64, device=DEV)
        assert _call(d_mu, W, H, pitch, plane, out, stream) == pv.OK
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy())
    assert torch.cuda.mem_get_info(DEV)[0] == free_before
    for o in outs:
        np.testing.assert_allclose(o[:6], xi, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(o[6], d_mean, rtol=1e-12, atol=1e-15)
    np.testing.assert_array_equal(outs[1], outs[2])
    np.testing.assert_array_equal(outs[0], outs[1])


def test_static_pose_mean_rejects_out_of_range_arguments():
    d_mu = torch.zeros(7 * 8 * 8, dtype=torch.float32, device=DEV)
    out = torch.zeros(7, dtype=torch.float64, device=DEV)
    s = torch.cuda.current_stream(DEV)
    lib = pv.lib
    too_tall = pv.lib.pixvod_pose_mean_static(d_mu.data_ptr(), 8, 4097, 8, 8 * 4097, out.data_ptr(), s.cuda_stream)
    assert too_tall == pv.EINVAL
    assert lib.pixvod_pose_mean_static(None, 8, 8, 8, 64, out.data_ptr(), s.cuda_stream) == pv.EINVAL
    assert lib.pixvod_pose_mean_static(d_mu.data_ptr(), 8, 8, 4, 64, out.data_ptr(), s.cuda_stream) == pv.EINVAL
    assert lib.pixvod_pose_mean_static(d_mu.data_ptr(), 8, 8, 8, 32, out.data_ptr(), s.cuda_stream) == pv.EINVAL
    # a constant field averages to itself
    d_mu[:] = 0.25
    assert lib.pixvod_pose_mean_static(d_mu.data_ptr(), 8, 8, 8, 64, out.data_ptr(), s.cuda_stream) == pv.OK
    torch.cuda.synchronize()
    np.testing.assert_allclose(out.cpu().numpy(), 0.25, rtol=0, atol=1e-15)
