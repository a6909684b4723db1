"""Adjoint of the unrolled sweeps of one frame (pixvod_backward) against central
finite differences of the FP64 oracle: gradients of
    L = |xi_est - xi_gt|^2 + mean_px (exp(-mu_6) - 1/z_gt)^2
with respect to sigma_D, sigma_N and the keyframe / target intensities, for a
16 x 12 realistic pair tracked with 5 sweeps (checkpoints every 2 sweeps, so
the recompute runs segments of 2, 2 and 1 sweeps). Tolerance: relative error
1e-3, the bound the derivative is specified to.

The iteration is very sensitive (the loss moves by ~4e3 relative per relative
change of sigma_D but ~0.07 per relative change of sigma_N), so no single
difference step suits every input: small steps drown in the rounding noise of
the FP64 trajectory, large ones in its curvature. Each finite difference is
therefore taken over a ladder of steps, and the value used is the best-agreeing
adjacent pair (the plateau), which must itself agree to 2e-3."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import synth  # noqa: E402
import paper_2606_03989_gb300 as pv  # noqa: E402
from oracle import gbp, lie  # noqa: E402
from oracle import tracker as otr  # noqa: E402
from helpers import f32, oracle_intrinsics  # noqa: E402

DEV = torch.device("cuda:0")
W, H, SWEEPS, EVERY = 16, 12, 5, 2
RTOL = 1e-3


@pytest.fixture(scope="module")
def case():
    seq = synth.realistic(5, 2, W, H)
    T = seq.relative_pose(0, 1)
    xi_gt = lie.se3_log(T[:3, :3], T[:3, 3])
    inv_gt = 1.0 / seq.depth(0)
    return {"seq": seq, "I_s": seq.frame(0), "I_t": seq.frame(1), "n": seq.normals(0),
            "xi_gt": xi_gt, "inv_gt": inv_gt}


def loss(c, xi, inv):
    return float(np.sum((xi - c["xi_gt"]) ** 2) + np.mean((inv - c["inv_gt"]) ** 2))


def oracle_params(seq, sigma_D=None, sigma_N=None):
    """The GPU's float32 parameters; sigma_D / sigma_N may be given unrounded."""
    p = pv.params_default()
    return gbp.Params(sigma_D=f32(p.sigma_D) if sigma_D is None else sigma_D, sigma_P=f32(seq.sigma_P),
                      sigma_R=f32(p.sigma_R), sigma_N=f32(p.sigma_N) if sigma_N is None else sigma_N,
                      sigma_Z=f32(p.sigma_Z), t_huber=f32(p.t_huber), damping=f32(p.damping))


def oracle_loss(c, I_s=None, I_t=None, **sig):
    seq = c["seq"]
    trk = otr.Tracker(oracle_intrinsics(seq.cam), oracle_params(seq, **sig), kf_interval=0)
    trk.track(np.asarray(c["I_s"] if I_s is None else I_s, np.float64), c["n"])
    xi = trk.track(np.asarray(c["I_t"] if I_t is None else I_t, np.float64), n_iters=SWEEPS)
    return loss(c, xi, np.exp(-trk.state.mu[..., 6]))


def gpu_run(c, precision=64, window=None, method=0, every=EVERY):
    seq = c["seq"]
    trk = pv.Tracker(seq.cam.as_tuple(), pv.params(precision=precision, kf_interval=0, sigma_P=seq.sigma_P), DEV)
    trk.set_recording(SWEEPS, every, method)
    if window is not None:
        trk.set_backward_window(window)
    trk.track(torch.from_numpy(c["I_s"]).to(DEV), torch.from_numpy(c["n"]).to(DEV))
    trk.track(torch.from_numpy(c["I_t"]).to(DEV), n_iters=SWEEPS)
    xi = trk.pose()
    inv = np.exp(-trk.state().mu[..., 6])   # the mean in the state's own precision
    g = trk.backward(2.0 * (xi - c["xi_gt"]), 2.0 * (inv - c["inv_gt"]) / inv.size)
    return trk, xi, inv, g


@pytest.fixture(scope="module")
def gpu64(case):
    return gpu_run(case, 64)


@pytest.fixture(scope="module")
def gpu64_tape(case):
    return gpu_run(case, 64, method=pv.ADJOINT_TAPE)


def central(f, x0, h):
    return (f(x0 + h) - f(x0 - h)) / (2.0 * h)


STEPS = [3e-3, 1e-3, 3e-4, 1e-4, 3e-5, 1e-5, 3e-6, 1e-6, 3e-7, 1e-7]


def plateau(f, x0, unit):
    """Central differences of f at x0 over steps unit * STEPS; the mean of the
    adjacent pair that agrees best, which must agree to 2e-3."""
    d = [central(f, x0, unit * h) for h in STEPS]
    spread = [abs(a - b) / max(abs(a), abs(b), 1e-300) for a, b in zip(d, d[1:])]
    k = int(np.argmin(spread))
    assert spread[k] <= 2e-3, (d, spread)
    return 0.5 * (d[k] + d[k + 1])


def assert_close(g, fd, scale):
    assert abs(g - fd) <= RTOL * max(abs(fd), scale), (g, fd, scale)


@pytest.mark.parametrize("precision", [64, 32])
def test_keeping_every_state_needs_no_recomputation(case, precision, gpu64):
    """checkpoint_every = 1: the frame's sweeps write every intermediate state
    and every sweep's decisions, and the reverse pass recomputes nothing. The
    tracked frame is bit-identical to the checkpointed run's (the same kernel on
    other buffers), the recompute check sees the same states, and in FP64 the
    gradients equal the checkpointed run's (to the order of the atomic sums)."""
    t1, xi1, inv1, g1 = gpu_run(case, precision, every=1)
    t5, xi5, inv5, g5 = gpu64 if precision == 64 else gpu_run(case, precision)
    assert np.array_equal(xi1, xi5) and np.array_equal(inv1, inv5)
    assert g1["status"] == pv.OK
    assert g1["recompute_mismatch"] == g5["recompute_mismatch"]
    if precision == 64:
        for k in ("sigma_D", "sigma_N"):
            assert float(g1[k]) == pytest.approx(float(g5[k]), rel=1e-9), k
        for k in ("I_s", "I_t"):
            err = float((g1[k] - g5[k]).norm() / g5[k].norm())
            assert err < 1e-9, (k, err)
    # the reverse pass launches no sweep kernel
    assert t1.launch_count() < t5.launch_count()


def test_recomputed_update_equals_the_sweep_kernel(gpu64, gpu64_tape):
    """Both reverse passes' own FP64 recomputation of every pixel update matches
    the sweep kernel's result, so they differentiate the function that ran."""
    for _, _, _, g in (gpu64, gpu64_tape):
        assert g["status"] == pv.OK
        assert g["recompute_mismatch"] < 1e-9, g["recompute_mismatch"]
    assert gpu64[3]["tape_nodes"] == 0
    assert 1000 < gpu64_tape[3]["tape_nodes"] < 8192


def test_hand_written_adjoint_equals_the_tape(gpu64, gpu64_tape):
    """The hand-written reverse pass and the FP64 tape of the same update give the
    same gradients, element by element, to FP64 rounding."""
    g, gt = gpu64[3], gpu64_tape[3]
    for k in ("sigma_D", "sigma_N"):
        assert float(g[k]) == pytest.approx(float(gt[k]), rel=1e-9), k
    for k in ("I_s", "I_t"):
        a, b = g[k].cpu().numpy(), gt[k].cpu().numpy()
        err = np.abs(a - b).max() / np.abs(b).max()
        print("\nhand-written vs tape, dL/d%s: normwise %.1e" % (k, err))
        assert err < 1e-9, (k, err)


def test_loss_matches_the_oracle(case, gpu64):
    _, xi, inv, _ = gpu64
    assert loss(case, xi, inv) == pytest.approx(oracle_loss(case), rel=1e-9)


def test_sigma_gradients_match_oracle_finite_differences(case, gpu64):
    _, _, _, g = gpu64
    p = pv.params_default()
    sD, sN = f32(p.sigma_D), f32(p.sigma_N)
    fd_D = plateau(lambda s: oracle_loss(case, sigma_D=s), sD, sD)
    fd_N = plateau(lambda s: oracle_loss(case, sigma_N=s), sN, sN)
    assert fd_D != 0.0 and fd_N != 0.0
    assert_close(float(g["sigma_D"]), fd_D, 0.0)
    assert_close(float(g["sigma_N"]), fd_N, 0.0)


def test_intensity_gradients_match_oracle_finite_differences(case, gpu64):
    _, _, _, g = gpu64
    rng = np.random.default_rng(11)
    pix = [(int(rng.integers(1, H - 1)), int(rng.integers(1, W - 1))) for _ in range(3)]
    for name in ("I_s", "I_t"):
        gg = g[name].cpu().numpy()
        fds = []
        for (v, u) in pix:
            def f(x, v=v, u=u):
                img = case[name].astype(np.float64).copy()
                img[v, u] = x
                return oracle_loss(case, **{name: img})
            fds.append(plateau(f, float(case[name][v, u]), 1.0))
        scale = 1e-2 * max(abs(x) for x in fds)
        assert scale > 0.0
        for (v, u), fd in zip(pix, fds):
            assert_close(float(gg[v, u]), fd, scale)


def test_autograd_function_gives_the_backward_gradients(case, gpu64):
    seq = case["seq"]
    trk = pv.Tracker(seq.cam.as_tuple(), pv.params(precision=64, kf_interval=0, sigma_P=seq.sigma_P), DEV)
    kf = torch.from_numpy(case["I_s"]).to(DEV).requires_grad_(True)
    fr = torch.from_numpy(case["I_t"]).to(DEV).requires_grad_(True)
    p = pv.params_default()
    sD = torch.tensor(f32(p.sigma_D), dtype=torch.float64, requires_grad=True)
    sN = torch.tensor(f32(p.sigma_N), dtype=torch.float64, requires_grad=True)
    trk.set_recording(SWEEPS, EVERY)
    trk.track(kf.detach(), torch.from_numpy(case["n"]).to(DEV))
    xi, inv = pv.track_frame(trk, fr, kf, sD, sN, SWEEPS)
    xi_gt = torch.as_tensor(case["xi_gt"], device=DEV)
    inv_gt = torch.as_tensor(case["inv_gt"], device=DEV)
    L = ((xi - xi_gt) ** 2).sum() + ((inv - inv_gt) ** 2).mean()
    L.backward()
    _, _, _, g = gpu64
    assert float(L) == pytest.approx(loss(case, *gpu64[1:3]), rel=1e-6)
    assert float(sD.grad) == pytest.approx(float(g["sigma_D"]), rel=1e-5)
    assert float(sN.grad) == pytest.approx(float(g["sigma_N"]), rel=1e-5)
    assert torch.allclose(kf.grad.double(), g["I_s"], rtol=1e-5, atol=1e-9 * float(g["I_s"].abs().max()))
    assert torch.allclose(fr.grad.double(), g["I_t"], rtol=1e-5, atol=1e-9 * float(g["I_t"].abs().max()))


def test_fp32_state_gives_close_gradients(case, gpu64):
    """FP32 forward and FP32 hand-written reverse pass on the realistic pair: the
    reverse pass's recomputation of every update is within the documented FP32
    bound of the sweep kernel's, and the gradients are close to the FP64 ones
    (the 5 sweeps amplify the FP32 rounding of the trajectory)."""
    _, _, _, g64 = gpu64
    _, _, _, g32 = gpu_run(case, 32)
    print("\nFP32 recompute mismatch %.1e; sigma_D %.4e vs %.4e, sigma_N %.4e vs %.4e"
          % (g32["recompute_mismatch"], float(g32["sigma_D"]), float(g64["sigma_D"]), float(g32["sigma_N"]),
             float(g64["sigma_N"])))
    assert g32["status"] == pv.OK
    assert g32["recompute_mismatch"] < 1e-2
    for k in ("sigma_D", "sigma_N"):
        assert np.isfinite(float(g32[k]))
        assert float(g32[k]) == pytest.approx(float(g64[k]), rel=0.1)


def test_fp32_adjoint_on_a_contracting_input():
    """On the exactly bilinear pair (64x48 tiny camera, 20 sweeps), where the
    iteration contracts, the FP32 reverse pass gives the FP64 gradients."""
    seq = synth.tiny_pair(0)
    aff = synth.affine_pair(seq)
    I_s, I_t, n = (aff["I_s"].astype(np.float32), aff["I_t"].astype(np.float32),
                   aff["normal"].astype(np.float32))
    xi_gt = lie.se3_log(aff["T_ts"][:3, :3], aff["T_ts"][:3, 3])
    inv_gt = 1.0 / aff["depth"]
    out = {}
    for prec in (64, 32):
        trk = pv.Tracker(seq.cam.as_tuple(), pv.params(precision=prec, kf_interval=0, sigma_P=seq.sigma_P), DEV)
        trk.set_recording(20, 5)
        trk.track(torch.from_numpy(I_s).to(DEV), torch.from_numpy(n).to(DEV))
        trk.track(torch.from_numpy(I_t).to(DEV), n_iters=20)
        xi = trk.pose()
        inv = np.exp(-trk.state().mu[..., 6])
        out[prec] = trk.backward(2.0 * (xi - xi_gt), 2.0 * (inv - inv_gt) / inv.size)
        assert out[prec]["status"] == pv.OK
    for k in ("sigma_D", "sigma_N"):
        a, b = float(out[32][k]), float(out[64][k])
        print("\nbilinear pair, FP32 vs FP64 dL/d%s: %.6e vs %.6e (rel %.1e)" % (k, a, b, abs(a - b) / abs(b)))
        assert a == pytest.approx(b, rel=1e-3), k
    for k in ("I_s", "I_t"):
        a, b = out[32][k].cpu().numpy(), out[64][k].cpu().numpy()
        err = np.abs(a - b).max() / np.abs(b).max()
        print("bilinear pair, FP32 vs FP64 dL/d%s: normwise %.1e" % (k, err))
        assert err < 1e-3, (k, err)


def test_reverse_pass_follows_the_forward_at_the_adjoint_workload_size():
    """320x240 frame of the adjoint workload family (30 sweeps, checkpoints every
    5), with the forward's recorded decisions. FP64: the reverse pass's
    recomputation of every pixel update equals the sweep kernel's result to FP64
    rounding, so it differentiates the update that ran (no validity or Huber
    branch taken differently, which would show as an O(1) difference). FP32: the
    same recomputation in float differs from the float sweep only by rounding
    (4.6e-4 measured, each output relative to the terms it is formed from and
    to its block's scale); the status stays OK under the documented bound."""
    seq = synth.adjoint_family(1, 2)[0]
    for prec, tol in ((64, 1e-9), (32, 2e-3)):
        trk = pv.Tracker(seq.cam.as_tuple(), pv.params(precision=prec, kf_interval=0, sigma_P=seq.sigma_P), DEV)
        trk.set_recording(30, 5)
        trk.track(torch.from_numpy(seq.frame(0)).to(DEV), torch.from_numpy(seq.normals(0)).to(DEV))
        trk.track(torch.from_numpy(seq.frame(1)).to(DEV), n_iters=30)
        g = trk.backward(np.ones(6), None)
        print("\n320x240 FP%d recompute mismatch %.1e" % (prec, g["recompute_mismatch"]))
        assert g["status"] == pv.OK
        assert g["recompute_mismatch"] < tol
        assert np.isfinite(float(g["sigma_D"])) and np.isfinite(float(g["sigma_N"]))


def oracle_loss_window(c, w, I_s=None, I_t=None, **sig):
    """The loss with the perturbed inputs used in the last w sweeps only (the first
    SWEEPS - w sweeps run with the base inputs): what a backward window of w
    sweeps differentiates."""
    seq = c["seq"]
    K = oracle_intrinsics(seq.cam)
    base, pert = oracle_params(seq), oracle_params(seq, **sig)
    f64 = lambda x: np.asarray(x, np.float64)
    win0 = gbp.make_window(K, f64(c["I_s"]), c["n"], f64(c["I_t"]), 0.0)
    win1 = gbp.make_window(K, f64(c["I_s"] if I_s is None else I_s), c["n"], f64(c["I_t"] if I_t is None else I_t), 0.0)
    st = gbp.reset_state(win0.shape, 0.0, base)
    for _ in range(SWEEPS - w):
        st = gbp.sweep(win0, st, base)
    for _ in range(w):
        st = gbp.sweep(win1, st, pert)
    return loss(c, gbp.pose_estimate(st.mu), np.exp(-st.mu[..., 6]))


@pytest.mark.parametrize("w", [1, 2])
def test_backward_window_matches_finite_differences_of_the_last_sweeps(case, w):
    _, _, _, g = gpu_run(case, 64, window=w)
    p = pv.params_default()
    sD, sN = f32(p.sigma_D), f32(p.sigma_N)
    assert_close(float(g["sigma_D"]), plateau(lambda s: oracle_loss_window(case, w, sigma_D=s), sD, sD), 0.0)
    assert_close(float(g["sigma_N"]), plateau(lambda s: oracle_loss_window(case, w, sigma_N=s), sN, sN), 0.0)
    v, u = 5, 7
    for name in ("I_s", "I_t"):
        def f(x):
            img = case[name].astype(np.float64).copy()
            img[v, u] = x
            return oracle_loss_window(case, w, **{name: img})
        fd = plateau(f, float(case[name][v, u]), 1.0)
        assert_close(float(g[name][v, u]), fd, 1e-2 * abs(fd) + 1e-12)


def test_window_covering_every_sweep_is_the_full_derivative(case, gpu64):
    _, _, _, g = gpu64
    for w in (0, SWEEPS, SWEEPS + 3):
        _, _, _, gw = gpu_run(case, 64, window=w)
        for k in ("sigma_D", "sigma_N"):
            assert float(gw[k]) == pytest.approx(float(g[k]), rel=1e-10)
        assert torch.allclose(gw["I_t"], g["I_t"], rtol=1e-10, atol=1e-12 * float(g["I_t"].abs().max()))


def test_backward_needs_a_recorded_frame(case):
    seq = case["seq"]
    trk = pv.Tracker(seq.cam.as_tuple(), pv.params(precision=64, kf_interval=2, sigma_P=seq.sigma_P), DEV)
    lib = pv.lib
    z = torch.zeros(H * W + 8, dtype=torch.float64, device=DEV)
    args = (None, None, z.data_ptr(), z.data_ptr(), z.data_ptr(), None)
    assert lib.pixvod_backward(trk._h, *args) == pv.ESTATE  # recording off
    trk.set_recording(SWEEPS, EVERY)
    I_s = torch.from_numpy(case["I_s"]).to(DEV)
    n = torch.from_numpy(case["n"]).to(DEV)
    trk.track(I_s, n)
    assert lib.pixvod_backward(trk._h, *args) == pv.ESTATE  # a keyframe, not a target
    with pytest.raises(pv.PixvodError):
        trk.track(torch.from_numpy(case["I_t"]).to(DEV), n_iters=SWEEPS + 1)  # more sweeps than recorded
    trk.track(torch.from_numpy(case["I_t"]).to(DEV), n_iters=SWEEPS)  # frame 1: a target
    assert lib.pixvod_backward(trk._h, *args) == pv.OK
    trk.track(I_s, n, n_iters=SWEEPS)  # frame 2 anchors a new keyframe
    assert lib.pixvod_backward(trk._h, *args) == pv.ESTATE
