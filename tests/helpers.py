"""Shared test utilities: running the oracle on the same inputs as the CUDA path,
and comparing the oracle's full 7x7 state with the library's compressed state
(checkpoint planes). Conversion goes through the documented checkpoint layout
only; nothing here calls into the CUDA path's internals."""
from __future__ import annotations

import numpy as np

from oracle import factors as fac
from oracle import gbp
from oracle.factors import Intrinsics
from oracle.gbp import Params

F32 = np.float32


def f32(x) -> float:
    """The value the C ABI receives for a float parameter."""
    return float(F32(x))


def oracle_intrinsics(cam) -> Intrinsics:
    fx, fy, cx, cy, w, h = cam.as_tuple()
    return Intrinsics(f32(fx), f32(fy), f32(cx), f32(cy), int(w), int(h))


def oracle_params(**kw) -> Params:
    """Oracle parameters rounded like the float32 fields of pixvod_params."""
    base = Params()
    vals = {k: f32(kw.get(k, getattr(base, k))) for k in
            ("sigma_D", "sigma_P", "sigma_R", "sigma_N", "sigma_Z", "t_huber", "damping")}
    return Params(**vals)


def gpu_params(pv, precision=32, kf_interval=10, **kw):
    return pv.params(precision=precision, kf_interval=kf_interval, **kw)


PACK6 = [(r, c) for r in range(6) for c in range(r + 1)]
N_PLANES, N_INPUT_PLANES = 151, 6


def pack6(M):
    return np.stack([M[..., r, c] for (r, c) in PACK6], -1)


def unpack6(v):
    M = np.zeros(v.shape[:-1] + (6, 6))
    for q, (r, c) in enumerate(PACK6):
        M[..., r, c] = v[..., q]
        M[..., c, r] = v[..., q]
    return M


def compressed_from_oracle(st: gbp.State, lam_P: float) -> dict:
    """Oracle state -> the fields the library stores (layout of include/pixvod.h):
    M_p = pose prior + identity-message pose blocks, P = depth-marginalised pose
    information of the belief (P - M_p is the rank-one photometric part, returned
    as u with u u^T = P - M_p), s = pose-marginalised depth information."""
    L = st.bel_L
    Lpp, Lpd, Ldd = L[..., :6, :6], L[..., :6, 6], L[..., 6, 6]
    P = Lpp - Lpd[..., :, None] * Lpd[..., None, :] / Ldd[..., None, None]
    s = Ldd - np.einsum("...i,...i->...", Lpd, np.linalg.solve(Lpp, Lpd[..., None])[..., 0])
    Mp = lam_P * np.eye(6) + st.msg_L[..., 0:4, :6, :6].sum(axis=-3)
    ev, evec = np.linalg.eigh(P - Mp)
    u = evec[..., :, -1] * np.sqrt(np.maximum(ev[..., -1], 0.0))[..., None]
    idm = np.concatenate([pack6(st.msg_L[..., 0:4, :6, :6]), st.msg_eta[..., 0:4, :6]], -1)
    nmm = np.stack([st.msg_L[..., 4:8, 6, 6], st.msg_eta[..., 4:8, 6]], -1)
    return {"mu": st.mu, "M_p": pack6(Mp), "u": u, "P": pack6(P), "s": s, "id": idm, "nm": nmm}


def compressed_from_view(view) -> dict:
    return {"mu": view.mu, "M_p": view.M_p, "u": view.u, "P": view.P, "s": view.s,
            "id": view.identity_messages, "nm": view.normal_messages}


def rounded(c: dict, precision: int) -> dict:
    """The same fields after a round trip through the checkpoint precision."""
    if precision == 64:
        return {k: np.array(v, dtype=np.float64) for k, v in c.items()}
    out = {k: np.asarray(v, np.float32).astype(np.float64) for k, v in c.items()}
    out["P"] = out["M_p"] + pack6(out["u"][..., :, None] * out["u"][..., None, :])
    return out


def oracle_state_from_compressed(c: dict, rows=slice(None), cols=slice(None)) -> gbp.State:
    """Compressed fields -> an oracle State that produces the same messages.

    The library keeps only the marginals P (pose) and s (depth) of each belief.
    A block-diagonal belief diag(P, s) with eta = 0 has exactly those marginals,
    and every variable-to-factor message the oracle forms from it (belief minus
    one message, then marginalised onto the factor's block) equals the one the
    library forms, so one oracle sweep from this state is the reference for one
    library sweep from the same fields."""
    P = np.asarray(c["P"])[rows, cols]
    sv = np.asarray(c["s"])[rows, cols]
    H, W = sv.shape
    bel = np.zeros((H, W, 7, 7))
    bel[..., :6, :6] = unpack6(P)
    bel[..., 6, 6] = sv
    idm = np.asarray(c["id"])[rows, cols]
    msg_L = np.zeros((H, W, 8, 7, 7))
    msg_eta = np.zeros((H, W, 8, 7))
    msg_L[..., 0:4, :6, :6] = unpack6(idm[..., :21])
    msg_eta[..., 0:4, :6] = idm[..., 21:27]
    nm = np.asarray(c["nm"])[rows, cols]
    msg_L[..., 4:8, 6, 6] = nm[..., 0]
    msg_eta[..., 4:8, 6] = nm[..., 1]
    return gbp.State(np.asarray(c["mu"])[rows, cols].copy(), bel, np.zeros((H, W, 7)), msg_L, msg_eta)


def input_planes(win: gbp.Window) -> list:
    """I_s, I_t, g_x, g_y, m_x, m_y as full-image planes (edge planes padded with 0)."""
    H, W = win.shape
    m_x = np.zeros((H, W))
    m_x[:, :-1] = win.m_x
    m_y = np.zeros((H, W))
    m_y[:-1, :] = win.m_y
    return [win.I_s, win.I_t, win.g_x, win.g_y, m_x, m_y]


def blob_from_compressed(c: dict, win: gbp.Window, precision: int, frame_index=2, d_prior=0.0) -> bytes:
    """A checkpoint (layout of include/pixvod.h) holding the given fields and the
    window's inputs, for pixvod_load_state."""
    H, W = np.asarray(c["s"]).shape
    pitch = (W + 31) // 32 * 32
    dt = np.float64 if precision == 64 else np.float32
    planes = np.zeros((N_PLANES + N_INPUT_PLANES, H, pitch), dt)
    fields = ([c["mu"][..., k] for k in range(7)] + [c["M_p"][..., k] for k in range(21)]
              + [c["u"][..., k] for k in range(6)] + [c["s"]]
              + [c["id"][..., k, q] for k in range(4) for q in range(27)]
              + [c["nm"][..., k, q] for k in range(4) for q in range(2)] + input_planes(win))
    for i, f in enumerate(fields):
        planes[i, :, :W] = f
    hd = np.zeros(32, "<i8")
    pb = H * pitch * planes.itemsize
    hd[:12] = [0x50495856, 1, precision, W, H, pitch, N_PLANES, frame_index, 256,
               256 + pb * (N_PLANES + N_INPUT_PLANES), N_INPUT_PLANES, 1]
    sc = np.zeros(40)
    sc[6:22] = np.eye(4).ravel()
    sc[22:38] = np.eye(4).ravel()
    sc[38] = d_prior
    return hd.tobytes() + planes.tobytes() + sc.tobytes()


def synthetic_state(H: int, W: int, p: Params, seed: int, xi0=None, logz=None) -> dict:
    """A seeded random GBP state with the magnitudes seen in tracking runs: pose
    means near xi0, log-depths near logz, identity messages with eigenvalues
    log-uniform between 1 and ~lam_R, normal messages up to ~lam_N, photometric
    marginals |u|^2 log-uniform up to 1e10, and M_p = prior + identity messages."""
    rng = np.random.default_rng(seed)
    lam_P, lam_R, lam_N, lam_Z = (1 / p.sigma_P ** 2, 1 / p.sigma_R ** 2, 1 / p.sigma_N ** 2,
                                  1 / p.sigma_Z ** 2)
    mu = np.zeros((H, W, 7))
    mu[..., :6] = (np.zeros(6) if xi0 is None else xi0) + 1e-3 * rng.normal(size=(H, W, 6))
    mu[..., 6] = (0.0 if logz is None else logz) + 0.05 * rng.normal(size=(H, W))
    Q = np.linalg.qr(rng.normal(size=(H, W, 4, 6, 6)))[0]
    ev = np.exp(rng.uniform(0, np.log(lam_R), size=(H, W, 4, 6)))
    L = Q @ (ev[..., :, None] * np.swapaxes(Q, -1, -2))
    eta = rng.normal(size=(H, W, 4, 6)) * np.sqrt(ev) * 1e-3
    idm = np.concatenate([pack6(L), eta], -1)
    n = np.exp(rng.uniform(0, np.log(lam_N), size=(H, W, 4)))
    nm = np.stack([n, rng.normal(size=(H, W, 4)) * np.sqrt(n) * 1e-2], -1)
    # no messages arrive from outside the image (slots 0 left, 1 right, 2 up, 3 down)
    out = np.zeros((H, W, 4), bool)
    out[:, 0, 0] = out[:, -1, 1] = out[0, :, 2] = out[-1, :, 3] = True
    L[out] = 0.0
    eta[out] = 0.0
    n[out] = 0.0
    idm = np.concatenate([pack6(L), eta], -1)
    nm = np.stack([n, rng.normal(size=(H, W, 4)) * np.sqrt(n) * 1e-2], -1)
    Mp = lam_P * np.eye(6) + L.sum(axis=-3)
    dirs = rng.normal(size=(H, W, 6))
    dirs /= np.linalg.norm(dirs, axis=-1, keepdims=True)
    u = dirs * np.exp(rng.uniform(0, np.log(1e5), size=(H, W)))[..., None]
    s = lam_Z + n.sum(-1) * rng.uniform(0.5, 1.5, size=(H, W))
    c = {"mu": mu, "M_p": pack6(Mp), "u": u, "s": s, "id": idm, "nm": nm}
    c["P"] = c["M_p"] + pack6(u[..., :, None] * u[..., None, :])
    return c


def oracle_sweep_at(c: dict, win: gbp.Window, p: Params, v: int, u: int):
    """One oracle sweep from compressed fields, evaluated at pixel (v, u) on the 3x3
    crop around it (a pixel's update depends on its 4-neighbourhood only).
    Returns the pixel's compressed fields and its tau."""
    H, W = np.asarray(c["s"]).shape
    v0, v1, u0, u1 = max(v - 1, 0), min(v + 2, H), max(u - 1, 0), min(u + 2, W)
    sub = gbp.Window(win.K, win.I_s[v0:v1, u0:u1], win.m_x[v0:v1, u0:u1 - 1], win.m_y[v0:v1 - 1, u0:u1],
                     win.I_t, win.g_x, win.g_y, u0, v0, win.d_prior)
    out = gbp.sweep(sub, oracle_state_from_compressed(c, slice(v0, v1), slice(u0, u1)), p)
    res = compressed_from_oracle(out, 1.0 / p.sigma_P ** 2)
    r, q = v - v0, u - u0
    return {k: np.asarray(x)[r, q] for k, x in res.items()}, out.diag["tau"][r, q]


def field_errors(gpu: dict, ora: dict) -> dict:
    """Normwise relative error per field: max |a - b| / max |b|."""
    out = {}
    for k in ("P", "M_p", "s", "id", "nm"):
        a, b = np.asarray(gpu[k]), np.asarray(ora[k])
        out[k] = float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
    out["mu_abs"] = float(np.abs(gpu["mu"] - ora["mu"]).max())
    return out


def inv_depth_rel_err(d_gpu, d_ora, mask=None):
    r = np.abs(np.exp(-(np.asarray(d_gpu) - np.asarray(d_ora))) - 1.0)
    if mask is not None:
        r = r[mask]
    return float(r.max()) if r.size else 0.0


def oracle_window(seq_or_imgs, K: Intrinsics, kf: int = 0, tgt: int = 1, d_prior=0.0):
    seq = seq_or_imgs
    I_s = seq.frame(kf).astype(np.float64)
    I_t = seq.frame(tgt).astype(np.float64)
    return gbp.make_window(K, I_s, seq.normals(kf).astype(np.float64), I_t, d_prior)


def run_oracle_pair(seq, K, p: Params, n_iters, record=()):
    """Keyframe frame 0, target frame 1, n_iters sweeps. Returns final state and
    the states after the sweep counts listed in ``record``."""
    win = oracle_window(seq, K)
    st = gbp.reset_state(win.shape, 0.0, p)
    rec = {}
    for k in range(1, n_iters + 1):
        st = gbp.sweep(win, st, p)
        if k in record:
            rec[k] = st
    return st, rec, win


def oracle_track(seq, K: Intrinsics, p: Params, kf: int, n_frames=None, eps: float = 0.0, sweeps=None):
    """The oracle tracker over frames 0..n_frames-1 of a sequence (frames scaled
    by 1 + eps). Per frame: (xi_est, T_cam<-world, log-depth prior mean, mu,
    valid-warp mask or None)."""
    from oracle.tracker import Tracker
    ora = Tracker(K, p, kf_interval=kf)
    out = []
    for k in range(seq.n_frames if n_frames is None else n_frames):
        f = seq.frame(k).astype(np.float64) * (1.0 + eps)
        xi = ora.track(f, seq.normals(k).astype(np.float64), n_iters=seq.sweeps if sweeps is None else sweeps)
        out.append((xi.copy(), ora.pose_global(), ora.win.d_prior, ora.state.mu.copy(),
                    ora.state.diag.get("valid")))
    return ora, out


def compare_tracks(gpu, ref, pert=None, label=""):
    """Per-frame results of a GPU run, ``gpu`` = [(xi, T, d_prior, mu)], against the
    oracle's ``ref``. The bar is the stated tolerance, or, when ``pert`` is given,
    max(stated tolerance, 100 x the oracle's own response ``pert`` to a 1e-15
    relative perturbation of the frames): a floor for the error any FP64
    implementation's rounding produces on an iteration that amplifies it. Returns
    the largest (pose, inverse-depth) errors."""
    worst = (0.0, 0.0)
    if pert is None:
        pert = ref
    for k, ((xi, T, dp, mu), (xi_o, T_o, dp_o, mu_o, valid), pk) in enumerate(zip(gpu, ref, pert)):
        sens_pose = np.abs(pk[0] - xi_o).max()
        sens_inv = inv_depth_rel_err(pk[3][..., 6], mu_o[..., 6], valid)
        e_pose = np.abs(xi - xi_o).max()
        e_inv = inv_depth_rel_err(mu[..., 6], mu_o[..., 6], valid)
        print("%s frame %d: pose %.1e (oracle sensitivity %.1e) inverse depth %.1e (sensitivity %.1e)"
              % (label, k, e_pose, sens_pose, e_inv, sens_inv))
        assert e_pose < max(1e-5, 100 * sens_pose), (label, k)
        assert np.abs(T - T_o).max() < max(1e-5, 100 * sens_pose), (label, k)
        # the prior mean is a mean log-depth: held like the inverse depths
        assert abs(dp - dp_o) < max(1e-4, 100 * abs(pk[2] - dp_o)), (label, k, dp - dp_o)
        assert e_inv < max(1e-4, 100 * sens_inv), (label, k)
        worst = (max(worst[0], e_pose), max(worst[1], e_inv))
    return worst
