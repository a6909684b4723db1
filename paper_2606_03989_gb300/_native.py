"""ctypes binding of the C ABI declared in include/pixvod.h.

Only argument marshalling lives here: every step of the sweep path runs in the
CUDA library. Importing this module loads lib/libpixvod.so and raises if it is
missing; there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# PIXVOD_LIBRARY=checked selects the checked build (lib/libpixvod_checked.so)
LIB_PATH = os.path.join(_PKG, "lib", "libpixvod_checked.so" if os.environ.get("PIXVOD_LIBRARY") == "checked"
                        else "libpixvod.so")

OK, EINVAL, ECUDA, ENUMERIC, ESTATE, ETIMEOUT, ENOMEM = range(7)
TOPOLOGY_GRID, TOPOLOGY_QUADTREE = 0, 1
SCHED_PLAIN, SCHED_BATCHED, SCHED_PERSISTENT = 0, 1, 2
SCHED_NAMES = {SCHED_PLAIN: "plain", SCHED_BATCHED: "batched", SCHED_PERSISTENT: "persistent"}
ADJOINT_HANDWRITTEN, ADJOINT_TAPE = 0, 1
FLAG_NONPOS_PIVOT, FLAG_NONFINITE, FLAG_TIMEOUT, FLAG_BOUNDS = 0x1, 0x2, 0x4, 0x10
N_PLANES = 151
N_INPUT_PLANES = 6
PL_MU, PL_MP, PL_U, PL_S, PL_ID, ID_STRIDE, PL_NM = 0, 7, 28, 34, 35, 27, 143


class PixvodError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__("%s: %s (status %d)" % (where, status_string(status), status))


class pixvod_intrinsics(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float),
                ("cy", ctypes.c_float), ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class pixvod_params(ctypes.Structure):
    _fields_ = [("sigma_D", ctypes.c_float), ("sigma_P", ctypes.c_float), ("sigma_R", ctypes.c_float),
                ("sigma_N", ctypes.c_float), ("sigma_Z", ctypes.c_float), ("t_huber", ctypes.c_float),
                ("damping", ctypes.c_float), ("kf_interval", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("topology", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 6)]


class pixvod_profile(ctypes.Structure):
    _fields_ = [("sweep_launches", ctypes.c_int64), ("sweep_ms", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("PixVOD CUDA library not built (%s); run "
                          "`python -m paper_2606_03989_gb300.build` first" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    P, S, I32, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int32, ctypes.c_int64
    H = ctypes.c_void_p
    sig = {
        "pixvod_status_string": (ctypes.c_char_p, [S]),
        "pixvod_abi_version": (ctypes.c_int, []),
        "pixvod_params_default": (pixvod_params, []),
        "pixvod_workspace_bytes": (S, [ctypes.POINTER(pixvod_intrinsics), ctypes.POINTER(pixvod_params),
                                       ctypes.POINTER(ctypes.c_size_t)]),
        "pixvod_state_bytes_per_pixel": (ctypes.c_size_t, [I32]),
        "pixvod_create": (S, [ctypes.POINTER(pixvod_intrinsics), ctypes.POINTER(pixvod_params), P,
                              ctypes.c_size_t, P, ctypes.POINTER(H)]),
        "pixvod_destroy": (S, [H]),
        "pixvod_track": (S, [H, P, P, I32]),
        "pixvod_track_host": (S, [H, P, P, I32]),
        "pixvod_sweep": (S, [H, I32]),
        "pixvod_get_pose": (S, [H, P]),
        "pixvod_get_pose_global": (S, [H, P]),
        "pixvod_get_pose_device": (S, [H, P]),
        "pixvod_get_depth": (S, [H, P]),
        "pixvod_get_inv_depth": (S, [H, P]),
        "pixvod_get_status": (S, [H, ctypes.POINTER(ctypes.c_uint32)]),
        "pixvod_state_size": (S, [H, ctypes.POINTER(ctypes.c_size_t)]),
        "pixvod_save_state": (S, [H, P, ctypes.c_size_t]),
        "pixvod_load_state": (S, [H, P, ctypes.c_size_t]),
        "pixvod_set_profiling": (S, [H, I32]),
        "pixvod_get_profile": (S, [H, ctypes.POINTER(pixvod_profile)]),
        "pixvod_launch_count": (S, [H, ctypes.POINTER(I64)]),
        "pixvod_backward_workspace_bytes": (S, [ctypes.POINTER(pixvod_intrinsics), ctypes.POINTER(pixvod_params),
                                                I32, I32, ctypes.POINTER(ctypes.c_size_t)]),
        "pixvod_set_recording": (S, [H, P, ctypes.c_size_t, I32, I32]),
        "pixvod_backward": (S, [H, P, P, P, P, P, P]),
        "pixvod_set_backward_window": (S, [H, I32]),
        "pixvod_set_backward_method": (S, [H, I32]),
        "pixvod_backward_tape_workspace_bytes": (S, [ctypes.POINTER(pixvod_intrinsics), ctypes.POINTER(pixvod_params),
                                                     I32, I32, ctypes.POINTER(ctypes.c_size_t)]),
        "pixvod_pose_mean_static": (S, [P, I32, I32, I64, I64, P, P]),
        "pixvod_batch_workspace_bytes": (S, [I32, P, ctypes.POINTER(pixvod_params), ctypes.POINTER(ctypes.c_size_t)]),
        "pixvod_batch_create": (S, [I32, P, ctypes.POINTER(pixvod_params), P, ctypes.c_size_t, P,
                                    ctypes.POINTER(H)]),
        "pixvod_batch_destroy": (S, [H]),
        "pixvod_batch_set_inputs": (S, [H, P, P]),
        "pixvod_batch_track": (S, [H, I32]),
        "pixvod_batch_get_poses": (S, [H, P]),
        "pixvod_batch_get_status": (S, [H, ctypes.POINTER(ctypes.c_uint32)]),
        "pixvod_batch_state_size": (S, [H, I32, ctypes.POINTER(ctypes.c_size_t)]),
        "pixvod_batch_save_state": (S, [H, I32, P, ctypes.c_size_t]),
        "pixvod_batch_set_schedule": (S, [H, I32, I32]),
        "pixvod_batch_get_schedule": (S, [H, ctypes.POINTER(I32), ctypes.POINTER(I32)]),
        "pixvod_batch_autotune": (S, [H, I32, I32, P]),
        "pixvod_batch_launch_count": (S, [H, ctypes.POINTER(I64)]),
        "pixvod_batch_set_wait_limit": (S, [H, I64]),
        "pixvod_batch_inject_barrier_fault": (S, [H, I32]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def status_string(s: int) -> str:
    return lib.pixvod_status_string(int(s)).decode()


def check(status: int, where: str):
    if status != OK:
        raise PixvodError(status, where)


def intrinsics(fx, fy, cx, cy, width, height) -> pixvod_intrinsics:
    return pixvod_intrinsics(float(fx), float(fy), float(cx), float(cy), int(width), int(height))


def params_default() -> pixvod_params:
    return lib.pixvod_params_default()


def params(**kw) -> pixvod_params:
    p = params_default()
    for k, v in kw.items():
        if not hasattr(p, k):
            raise TypeError("unknown parameter %r" % k)
        setattr(p, k, v)
    return p


def workspace_bytes(K: pixvod_intrinsics, p: pixvod_params) -> int:
    out = ctypes.c_size_t(0)
    check(lib.pixvod_workspace_bytes(ctypes.byref(K), ctypes.byref(p), ctypes.byref(out)),
          "pixvod_workspace_bytes")
    return out.value


@dataclass
class StateView:
    """Decoded checkpoint (see the layout in include/pixvod.h)."""
    precision: int
    width: int
    height: int
    frame_index: int
    has_target: bool
    planes: np.ndarray      # (151, H, W)
    inputs: np.ndarray      # (6, H, W): I_s, I_t, g_x, g_y, m_x, m_y
    scalars: np.ndarray     # (40,)
    nodes: Optional[np.ndarray] = None   # quadtree handles: (162, n_nodes), else None

    @property
    def node_pose(self):
        """(n_nodes, 6) poses of the quadtree nodes, level 1 first (None for the grid)."""
        return None if self.nodes is None else self.nodes[0:6].T

    @property
    def mu(self):
        return np.moveaxis(self.planes[PL_MU:PL_MU + 7], 0, -1)

    @property
    def M_p(self):
        """(H, W, 21) packed pose information without the photometric factor."""
        return np.moveaxis(self.planes[PL_MP:PL_MP + 21], 0, -1)

    @property
    def u(self):
        return np.moveaxis(self.planes[PL_U:PL_U + 6], 0, -1)

    @property
    def P(self):
        """(H, W, 21) packed depth-marginalised pose information M_p + u u^T."""
        u = self.u
        rows = [(r, c) for r in range(6) for c in range(r + 1)]
        return self.M_p + np.stack([u[..., r] * u[..., c] for (r, c) in rows], -1)

    @property
    def s(self):
        return self.planes[PL_S]

    @property
    def identity_messages(self):
        """(H, W, 4, 27): 21 packed Lambda then 6 eta per slot."""
        blk = self.planes[PL_ID:PL_ID + 4 * ID_STRIDE].reshape(4, ID_STRIDE, self.height, self.width)
        return np.moveaxis(blk, (2, 3), (0, 1))

    @property
    def normal_messages(self):
        """(H, W, 4, 2): Lambda, eta per slot."""
        blk = self.planes[PL_NM:PL_NM + 8].reshape(4, 2, self.height, self.width)
        return np.moveaxis(blk, (2, 3), (0, 1))

    @property
    def xi_est(self):
        return self.scalars[0:6]

    @property
    def T_kf(self):
        return self.scalars[6:22].reshape(4, 4)

    @property
    def T_cur(self):
        return self.scalars[22:38].reshape(4, 4)

    @property
    def d_prior(self):
        return float(self.scalars[38])


def parse_state(blob: bytes) -> StateView:
    hd = np.frombuffer(blob, dtype="<i8", count=10)
    if hd[0] != 0x50495856 or hd[1] != 1:
        raise ValueError("not a PixVOD state checkpoint")
    hd = np.frombuffer(blob, dtype="<i8", count=12)
    prec, W, H, pitch, nplanes, fidx, off_p, off_s, ninp, has_t = (int(x) for x in hd[2:12])
    dt = np.float64 if prec == 64 else np.float32
    allp = np.frombuffer(blob, dtype=dt, count=(nplanes + ninp) * H * pitch, offset=off_p)
    allp = allp.reshape(nplanes + ninp, H, pitch)[:, :, :W].astype(np.float64)
    sc = np.frombuffer(blob, dtype=np.float64, count=40, offset=off_s).copy()
    n_nodes, node_planes, off_n = (int(x) for x in np.frombuffer(blob, dtype="<i8", count=15)[12:15])
    nodes = None
    if node_planes:
        nodes = np.frombuffer(blob, dtype=dt, count=node_planes * n_nodes, offset=off_n)
        nodes = nodes.reshape(node_planes, n_nodes).astype(np.float64)
    return StateView(prec, W, H, fidx, bool(has_t), allp[:nplanes], allp[nplanes:], sc, nodes)
