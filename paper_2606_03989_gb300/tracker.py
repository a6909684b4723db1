"""High-level handle over the C ABI, with PyTorch owning device memory and streams.

    import torch, paper_2606_03989_gb300 as pv
    trk = pv.Tracker((fx, fy, cx, cy, W, H), pv.params(kf_interval=10))
    trk.track(frame0_cuda, normals0_cuda)          # keyframe
    trk.track(frame1_cuda, n_iters=20)             # target: 20 GBP sweeps
    xi = trk.pose()                                # se(3) [theta; rho] vs keyframe
    depth = trk.depth()                            # (H, W) float32 CUDA tensor
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native as nat


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


class Tracker:
    def __init__(self, K, params=None, device=None, stream=None):
        import torch
        self._torch = torch
        if not torch.cuda.is_available():
            raise RuntimeError("PixVOD needs a CUDA device; no CPU implementation exists")
        if not isinstance(K, nat.pixvod_intrinsics):
            K = nat.intrinsics(*K)
        self.K = K
        self.params = params if params is not None else nat.params_default()
        self.device = torch.device(device if device is not None else "cuda")
        nbytes = nat.workspace_bytes(K, self.params)
        # over-allocate so the workspace can be aligned to 256 bytes
        self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self._ws.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        nat.check(nat.lib.pixvod_create(ctypes.byref(K), ctypes.byref(self.params), self._ws_ptr, nbytes,
                                        self.stream.cuda_stream, ctypes.byref(h)), "pixvod_create")
        self._h = h

    @property
    def shape(self):
        return (self.K.height, self.K.width)

    def close(self):
        if getattr(self, "_h", None):
            nat.lib.pixvod_destroy(self._h)
            self._h = None

    __del__ = close

    def _check_image(self, t, channels=1):
        torch = self._torch
        if t is None:
            return None
        shape = self.shape if channels == 1 else self.shape + (channels,)
        if tuple(t.shape) != shape or t.dtype != torch.float32 or not t.is_contiguous():
            raise ValueError("expected a contiguous float32 tensor of shape %s" % (shape,))
        return t

    def track(self, frame, normals=None, n_iters: int = 20):
        """frame: (H, W) float32 CUDA tensor; normals: (H, W, 3) float32 CUDA tensor
        when this frame becomes a keyframe."""
        frame = self._check_image(frame)
        normals = self._check_image(normals, 3)
        nat.check(nat.lib.pixvod_track(self._h, _ptr(frame), _ptr(normals), int(n_iters)), "pixvod_track")

    def track_host(self, frame, normals=None, n_iters: int = 20):
        """Host inputs (pinned CPU tensors or numpy arrays); copies run inside the library."""
        torch = self._torch
        keep = []

        def host_ptr(x, channels):
            if x is None:
                return 0
            if isinstance(x, np.ndarray):
                x = np.ascontiguousarray(x, dtype=np.float32)
                keep.append(x)
                return x.ctypes.data
            self._check_image(x, channels)
            if x.device.type != "cpu":
                raise ValueError("track_host expects host memory")
            keep.append(x)
            return x.data_ptr()

        st = nat.lib.pixvod_track_host(self._h, host_ptr(frame, 1), host_ptr(normals, 3), int(n_iters))
        nat.check(st, "pixvod_track_host")
        if any(isinstance(k, np.ndarray) for k in keep):
            self.stream.synchronize()   # pageable numpy buffers must outlive the copies
        return keep

    def sweep(self, n_iters: int):
        nat.check(nat.lib.pixvod_sweep(self._h, int(n_iters)), "pixvod_sweep")

    def pose(self) -> np.ndarray:
        xi = np.zeros(6)
        nat.check(nat.lib.pixvod_get_pose(self._h, xi.ctypes.data), "pixvod_get_pose")
        return xi

    def pose_global(self) -> np.ndarray:
        T = np.zeros(16)
        nat.check(nat.lib.pixvod_get_pose_global(self._h, T.ctypes.data), "pixvod_get_pose_global")
        return T.reshape(4, 4)

    def pose_device(self, out=None):
        torch = self._torch
        out = out if out is not None else torch.empty(6, dtype=torch.float64, device=self.device)
        nat.check(nat.lib.pixvod_get_pose_device(self._h, out.data_ptr()), "pixvod_get_pose_device")
        return out

    def depth(self, out=None):
        torch = self._torch
        out = out if out is not None else torch.empty(self.shape, dtype=torch.float32, device=self.device)
        nat.check(nat.lib.pixvod_get_depth(self._h, out.data_ptr()), "pixvod_get_depth")
        return out

    def inv_depth(self, out=None):
        torch = self._torch
        out = out if out is not None else torch.empty(self.shape, dtype=torch.float32, device=self.device)
        nat.check(nat.lib.pixvod_get_inv_depth(self._h, out.data_ptr()), "pixvod_get_inv_depth")
        return out

    def status(self) -> int:
        flags = ctypes.c_uint32(0)
        st = nat.lib.pixvod_get_status(self._h, ctypes.byref(flags))
        if st not in (nat.OK, nat.ENUMERIC, nat.ETIMEOUT):
            nat.check(st, "pixvod_get_status")
        return flags.value

    def save_state(self) -> bytes:
        n = ctypes.c_size_t(0)
        nat.check(nat.lib.pixvod_state_size(self._h, ctypes.byref(n)), "pixvod_state_size")
        buf = ctypes.create_string_buffer(n.value)
        nat.check(nat.lib.pixvod_save_state(self._h, buf, n.value), "pixvod_save_state")
        return buf.raw

    def load_state(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        nat.check(nat.lib.pixvod_load_state(self._h, buf, len(blob)), "pixvod_load_state")
        self.stream.synchronize()

    def state(self) -> nat.StateView:
        return nat.parse_state(self.save_state())

    def set_profiling(self, enable: bool):
        nat.check(nat.lib.pixvod_set_profiling(self._h, int(bool(enable))), "pixvod_set_profiling")

    def profile(self) -> dict:
        pr = nat.pixvod_profile()
        nat.check(nat.lib.pixvod_get_profile(self._h, ctypes.byref(pr)), "pixvod_get_profile")
        return {"sweep_launches": pr.sweep_launches, "sweep_ms": pr.sweep_ms,
                "kernel_launches": pr.kernel_launches}

    def launch_count(self) -> int:
        n = ctypes.c_int64(0)
        nat.check(nat.lib.pixvod_launch_count(self._h, ctypes.byref(n)), "pixvod_launch_count")
        return n.value

    # --- adjoint ---------------------------------------------------------
    def set_recording(self, max_iters: int, checkpoint_every: int = 5, method: int = 0):
        """Record target frames (up to max_iters sweeps) for backward(); method
        ADJOINT_HANDWRITTEN (0, default) or ADJOINT_TAPE (1, the FP64 tape kept
        for cross-checks)."""
        torch = self._torch
        nat.check(nat.lib.pixvod_set_backward_method(self._h, int(method)), "pixvod_set_backward_method")
        need = ctypes.c_size_t(0)
        query = (nat.lib.pixvod_backward_tape_workspace_bytes if method == nat.ADJOINT_TAPE
                 else nat.lib.pixvod_backward_workspace_bytes)
        nat.check(query(ctypes.byref(self.K), ctypes.byref(self.params), int(max_iters), int(checkpoint_every),
                        ctypes.byref(need)), "pixvod_backward_workspace_bytes")
        self._rec = torch.empty(need.value + 256, dtype=torch.uint8, device=self.device)
        ptr = (self._rec.data_ptr() + 255) // 256 * 256
        nat.check(nat.lib.pixvod_set_recording(self._h, ptr, need.value, int(max_iters), int(checkpoint_every)),
                  "pixvod_set_recording")

    def set_backward_window(self, last_sweeps: int):
        """Differentiate only the last `last_sweeps` sweeps (0 = all)."""
        nat.check(nat.lib.pixvod_set_backward_window(self._h, int(last_sweeps)), "pixvod_set_backward_window")

    def stop_recording(self):
        nat.check(nat.lib.pixvod_set_recording(self._h, None, 0, 1, 1), "pixvod_set_recording")
        self._rec = None

    def backward(self, grad_xi=None, grad_invdepth=None) -> dict:
        """Gradients of a loss through the last recorded frame's sweeps, given
        dL/dxi_est (6) and dL/d(inverse depth) (H, W); FP64 CUDA tensors out."""
        torch = self._torch
        H, W = self.shape
        f64 = dict(dtype=torch.float64, device=self.device)
        gx = None if grad_xi is None else torch.as_tensor(grad_xi).to(**f64).reshape(6).contiguous()
        gi = None if grad_invdepth is None else torch.as_tensor(grad_invdepth).to(**f64).reshape(H, W).contiguous()
        g_sig = torch.empty(2, **f64)
        g_Is = torch.empty(H, W, **f64)
        g_It = torch.empty(H, W, **f64)
        check = (ctypes.c_double * 2)()
        st = nat.lib.pixvod_backward(self._h, _ptr(gx), _ptr(gi), g_sig.data_ptr(), g_Is.data_ptr(),
                                     g_It.data_ptr(), ctypes.cast(check, ctypes.c_void_p))
        if st not in (nat.OK, nat.ENUMERIC):
            nat.check(st, "pixvod_backward")
        # ENUMERIC: a tape overflowed or the recomputed update differs from the
        # forward's beyond the documented bound; the caller decides
        return {"sigma_D": g_sig[0], "sigma_N": g_sig[1], "I_s": g_Is, "I_t": g_It, "status": st,
                "recompute_mismatch": check[0], "tape_nodes": int(check[1])}


def _track_frame_function():
    import torch

    class TrackFrame(torch.autograd.Function):
        """One recorded target frame as a differentiable function of the keyframe
        image, the target frame and the photometric / normal-prior sigmas."""

        @staticmethod
        def forward(ctx, trk, n_iters, keyframe, frame, sigma_D, sigma_N):
            for name, t in (("sigma_D", sigma_D), ("sigma_N", sigma_N)):
                if abs(float(t) - getattr(trk.params, name)) > 1e-6 * abs(float(t)):
                    raise ValueError("%s must equal the tracker's parameter" % name)
            trk.track(frame.detach().contiguous(), None, n_iters)
            xi = trk.pose_device().clone()
            inv = trk.inv_depth().to(torch.float64)
            ctx.trk = trk
            ctx.dtypes = (keyframe.dtype, frame.dtype, sigma_D.dtype, sigma_N.dtype)
            return xi, inv

        @staticmethod
        def backward(ctx, g_xi, g_inv):
            g = ctx.trk.backward(g_xi, g_inv)
            dk, df, ds, dn = ctx.dtypes
            return (None, None, g["I_s"].to(dk), g["I_t"].to(df), g["sigma_D"].to(ds).reshape(()),
                    g["sigma_N"].to(dn).reshape(()))

    return TrackFrame


_TrackFrame = None


def track_frame(trk: Tracker, frame, keyframe, sigma_D, sigma_N, n_iters: int = 20):
    """Track `frame` (a target frame) with recording on and return (xi_est,
    inverse depth) as autograd outputs of (keyframe, frame, sigma_D, sigma_N).
    `keyframe` must be the image the tracker holds as its keyframe, and the
    sigmas (0-dim tensors) its parameters; gradients flow to all four."""
    global _TrackFrame
    if _TrackFrame is None:
        _TrackFrame = _track_frame_function()
    if getattr(trk, "_rec", None) is None:
        trk.set_recording(max(int(n_iters), 1))
    return _TrackFrame.apply(trk, int(n_iters), keyframe, frame, sigma_D, sigma_N)


class Batch:
    """Many sequences (own intrinsics and state, shared params) advanced together.

    ``set_inputs`` registers one frame buffer and one normals buffer per
    sequence (CUDA tensors); ``track(n_iters)`` consumes what they hold."""

    def __init__(self, Ks, params=None, device=None, stream=None):
        import torch
        self._torch = torch
        if not torch.cuda.is_available():
            raise RuntimeError("PixVOD needs a CUDA device; no CPU implementation exists")
        self.K = [k if isinstance(k, nat.pixvod_intrinsics) else nat.intrinsics(*k) for k in Ks]
        self.n = len(self.K)
        self.params = params if params is not None else nat.params_default()
        self.device = torch.device(device if device is not None else "cuda")
        arr = (nat.pixvod_intrinsics * self.n)(*self.K)
        self._karr = arr
        need = ctypes.c_size_t(0)
        nat.check(nat.lib.pixvod_batch_workspace_bytes(self.n, ctypes.cast(arr, ctypes.c_void_p),
                                                        ctypes.byref(self.params), ctypes.byref(need)),
                  "pixvod_batch_workspace_bytes")
        self._ws = torch.empty(need.value + 256, dtype=torch.uint8, device=self.device)
        ptr = (self._ws.data_ptr() + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        nat.check(nat.lib.pixvod_batch_create(self.n, ctypes.cast(arr, ctypes.c_void_p), ctypes.byref(self.params),
                                              ptr, need.value, self.stream.cuda_stream, ctypes.byref(h)),
                  "pixvod_batch_create")
        self._h = h
        self._inputs = None

    def close(self):
        if getattr(self, "_h", None):
            nat.lib.pixvod_batch_destroy(self._h)
            self._h = None

    __del__ = close

    def set_inputs(self, frames, normals):
        assert len(frames) == self.n and len(normals) == self.n
        fp = (ctypes.c_void_p * self.n)(*[f.data_ptr() for f in frames])
        npp = (ctypes.c_void_p * self.n)(*[x.data_ptr() for x in normals])
        nat.check(nat.lib.pixvod_batch_set_inputs(self._h, ctypes.cast(fp, ctypes.c_void_p),
                                                  ctypes.cast(npp, ctypes.c_void_p)), "pixvod_batch_set_inputs")
        self._inputs = (list(frames), list(normals))   # keep the buffers alive

    def track(self, n_iters: int = 20):
        nat.check(nat.lib.pixvod_batch_track(self._h, int(n_iters)), "pixvod_batch_track")

    def poses(self) -> np.ndarray:
        xi = np.zeros((self.n, 6))
        nat.check(nat.lib.pixvod_batch_get_poses(self._h, xi.ctypes.data), "pixvod_batch_get_poses")
        return xi

    def status(self) -> int:
        flags = ctypes.c_uint32(0)
        st = nat.lib.pixvod_batch_get_status(self._h, ctypes.byref(flags))
        if st not in (nat.OK, nat.ENUMERIC, nat.ETIMEOUT):
            nat.check(st, "pixvod_batch_get_status")
        return flags.value

    def save_state(self, i: int) -> bytes:
        n = ctypes.c_size_t(0)
        nat.check(nat.lib.pixvod_batch_state_size(self._h, int(i), ctypes.byref(n)), "pixvod_batch_state_size")
        buf = ctypes.create_string_buffer(n.value)
        nat.check(nat.lib.pixvod_batch_save_state(self._h, int(i), buf, n.value), "pixvod_batch_save_state")
        return buf.raw

    def state(self, i: int) -> nat.StateView:
        return nat.parse_state(self.save_state(i))

    def set_schedule(self, schedule: int, blocks_per_sm: int = 4):
        nat.check(nat.lib.pixvod_batch_set_schedule(self._h, int(schedule), int(blocks_per_sm)),
                  "pixvod_batch_set_schedule")

    def schedule(self):
        s, b = ctypes.c_int32(0), ctypes.c_int32(0)
        nat.check(nat.lib.pixvod_batch_get_schedule(self._h, ctypes.byref(s), ctypes.byref(b)),
                  "pixvod_batch_get_schedule")
        return s.value, b.value

    def autotune(self, n_iters: int = 20, reps: int = 2):
        times = (ctypes.c_float * 5)()
        nat.check(nat.lib.pixvod_batch_autotune(self._h, int(n_iters), int(reps), ctypes.cast(times, ctypes.c_void_p)),
                  "pixvod_batch_autotune")
        names = ["plain", "batched", "persistent2", "persistent3", "persistent4"]
        return dict(zip(names, list(times))), self.schedule()

    def launch_count(self) -> int:
        n = ctypes.c_int64(0)
        nat.check(nat.lib.pixvod_batch_launch_count(self._h, ctypes.byref(n)), "pixvod_batch_launch_count")
        return n.value

    def set_wait_limit(self, polls: int):
        """Polls of the persistent schedule's grid barrier before it gives up (0: default)."""
        nat.check(nat.lib.pixvod_batch_set_wait_limit(self._h, int(polls)), "pixvod_batch_set_wait_limit")

    def inject_barrier_fault(self, on: bool):
        """Test hook: make every grid barrier of the persistent schedule time out."""
        nat.check(nat.lib.pixvod_batch_inject_barrier_fault(self._h, 1 if on else 0),
                  "pixvod_batch_inject_barrier_fault")
