"""Per-frame tracking schedule with keyframe anchoring, FP64 (numpy).

Sec. 3.5 and Sec. 4.3: a keyframe stays the source image while target frames
arrive; each target frame runs n_iters synchronous sweeps starting from the
previous frame's solution; its pose is the pixel average of the pose components.
App. A: after a fixed number of frames a new keyframe is designated.

Readings taken where the paper is silent:
* count rule: frame 0 is a keyframe; frame k > 0 is first tracked as a target
  and, if k is a multiple of kf_interval, then becomes the next keyframe;
* at a new keyframe: pose means and all messages are reset to zero, and the
  log-depth mean and the log-depth prior mean both become the mean log-depth of
  the finished segment (0 for the first keyframe), so every prior residual is
  zero at the reset point;
* between target frames the whole state (means, beliefs, messages) is carried;
* the camera pose is composed as T_cam<-world = Exp(xi_est) T_kf<-world, the world
  frame being the first keyframe's camera.

Test infrastructure: this package is the CPU oracle. Only tests/, the smoke check
and the bench's CPU-baseline leg may import it.
"""
from __future__ import annotations

import numpy as np

from . import factors as fac
from . import gbp, lie
from .factors import Intrinsics
from .gbp import Params


class Tracker:
    def __init__(self, K: Intrinsics, params: Params = Params(), kf_interval: int = 10):
        self.K = K
        self.params = params
        self.kf_interval = kf_interval
        self.frame_index = 0
        self.T_kf = np.eye(4)
        self.xi_est = np.zeros(6)
        self.win = None
        self.state = None

    def _set_keyframe(self, I_s, normals, d_prior):
        K = self.K
        m_x, m_y = fac.normal_edge_measurements(normals, K)
        I_s = np.asarray(I_s, np.float64)
        self.win = gbp.Window(K, I_s, m_x, m_y, I_s, *fac.image_gradient(I_s), 0, 0, d_prior)
        self.state = gbp.reset_state(I_s.shape, d_prior, self.params)

    def track(self, frame, normals=None, n_iters: int = 20) -> np.ndarray:
        """Consume one frame; returns xi_est of this frame relative to the keyframe
        it was tracked against (zeros for the very first frame)."""
        frame = np.asarray(frame, np.float64)
        if self.frame_index == 0:
            if normals is None:
                raise ValueError("the first frame is a keyframe and needs normals")
            self._set_keyframe(frame, normals, 0.0)
            self.xi_est = np.zeros(6)
        else:
            w = self.win
            w.I_t = frame
            w.g_x, w.g_y = fac.image_gradient(frame)
            for _ in range(n_iters):
                self.state = gbp.sweep(w, self.state, self.params)
            self.xi_est = gbp.pose_estimate(self.state.mu)
            if self.kf_interval > 0 and self.frame_index % self.kf_interval == 0:
                if normals is None:
                    raise ValueError("frame %d becomes a keyframe and needs normals" % self.frame_index)
                self.T_kf = lie.se3_matrix(self.xi_est) @ self.T_kf
                self._set_keyframe(frame, normals, float(self.state.mu[..., 6].mean()))
        self.frame_index += 1
        return self.xi_est

    def pose_global(self) -> np.ndarray:
        """T_cam<-world of the last frame (4x4)."""
        if self.frame_index > 1 and self.kf_interval > 0 and (self.frame_index - 1) % self.kf_interval == 0:
            return self.T_kf.copy()
        return lie.se3_matrix(self.xi_est) @ self.T_kf

    def depth(self) -> np.ndarray:
        return np.exp(self.state.mu[..., 6])
