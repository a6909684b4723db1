"""The checked build (libpixvod_checked.so, compiled with PIXVOD_CHECKED): every
index the sweep computes is tested against its buffer (PIXVOD_FLAG_BOUNDS on a
violation, the access skipped) and the out-of-image lanes of ragged tiles hold
NaN, so a read of them shows as PIXVOD_FLAG_NONFINITE. Ragged images through
every path (grid tracking with keyframes in both precisions, every batch
schedule, the quadtree topology, the adjoint) must raise no flag, and give the
plain build's results. The checked library runs in a child process (the
library is chosen when the package is imported)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCENARIOS = r'''
import json, sys
import numpy as np
import torch
sys.path.insert(0, ROOT)
import synth
import paper_2606_03989_gb300 as pv
dev = torch.device("cuda:0")
out = {"lib": pv.LIB_PATH}
cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
# grid tracking, ragged 70x45, a keyframe every 3 frames
seq = synth.realistic(11, 5, 70, 45, sweeps=3)
for prec in (32, 64):
    trk = pv.Tracker(seq.cam.as_tuple(), pv.params(precision=prec, kf_interval=3, sigma_P=seq.sigma_P), dev)
    poses = []
    for k in range(5):
        trk.track(cu(seq.frame(k)), cu(seq.normals(k)) if k % 3 == 0 else None, 3)
        poses.append(trk.pose().tolist())
    out["grid%d" % prec] = {"flags": trk.status(), "poses": poses}
# batches of ragged sizes in every schedule
seqs = [synth.realistic(40 + i, 3, w, h) for i, (w, h) in enumerate([(70, 45), (33, 17)])]
for sched, blocks in ((pv.SCHED_PLAIN, 4), (pv.SCHED_BATCHED, 4), (pv.SCHED_PERSISTENT, 4)):
    b = pv.Batch([s.cam.as_tuple() for s in seqs], pv.params(precision=32, kf_interval=2, sigma_P=0.05), dev)
    b.set_schedule(sched, blocks)
    for k in range(3):
        b.set_inputs([cu(s.frame(k)) for s in seqs], [cu(s.normals(k)) for s in seqs])
        b.track(3)
    out["batch%d" % sched] = {"flags": b.status(), "poses": b.poses().tolist()}
# quadtree topology, ragged 33x17
q = synth.realistic(12, 2, 33, 17)
trk = pv.Tracker(q.cam.as_tuple(), pv.params(precision=32, kf_interval=0, sigma_P=q.sigma_P,
                                              topology=pv.TOPOLOGY_QUADTREE), dev)
trk.track(cu(q.frame(0)), cu(q.normals(0)))
trk.track(cu(q.frame(1)), None, 4)
out["quadtree"] = {"flags": trk.status(), "poses": [trk.pose().tolist()]}
# adjoint, 16x12 (ragged against the 32-wide tiles), FP64 (the FP32 gradient
# through 5 sweeps carries percent-level amplified rounding)
a = synth.realistic(5, 2, 16, 12)
trk = pv.Tracker(a.cam.as_tuple(), pv.params(precision=64, kf_interval=0, sigma_P=a.sigma_P), dev)
trk.set_recording(5, 2)
trk.track(cu(a.frame(0)), cu(a.normals(0)))
trk.track(cu(a.frame(1)), None, 5)
g = trk.backward(np.ones(6), None)
out["adjoint"] = {"flags": trk.status(), "status": g["status"], "sigma": [float(g["sigma_D"]), float(g["sigma_N"])],
                  "poses": [trk.pose().tolist()]}
print("RESULT " + json.dumps(out))
'''


def run(checked):
    env = dict(os.environ)
    if checked:
        env["PIXVOD_LIBRARY"] = "checked"
    else:
        env.pop("PIXVOD_LIBRARY", None)
    res = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + SCENARIOS], env=env, capture_output=True,
                         text=True, timeout=900)
    assert res.returncode == 0, res.stderr[-3000:]
    line = [l for l in res.stdout.splitlines() if l.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):])


def test_checked_build_raises_no_flag_and_matches_the_plain_build():
    checked, plain = run(True), run(False)
    assert checked["lib"].endswith("libpixvod_checked.so") and plain["lib"].endswith("libpixvod.so")
    for key, r in checked.items():
        if key == "lib":
            continue
        assert r["flags"] == 0, (key, r["flags"])
        a, b = np.array(r["poses"]), np.array(plain[key]["poses"])
        assert np.isfinite(a).all(), key
        tol = 1e-9 if key in ("grid64", "adjoint") else 1e-3
        assert np.abs(a - b).max() < tol, (key, np.abs(a - b).max())
    assert checked["adjoint"]["status"] == 0
    assert np.allclose(checked["adjoint"]["sigma"], plain["adjoint"]["sigma"], rtol=1e-6)
