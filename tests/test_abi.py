"""The C-ABI library builds, loads and exports every symbol include/pixvod.h
declares; host-side validation works without a GPU (no compute calls here)."""
import ctypes
import json
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pv():
    from paper_2606_03989_gb300 import build
    build.build()
    import paper_2606_03989_gb300 as pv
    return pv


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pixvod.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pixvod_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(pv):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(pv.lib, n), n
    # and nothing the binding binds is missing from the header
    from paper_2606_03989_gb300 import _native
    assert pv.lib.pixvod_abi_version() == 1
    assert set(names) >= {"pixvod_create", "pixvod_track", "pixvod_get_pose", "pixvod_get_depth"}


def test_default_params_are_the_papers(pv):
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_constants.json")))["sec4_2_leaf"]
    p = pv.params_default()
    for k, v in g.items():
        assert getattr(p, k) == pytest.approx(v, rel=1e-7), k
    assert p.precision == 32 and p.damping == 0.5 and p.sigma_Z == 1.0 and p.kf_interval == 10
    assert pv.status_string(pv.EINVAL) == "invalid argument"


def test_workspace_and_validation_without_a_gpu(pv):
    K = pv.intrinsics(525, 525, 319.5, 239.5, 640, 480)
    p = pv.params_default()
    n32 = pv.workspace_bytes(K, p)
    n64 = pv.workspace_bytes(K, pv.params(precision=64))
    # two ping-pong copies of 151 planes dominate: 640-wide rows are already 32-aligned
    assert n32 >= 2 * 151 * 640 * 480 * 4 and n64 >= 2 * 151 * 640 * 480 * 8
    assert pv.lib.pixvod_state_bytes_per_pixel(32) == 604
    assert pv.lib.pixvod_state_bytes_per_pixel(64) == 1208
    bad = [pv.params(sigma_D=0.0), pv.params(sigma_R=-1.0), pv.params(damping=1.0),
           pv.params(precision=16), pv.params(kf_interval=-1)]
    q = pv.params_default()
    q.reserved[3] = 1
    bad.append(q)
    out = ctypes.c_size_t()
    for b in bad:
        assert pv.lib.pixvod_workspace_bytes(ctypes.byref(K), ctypes.byref(b), ctypes.byref(out)) == pv.EINVAL
    for Kb in (pv.intrinsics(0, 1, 0, 0, 10, 10), pv.intrinsics(1, 1, 0, 0, 1, 10),
               pv.intrinsics(float("nan"), 1, 0, 0, 10, 10)):
        assert pv.lib.pixvod_workspace_bytes(ctypes.byref(Kb), ctypes.byref(p), ctypes.byref(out)) == pv.EINVAL
    h = ctypes.c_void_p()
    # argument errors are caught before any CUDA call
    assert pv.lib.pixvod_create(ctypes.byref(K), ctypes.byref(p), None, n32, None, ctypes.byref(h)) == pv.EINVAL
    assert pv.lib.pixvod_create(ctypes.byref(K), ctypes.byref(p), 0x1001, n32, None, ctypes.byref(h)) == pv.EINVAL
    assert pv.lib.pixvod_create(ctypes.byref(K), ctypes.byref(p), 0x100000, 16, None, ctypes.byref(h)) == pv.ENOMEM
    assert pv.lib.pixvod_track(None, None, None, 1) == pv.EINVAL
    assert pv.lib.pixvod_destroy(None) == pv.OK


def test_quadtree_workspace_holds_two_node_buffers(pv):
    """A quadtree handle adds two ping-pong buffers of 162 node planes; the node
    count follows the level shapes of the quadtree oracle (ceil halving down to one
    node): 102,409 nodes in 10 levels at 640x480."""
    from oracle import quadtree as qt
    for (w, h) in ((640, 480), (33, 17), (2, 9)):
        K = pv.intrinsics(525, 525, (w - 1) / 2, (h - 1) / 2, w, h)
        grid = pv.workspace_bytes(K, pv.params_default())
        quad = pv.workspace_bytes(K, pv.params(topology=pv.TOPOLOGY_QUADTREE))
        n = sum(a * b for a, b in qt.level_shapes(h, w))
        stride = (n + 63) // 64 * 64
        assert quad - grid >= 2 * 162 * stride * 4
        assert quad - grid < 2 * 162 * stride * 4 + 2 * 4096
    assert sum(a * b for a, b in qt.level_shapes(480, 640)) == 102409
    assert len(qt.level_shapes(480, 640)) == 10


def test_binding_fails_loudly_without_the_library(tmp_path):
    """Importing the binding from a copy with no built library raises."""
    import shutil
    import subprocess
    import sys
    dst = tmp_path / "paper_2606_03989_gb300"
    shutil.copytree(os.path.join(ROOT, "paper_2606_03989_gb300"), dst,
                    ignore=shutil.ignore_patterns("lib", "__pycache__"))
    code = "import paper_2606_03989_gb300 as pv\ntry:\n    pv.Tracker\nexcept ImportError as e:\n    print('IMPORT-ERROR', e)\n"
    out = subprocess.run([sys.executable, "-c", code], cwd=tmp_path, capture_output=True, text=True)
    assert "IMPORT-ERROR" in out.stdout, out.stdout + out.stderr
