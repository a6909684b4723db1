"""FP64 CPU oracle of the PixVOD GBP sweep path (numpy).

TEST INFRASTRUCTURE. Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import, call or execute anything here; the product path
(the C-ABI library and its Python binding) never does.

Modules: ``lie`` (SE(3) Exp/Log), ``factors`` (Eqs. 2-6 linearised),
``gbp`` (synchronous sweeps, frozen-linearisation GBP, dense Gauss-Newton
system), ``tracker`` (per-frame schedule and keyframe anchoring).

Every function here is pinned by a CPU test against something other than
itself (library routines, closed forms, finite differences, brute-force dense
solves, invariants); see tests/test_oracle_*.py.
"""
from . import factors, gbp, lie, tracker
from .factors import Intrinsics
from .gbp import Params

__all__ = ["factors", "gbp", "lie", "tracker", "Intrinsics", "Params"]
