"""The C-ABI library builds, loads and exports every function declared in
include/*.h (no GPU work: symbol lookup only)."""
import ctypes
import glob
import os
import re

import pytest

import paper_2504_02627_gb300 as g
from paper_2504_02627_gb300 import _binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:smc_status|void|int64_t)\s+(smc_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("smc_init", "smc_step", "smc_run", "smc_log_evidence", "smc_init_batch",
                     "smc_get_particles", "smc_moments", "smc_last_error", "smc_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = g.lib()
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert _declared() <= set(_binding.EXPORTS), _declared() - set(_binding.EXPORTS)


def test_library_is_sm103a_only():
    # the build passes exactly one -gencode for sm_103a
    from paper_2504_02627_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_invalid_config_is_rejected_without_gpu_work():
    lib = g.lib()
    h = ctypes.c_void_p()
    m = g.ModelData(g.BANANA, 3, hyper=(10.0, 0.1))    # odd dim: rejected before any launch
    cfg = g.make_config(16, 2, 1, 0.1)
    assert lib.smc_init(ctypes.byref(h), ctypes.byref(cfg), ctypes.byref(m.struct), None) == -1
    assert lib.smc_init(None, ctypes.byref(cfg), ctypes.byref(m.struct), None) == -1


def test_flow_parameter_count_matches_the_oracle_layout():
    import oracle
    lib = g.lib()
    for D, H, L in [(4, 8, 2), (10, 32, 4), (50, 128, 4), (100, 128, 4)]:
        assert lib.smc_flow_num_params(D, H, L) == oracle.num_flow_params(D, H, L)
    assert lib.smc_flow_num_params(1, 8, 2) == 0
