"""The C ABI library builds for sm_103a and exports every function include/bgs.h declares (no GPU)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "bgs.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"\b(bgs_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="nvcc not available")
def test_library_builds_and_exports_every_declared_symbol():
    from paper_2602_13079_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 18
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_options_struct_matches_header_defaults():
    import paper_2602_13079_gb300 as bgs
    from paper_2602_13079_gb300 import _build
    _build.build()
    o = bgs.bgs_default_options()
    assert o.restart == 50 and o.maxit == 1000 and o.rtol == 1e-8
    assert list(o.cheb_degree)[:5] == [4, 4, 2, 2, 2]
    assert abs(o.theta[0] - 0.04) < 1e-15 and o.theta[1] == 0.0
    assert o.max_coarse == 500 and o.max_levels == 10 and o.filter_diag == 1 and o.reorth_eta == 0.01
    assert o.jacobi == 0
    # the later options, as include/bgs.h documents their defaults
    assert o.precision == 0 and o.graph == 1 and o.autotune == 1
    assert o.cheb_ratio == 30.0 and abs(o.cheb_boost - 1.1) < 1e-15 and o.power_iters == 10
    assert list(o.subsolver) == [0] * 8 and o.ilu_rows == 4096
    assert o.ngroups == 0 and o.inner_restart == 30 and o.inner_maxit == 30 and o.inner_rtol == 1e-6
    assert o.cheb_ellipse == 0
    assert bgs.status_string(3) == "no convergence within maxit"
