"""The C-ABI library builds for sm_103a, loads, and exports every function
declared in include/gcvo.h (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*?\**\s*\b(gcvo_[a-z0-9_]+)\s*\(", src, re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2606_10019_gb300 import build as B
    return B.build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("gcvo_estimate_covariances", "gcvo_build_grid", "gcvo_eval", "gcvo_register"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings_and_defaults(libpath):
    from paper_2606_10019_gb300 import gcvo as G
    assert G.status_string(0) == "ok"
    assert "cutoff" in G.status_string(G.GCVO_ERR_NO_OVERLAP)
    kp = G.kernel_params()
    assert kp.cutoff == 3.0 and kp.knn == 10 and kp.sigma2 == 1.0
    sp = G.solver_params()
    assert sp.order == 2 and sp.k_max == 200


def test_invalid_arguments_are_rejected_before_any_device_work(libpath):
    from paper_2606_10019_gb300 import gcvo as G
    L = G.lib()
    assert L.gcvo_create(None, 0, None) == G.GCVO_ERR_INVALID_ARG
    assert L.gcvo_destroy(None) == G.GCVO_ERR_INVALID_ARG
    assert L.gcvo_grid_destroy(None) == G.GCVO_ERR_INVALID_ARG
    assert L.gcvo_eval(None, None, None, None, None, 0, None, None, None, None, None, None) == G.GCVO_ERR_INVALID_ARG
    assert L.gcvo_register(None, None, None, None, None, 0, None, None, None, None, None) == G.GCVO_ERR_INVALID_ARG
