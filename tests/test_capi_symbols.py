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
    assert L.gcvo_eval_exact(None, None, None, None, None, 0, None, None, None, None, None,
                             None) == G.GCVO_ERR_INVALID_ARG
    assert L.gcvo_register(None, None, None, None, None, 0, None, None, None, None, None) == G.GCVO_ERR_INVALID_ARG
    assert L.gcvo_register_batched(None, 0, None, None, None, None, None, None) == G.GCVO_ERR_INVALID_ARG
    assert L.gcvo_register_clouds(None, 1, None, None, None, None, None, None, None) == G.GCVO_ERR_INVALID_ARG
    assert L.gcvo_estimate_covariances_batched(None, 1, None, None, None, None) == G.GCVO_ERR_INVALID_ARG
    assert L.gcvo_build_grids_batched(None, 1, None, None, None, None, None, None) == G.GCVO_ERR_INVALID_ARG
    assert L.gcvo_pair_schedule(None, 8, None) == G.GCVO_ERR_INVALID_ARG
    assert L.gcvo_profile_enable(None, 1) == G.GCVO_ERR_INVALID_ARG
    P = ctypes.c_void_p
    L.gcvo_proposal_get_state.argtypes = [P, P, P, P]
    L.gcvo_proposal_set_state.argtypes = [P, P, P, ctypes.c_int64]
    assert L.gcvo_proposal_get_state(None, None, None, None) == G.GCVO_ERR_INVALID_ARG
    assert L.gcvo_proposal_set_state(None, None, None, 0) == G.GCVO_ERR_INVALID_ARG


def test_eval_static_rejects_bad_arguments_without_touching_a_device(libpath):
    """The no-allocation entry point checks its arguments (missing inputs,
    empty input, more points than its static scratch holds) before any CUDA
    call."""
    from paper_2606_10019_gb300 import gcvo as G
    L = G.lib()
    P = ctypes.c_void_p
    L.gcvo_eval_static.argtypes = [P, P, P, P, ctypes.c_int64, P, P, P, P, P]
    f = ctypes.c_double()
    g = (ctypes.c_double * 6)()
    H = (ctypes.c_double * 36)()
    T = (ctypes.c_double * 16)(*[1.0 if k % 5 == 0 else 0.0 for k in range(16)])
    assert L.gcvo_eval_static(None, None, None, None, 10, T, None, ctypes.byref(f), g, H) == G.GCVO_ERR_INVALID_ARG



def test_workspace_size_follows_the_limits(libpath):
    """gcvo_workspace_size needs no device: it grows with every limit and
    refuses limits outside the documented ranges."""
    from paper_2606_10019_gb300 import gcvo as G
    a = G.gcvo_workspace_size(10_000, 1, 0)
    b = G.gcvo_workspace_size(20_000, 1, 0)
    c = G.gcvo_workspace_size(20_000, 64, 0)
    d = G.gcvo_workspace_size(20_000, 64, 64 * 200)
    assert 0 < a < b < c < d
    # per point: source records, transformed records and partials dominate
    assert 400 < (b - a) / 10_000 < 2000
    L = G.lib()
    s = ctypes.c_size_t()
    assert L.gcvo_workspace_size(None, 0, 1, 0, ctypes.byref(s)) == G.GCVO_ERR_INVALID_ARG
    assert L.gcvo_workspace_size(None, 10, 0, 0, ctypes.byref(s)) == G.GCVO_ERR_INVALID_ARG
    assert L.gcvo_workspace_size(None, 10, 1, -1, ctypes.byref(s)) == G.GCVO_ERR_INVALID_ARG
    assert L.gcvo_set_workspace(None, None, 0, 1, 1, 0) == G.GCVO_ERR_INVALID_ARG
