"""Python binding of libgcvo (include/gcvo.h): argument marshalling only.

Functions keep the C names.  Point arrays are structure-of-arrays float32:
xyz (3, n), cov (6, n) with (xx, xy, xz, yy, yz, zz), feat (l, n).  They may
be CUDA tensors (used in place) or host arrays (NumPy or CPU tensors; the
library copies them).  Poses are 4x4 float64 arrays, row-major.

The CUDA library must have been built (``paper_2606_10019_gb300.build``);
nothing here computes any part of the method.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgcvo.so")

GCVO_OK = 0
GCVO_ERR_INVALID_ARG = 1
GCVO_ERR_CUDA = 2
GCVO_ERR_WORKSPACE = 3
GCVO_ERR_SINGULAR = 4
GCVO_ERR_NO_OVERLAP = 5
GCVO_ERR_NOT_CONVERGED = 6
GCVO_ERR_NONFINITE = 7
GCVO_ERR_TIMEOUT = 8
GCVO_ERR_CAPACITY = 9


class gcvo_kernel_params(ctypes.Structure):
    _fields_ = [("kernel_mode", ctypes.c_int), ("sigma2", ctypes.c_double), ("cutoff", ctypes.c_double),
                ("iso_ell", ctypes.c_double), ("knn", ctypes.c_int), ("eig_max", ctypes.c_double),
                ("eig_ratio", ctypes.c_double), ("feat_dim", ctypes.c_int), ("cell_size", ctypes.c_double)]


class gcvo_solver_params(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int), ("k_max", ctypes.c_int), ("eps_tol", ctypes.c_double),
                ("mu0", ctypes.c_double)]


class gcvo_iter_log(ctypes.Structure):
    _fields_ = [("f", ctypes.c_double), ("g", ctypes.c_double * 6), ("xi", ctypes.c_double * 6),
                ("xi_l1", ctypes.c_double), ("T", ctypes.c_double * 16), ("n_pairs", ctypes.c_int64),
                ("n_kept", ctypes.c_int64)]


class gcvo_eval_stats(ctypes.Structure):
    _fields_ = [("n_pairs", ctypes.c_int64), ("n_kept", ctypes.c_int64), ("n_candidates", ctypes.c_int64),
                ("rho", ctypes.c_double)]


class gcvo_problem(ctypes.Structure):
    _fields_ = [("target", ctypes.c_void_p), ("src_xyz", ctypes.c_void_p), ("src_cov", ctypes.c_void_p),
                ("src_feat", ctypes.c_void_p), ("n_src", ctypes.c_int64), ("T0", ctypes.c_double * 16)]


class gcvo_cloud_pair(ctypes.Structure):
    _fields_ = [("tgt_xyz", ctypes.c_void_p), ("tgt_feat", ctypes.c_void_p), ("n_tgt", ctypes.c_int64),
                ("src_xyz", ctypes.c_void_p), ("src_feat", ctypes.c_void_p), ("n_src", ctypes.c_int64),
                ("T0", ctypes.c_double * 16), ("params", ctypes.c_void_p)]


class gcvo_profile(ctypes.Structure):
    _fields_ = [("n_launches", ctypes.c_int64), ("n_pair_launches", ctypes.c_int64),
                ("pair_kernel_ms", ctypes.c_double), ("n_device_allocs", ctypes.c_int64),
                ("n_finalize_launches", ctypes.c_int64),
                ("finalize_ms", ctypes.c_double), ("transform_ms", ctypes.c_double),
                ("clouds_covariance_ms", ctypes.c_double), ("clouds_grid_ms", ctypes.c_double)]


class GcvoError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        detail = ""
        if status == GCVO_ERR_CUDA:
            detail = " -- " + lib().gcvo_last_error_detail().decode(errors="replace")
        super().__init__(f"{where}: {status_string(status)} ({status}){detail}")


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded libgcvo.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libgcvo.so is missing ({LIB_PATH}); run paper_2606_10019_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, I64, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        L.gcvo_status_string.restype = ctypes.c_char_p
        L.gcvo_status_string.argtypes = [I]
        L.gcvo_last_error_detail.restype = ctypes.c_char_p
        L.gcvo_last_error_detail.argtypes = []
        L.gcvo_default_kernel_params.argtypes = [P]
        L.gcvo_default_solver_params.argtypes = [P]
        L.gcvo_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), I, P]
        L.gcvo_destroy.argtypes = [P]
        L.gcvo_estimate_covariances.argtypes = [P, P, I64, P, P]
        L.gcvo_build_grid.argtypes = [P, P, P, P, I64, P, ctypes.POINTER(ctypes.c_void_p)]
        L.gcvo_grid_destroy.argtypes = [P]
        L.gcvo_rebuild_grid.argtypes = [P, P, P, P, P, I64, P]
        L.gcvo_grid_info.argtypes = [P, P, P, P]
        L.gcvo_eval.argtypes = [P, P, P, P, P, I64, P, P, P, P, P, P]
        L.gcvo_eval_exact.argtypes = [P, P, P, P, P, I64, P, P, P, P, P, P]
        L.gcvo_register.argtypes = [P, P, P, P, P, I64, P, P, P, P, P]
        L.gcvo_register_batched.argtypes = [P, I, P, P, P, P, P, P]
        L.gcvo_register_clouds.argtypes = [P, I, P, P, P, P, P, P, P]
        L.gcvo_workspace_size.argtypes = [P, I64, I, I64, ctypes.POINTER(ctypes.c_size_t)]
        L.gcvo_set_workspace.argtypes = [P, P, ctypes.c_size_t, I64, I, I64]
        L.gcvo_estimate_covariances_batched.argtypes = [P, I, P, P, P, P]
        L.gcvo_build_grids_batched.argtypes = [P, I, P, P, P, P, P, P]
        L.gcvo_pair_schedule.argtypes = [P, I, P]
        L.gcvo_profile_enable.argtypes = [P, I]
        L.gcvo_profile_read.argtypes = [P, P]
        _lib = L
    return _lib


def status_string(s: int) -> str:
    return lib().gcvo_status_string(int(s)).decode()


def _check(s: int, where: str, ok=(GCVO_OK,)):
    if s not in ok:
        raise GcvoError(s, where)
    return s


def _ptr(a) -> int | None:
    """Device or host address of a contiguous float32 array (or None)."""
    if a is None:
        return None
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.float32 or not a.is_contiguous():
                raise ValueError("point arrays must be contiguous float32")
            return a.data_ptr()
    except ImportError:
        pass
    if isinstance(a, np.ndarray):
        if a.dtype != np.float32 or not a.flags.c_contiguous:
            raise ValueError("point arrays must be contiguous float32")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def _n(a) -> int:
    return int(a.shape[-1])


def _pose(T) -> np.ndarray:
    T = np.ascontiguousarray(np.asarray(T, dtype=np.float64).reshape(4, 4))
    return T


def kernel_params(**kw) -> gcvo_kernel_params:
    p = gcvo_kernel_params()
    lib().gcvo_default_kernel_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def solver_params(**kw) -> gcvo_solver_params:
    p = gcvo_solver_params()
    lib().gcvo_default_solver_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


class Context:
    def __init__(self, handle: int, device: int):
        self.handle = handle
        self.device = device

    def close(self):
        if self.handle:
            lib().gcvo_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Grid:
    def __init__(self, handle: int, ctx: Context, keep):
        self.handle = handle
        self.ctx = ctx
        self._keep = keep

    def info(self):
        n = ctypes.c_int64()
        c = ctypes.c_int64()
        h = ctypes.c_double()
        _check(lib().gcvo_grid_info(self.handle, ctypes.byref(n), ctypes.byref(c), ctypes.byref(h)), "grid_info")
        return n.value, c.value, h.value

    def close(self):
        if self.handle:
            lib().gcvo_grid_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gcvo_create(device: int = 0, stream=None) -> Context:
    """stream: a torch.cuda.Stream, a raw cudaStream_t int, or None (the
    current torch stream if torch is importable, else the default stream)."""
    raw = 0
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                raw = torch.cuda.current_stream(device).cuda_stream
        except ImportError:
            pass
    elif isinstance(stream, int):
        raw = stream
    else:
        raw = stream.cuda_stream
    h = ctypes.c_void_p()
    _check(lib().gcvo_create(ctypes.byref(h), int(device), ctypes.c_void_p(raw) if raw else None), "gcvo_create")
    return Context(h.value, device)


def gcvo_destroy(ctx: Context) -> None:
    ctx.close()


def gcvo_estimate_covariances(ctx: Context, xyz, params: gcvo_kernel_params, cov_out) -> None:
    _check(lib().gcvo_estimate_covariances(ctx.handle, _ptr(xyz), _n(xyz), ctypes.byref(params), _ptr(cov_out)),
           "gcvo_estimate_covariances")


def gcvo_build_grid(ctx: Context, xyz, cov, feat, params: gcvo_kernel_params) -> Grid:
    h = ctypes.c_void_p()
    _check(lib().gcvo_build_grid(ctx.handle, _ptr(xyz), _ptr(cov), _ptr(feat), _n(xyz), ctypes.byref(params),
                                 ctypes.byref(h)), "gcvo_build_grid")
    return Grid(h.value, ctx, (xyz, cov, feat))


def gcvo_rebuild_grid(ctx: Context, grid: Grid, xyz, cov, feat, params: gcvo_kernel_params) -> Grid:
    _check(lib().gcvo_rebuild_grid(ctx.handle, grid.handle, _ptr(xyz), _ptr(cov), _ptr(feat), _n(xyz),
                                   ctypes.byref(params)), "gcvo_rebuild_grid")
    grid._keep = (xyz, cov, feat)
    return grid


def _ptr_array(arrs):
    out = (ctypes.c_void_p * len(arrs))()
    for k, a in enumerate(arrs):
        out[k] = _ptr(a)
    return out


def gcvo_estimate_covariances_batched(ctx: Context, xyz_list, params: gcvo_kernel_params, cov_list) -> None:
    """Covariances of several device clouds in one call (one set of launches)."""
    n = (ctypes.c_int64 * len(xyz_list))(*[_n(x) for x in xyz_list])
    _check(lib().gcvo_estimate_covariances_batched(ctx.handle, len(xyz_list), _ptr_array(xyz_list), n,
                                                   ctypes.byref(params), _ptr_array(cov_list)),
           "gcvo_estimate_covariances_batched")


def gcvo_build_grids_batched(ctx: Context, xyz_list, cov_list, feat_list, params: gcvo_kernel_params,
                             grids=None) -> list:
    """Build (grids[k] None) or rebuild grids for several device clouds in one
    call (one set of launches).  Returns the list of Grid objects."""
    m = len(xyz_list)
    grids = list(grids) if grids is not None else [None] * m
    h = (ctypes.c_void_p * m)(*[g.handle if g is not None else None for g in grids])
    n = (ctypes.c_int64 * m)(*[_n(x) for x in xyz_list])
    covs = _ptr_array(cov_list) if cov_list is not None else None
    st = lib().gcvo_build_grids_batched(ctx.handle, m, _ptr_array(xyz_list), covs, _ptr_array(feat_list), n,
                                        ctypes.byref(params), h)
    out = []
    for k in range(m):
        keep = (xyz_list[k], cov_list[k] if cov_list is not None else None, feat_list[k])
        if grids[k] is not None:
            grids[k]._keep = keep
            out.append(grids[k])
        elif h[k]:
            out.append(Grid(h[k], ctx, keep))
        else:
            out.append(None)
    _check(st, "gcvo_build_grids_batched")
    return out


@dataclass
class EvalResult:
    f: float
    g: np.ndarray
    H: np.ndarray
    M: np.ndarray
    n_pairs: int
    n_kept: int
    n_candidates: int
    rho: float


def gcvo_eval(ctx: Context, grid: Grid, src_xyz, src_cov, src_feat, T) -> EvalResult:
    T = _pose(T)
    f = ctypes.c_double()
    g = np.zeros(6)
    H = np.zeros(36)
    M = np.zeros(36)
    st = gcvo_eval_stats()
    _check(lib().gcvo_eval(ctx.handle, grid.handle, _ptr(src_xyz), _ptr(src_cov), _ptr(src_feat), _n(src_xyz),
                           T.ctypes.data, ctypes.byref(f), g.ctypes.data, H.ctypes.data, M.ctypes.data,
                           ctypes.byref(st)), "gcvo_eval")
    return EvalResult(f.value, g, H.reshape(6, 6), M.reshape(6, 6), st.n_pairs, st.n_kept, st.n_candidates, st.rho)


@dataclass
class ExactEvalResult:
    f: float
    g: np.ndarray
    H: np.ndarray       # H_E = D(g) + Gamma
    D: np.ndarray       # D(g), the exact derivative of the gradient field
    n_pairs: int
    n_kept: int
    n_candidates: int
    rho: float


def gcvo_eval_exact(ctx: Context, grid: Grid, src_xyz, src_cov, src_feat, T) -> ExactEvalResult:
    T = _pose(T)
    f = ctypes.c_double()
    g = np.zeros(6)
    H = np.zeros(36)
    D = np.zeros(36)
    st = gcvo_eval_stats()
    _check(lib().gcvo_eval_exact(ctx.handle, grid.handle, _ptr(src_xyz), _ptr(src_cov), _ptr(src_feat),
                                 _n(src_xyz), T.ctypes.data, ctypes.byref(f), g.ctypes.data, H.ctypes.data,
                                 D.ctypes.data, ctypes.byref(st)), "gcvo_eval_exact")
    return ExactEvalResult(f.value, g, H.reshape(6, 6), D.reshape(6, 6), st.n_pairs, st.n_kept, st.n_candidates,
                           st.rho)


# The iteration log as a NumPy record type with the layout of gcvo_iter_log:
# rows index like dicts (row["f"], row["T"] as a 4 x 4 pose, ...) and whole
# columns are vectors (log["n_pairs"]), without copying the C buffer.
LOG_DTYPE = np.dtype([("f", "<f8"), ("g", "<f8", (6,)), ("xi", "<f8", (6,)), ("xi_l1", "<f8"),
                      ("T", "<f8", (4, 4)), ("n_pairs", "<i8"), ("n_kept", "<i8")])
assert LOG_DTYPE.itemsize == ctypes.sizeof(gcvo_iter_log)


def _logs_view(logs, k_max: int, n_iter) -> list:
    """Per problem, the first n_iter[k] rows of its k_max log rows, as
    record arrays sharing the memory of the ctypes buffer."""
    rec = np.frombuffer(logs, dtype=LOG_DTYPE)
    return [rec[k * k_max:k * k_max + int(n)] for k, n in enumerate(n_iter)]


def gcvo_register(ctx: Context, grid: Grid, src_xyz, src_cov, src_feat, T0, params: gcvo_solver_params,
                  want_log: bool = True):
    """Returns (T, log list, n_iter, status); status is GCVO_OK or
    GCVO_ERR_NOT_CONVERGED (other statuses raise)."""
    T0 = _pose(T0)
    T = np.zeros(16)
    logs = (gcvo_iter_log * params.k_max)() if want_log else None
    n_iter = ctypes.c_int()
    s = lib().gcvo_register(ctx.handle, grid.handle, _ptr(src_xyz), _ptr(src_cov), _ptr(src_feat), _n(src_xyz),
                            T0.ctypes.data, ctypes.byref(params), T.ctypes.data,
                            ctypes.cast(logs, ctypes.c_void_p) if logs is not None else None, ctypes.byref(n_iter))
    _check(s, "gcvo_register", ok=(GCVO_OK, GCVO_ERR_NOT_CONVERGED))
    return T.reshape(4, 4), (_logs_view(logs, params.k_max, [n_iter.value])[0] if logs is not None else None), \
        n_iter.value, s


def gcvo_register_batched(ctx: Context, problems: list[tuple], params: gcvo_solver_params, want_log: bool = False):
    """problems: list of (grid, src_xyz, src_cov, src_feat, T0).  Returns
    (T (n, 4, 4), logs or None, n_iter (n,), status (n,))."""
    n = len(problems)
    arr = (gcvo_problem * n)()
    for k, (grid, xyz, cov, feat, T0) in enumerate(problems):
        arr[k].target = grid.handle
        arr[k].src_xyz = _ptr(xyz)
        arr[k].src_cov = _ptr(cov)
        arr[k].src_feat = _ptr(feat)
        arr[k].n_src = _n(xyz)
        arr[k].T0[:] = list(_pose(T0).ravel())
    T = np.zeros((n, 16))
    n_iter = np.zeros(n, dtype=np.int32)
    status = np.zeros(n, dtype=np.int32)
    logs = (gcvo_iter_log * (n * params.k_max))() if want_log else None
    _check(lib().gcvo_register_batched(ctx.handle, n, ctypes.cast(arr, ctypes.c_void_p), ctypes.byref(params),
                                       T.ctypes.data, ctypes.cast(logs, ctypes.c_void_p) if logs is not None else None,
                                       n_iter.ctypes.data, status.ctypes.data), "gcvo_register_batched")
    out_logs = None
    if logs is not None:
        out_logs = _logs_view(logs, params.k_max, n_iter)
    return T.reshape(n, 4, 4), out_logs, n_iter, status


def gcvo_register_clouds(ctx: Context, pairs: list[tuple], params: gcvo_kernel_params, solver: gcvo_solver_params,
                         want_log: bool = False):
    """The whole hot path from raw clouds in one call.  pairs: list of
    (tgt_xyz, tgt_feat, src_xyz, src_feat, T0) or (..., T0, kernel_params);
    arrays on the device or on the host (host arrays are copied in by the
    library).  Returns (T (n, 4, 4), logs or None, n_iter (n,), status (n,))."""
    n = len(pairs)
    arr = (gcvo_cloud_pair * n)()
    keep = []
    for k, pr in enumerate(pairs):
        tx, tf, sx, sf, T0 = pr[:5]
        arr[k].tgt_xyz, arr[k].tgt_feat, arr[k].n_tgt = _ptr(tx), _ptr(tf), _n(tx)
        arr[k].src_xyz, arr[k].src_feat, arr[k].n_src = _ptr(sx), _ptr(sf), _n(sx)
        arr[k].T0[:] = list(_pose(T0).ravel())
        if len(pr) > 5 and pr[5] is not None:
            keep.append(pr[5])
            arr[k].params = ctypes.cast(ctypes.byref(pr[5]), ctypes.c_void_p)
    T = np.zeros((n, 16))
    n_iter = np.zeros(n, dtype=np.int32)
    status = np.zeros(n, dtype=np.int32)
    logs = (gcvo_iter_log * (n * solver.k_max))() if want_log else None
    _check(lib().gcvo_register_clouds(ctx.handle, n, ctypes.cast(arr, ctypes.c_void_p), ctypes.byref(params),
                                      ctypes.byref(solver), T.ctypes.data,
                                      ctypes.cast(logs, ctypes.c_void_p) if logs is not None else None,
                                      n_iter.ctypes.data, status.ctypes.data), "gcvo_register_clouds")
    out_logs = None
    if logs is not None:
        out_logs = _logs_view(logs, solver.k_max, n_iter)
    return T.reshape(n, 4, 4), out_logs, n_iter, status


def gcvo_workspace_size(max_points: int, max_problems: int = 1, max_log_rows: int = 0) -> int:
    """Bytes of a caller-owned workspace for calls of at most max_points
    points, max_problems problems and max_log_rows iteration-log rows."""
    b = ctypes.c_size_t()
    _check(lib().gcvo_workspace_size(None, int(max_points), int(max_problems), int(max_log_rows), ctypes.byref(b)),
           "gcvo_workspace_size")
    return int(b.value)


def gcvo_set_workspace(ctx: Context, buf, max_points: int = 1, max_problems: int = 1, max_log_rows: int = 0) -> None:
    """Hand the context a caller-owned device buffer (a CUDA uint8 tensor of
    at least gcvo_workspace_size bytes) as its scratch, or None to return to
    library-owned scratch.  The buffer must outlive its use by the context."""
    if buf is None:
        _check(lib().gcvo_set_workspace(ctx.handle, None, 0, 1, 1, 0), "gcvo_set_workspace")
        ctx._workspace = None
        return
    _check(lib().gcvo_set_workspace(ctx.handle, buf.data_ptr(), buf.numel() * buf.element_size(), int(max_points),
                                    int(max_problems), int(max_log_rows)), "gcvo_set_workspace")
    ctx._workspace = buf


def gcvo_pair_schedule(ctx: Context, set: int = -1) -> int:
    """Force the pair-pass schedule (4, 8, 16, 32 points per sub-tile), hand it
    back to the autotuner (0) or leave it (-1); returns the last one used."""
    last = ctypes.c_int()
    _check(lib().gcvo_pair_schedule(ctx.handle, int(set), ctypes.byref(last)), "gcvo_pair_schedule")
    return last.value


def gcvo_profile_enable(ctx: Context, enable: bool = True) -> None:
    _check(lib().gcvo_profile_enable(ctx.handle, int(bool(enable))), "gcvo_profile_enable")


def gcvo_profile_read(ctx: Context) -> dict:
    p = gcvo_profile()
    _check(lib().gcvo_profile_read(ctx.handle, ctypes.byref(p)), "gcvo_profile_read")
    return dict(n_launches=p.n_launches, n_pair_launches=p.n_pair_launches, pair_kernel_ms=p.pair_kernel_ms,
                n_device_allocs=p.n_device_allocs,
                n_finalize_launches=p.n_finalize_launches, finalize_ms=p.finalize_ms, transform_ms=p.transform_ms,
                clouds_covariance_ms=p.clouds_covariance_ms, clouds_grid_ms=p.clouds_grid_ms)


# ---------------------------------------------------------------------------
# Learned initial-pose proposal
# ---------------------------------------------------------------------------

def _prop_lib():
    L = lib()
    if not getattr(L, "_prop_ready", False):
        P, I = ctypes.c_void_p, ctypes.c_int
        L.gcvo_proposal_n_params.restype = ctypes.c_int64
        L.gcvo_proposal_n_params.argtypes = []
        L.gcvo_proposal_create.argtypes = [P, ctypes.POINTER(ctypes.c_void_p)]
        L.gcvo_proposal_destroy.argtypes = [P]
        L.gcvo_proposal_set_params.argtypes = [P, P, P]
        L.gcvo_proposal_get_params.argtypes = [P, P, P]
        L.gcvo_proposal_get_state.argtypes = [P, P, P, ctypes.POINTER(ctypes.c_int64)]
        L.gcvo_proposal_set_state.argtypes = [P, P, P, ctypes.c_int64]
        L.gcvo_proposal_infer.argtypes = [P, P, I, I, P, P, I, P, P, I, P, P]
        L.gcvo_proposal_train_step.argtypes = [P, P, I, I, P, P, I, P, P, I, P, ctypes.c_float, P, P]
        L._prop_ready = True
    return L


class Proposal:
    """Handle of a proposal network (gcvo_proposal_*)."""

    def __init__(self, ctx: Context):
        L = _prop_lib()
        h = ctypes.c_void_p()
        _check(L.gcvo_proposal_create(ctx.handle, ctypes.byref(h)), "gcvo_proposal_create")
        self.handle = h.value
        self.ctx = ctx
        self.n_params = int(L.gcvo_proposal_n_params())

    def close(self):
        if self.handle:
            _prop_lib().gcvo_proposal_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params: np.ndarray) -> None:
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == self.n_params
        _check(_prop_lib().gcvo_proposal_set_params(self.ctx.handle, self.handle, p.ctypes.data), "set_params")

    def get_params(self) -> np.ndarray:
        p = np.zeros(self.n_params, dtype=np.float32)
        _check(_prop_lib().gcvo_proposal_get_params(self.ctx.handle, self.handle, p.ctypes.data), "get_params")
        return p

    def get_state(self):
        """(state (3, n_params) float32: parameters, Adam m, Adam v; Adam step)."""
        st = np.zeros((3, self.n_params), dtype=np.float32)
        step = ctypes.c_int64()
        _check(_prop_lib().gcvo_proposal_get_state(self.ctx.handle, self.handle, st.ctypes.data, ctypes.byref(step)),
               "get_state")
        return st, int(step.value)

    def set_state(self, state: np.ndarray, step: int) -> None:
        st = np.ascontiguousarray(state, dtype=np.float32)
        assert st.size == 3 * self.n_params
        _check(_prop_lib().gcvo_proposal_set_state(self.ctx.handle, self.handle, st.ctypes.data, int(step)),
               "set_state")

    def infer(self, src_xyz, src_feat, tgt_xyz, tgt_feat):
        """Batched clouds: xyz (B, 3, n), feat (B, n) device tensors.
        Returns (twists (B, 6) normalised, T0 (B, 4, 4))."""
        B, _, n = src_xyz.shape
        tw = np.zeros((B, 6), dtype=np.float32)
        T0 = np.zeros((B, 16))
        _check(_prop_lib().gcvo_proposal_infer(self.ctx.handle, self.handle, B, n, _ptr(src_xyz), _ptr(src_feat),
                                               int(src_feat.stride(0)), _ptr(tgt_xyz), _ptr(tgt_feat),
                                               int(tgt_feat.stride(0)), tw.ctypes.data, T0.ctypes.data),
               "gcvo_proposal_infer")
        return tw, T0.reshape(B, 4, 4)

    def train_step(self, src_xyz, src_feat, tgt_xyz, tgt_feat, T_label, lr: float, want_grad: bool = False):
        B, _, n = src_xyz.shape
        lab = np.ascontiguousarray(np.asarray(T_label, dtype=np.float64).reshape(B, 16))
        loss = ctypes.c_float()
        grad = np.zeros(self.n_params, dtype=np.float32) if want_grad else None
        _check(_prop_lib().gcvo_proposal_train_step(self.ctx.handle, self.handle, B, n, _ptr(src_xyz),
                                                    _ptr(src_feat), int(src_feat.stride(0)), _ptr(tgt_xyz),
                                                    _ptr(tgt_feat), int(tgt_feat.stride(0)), lab.ctypes.data,
                                                    float(lr), ctypes.byref(loss),
                                                    grad.ctypes.data if grad is not None else None),
               "gcvo_proposal_train_step")
        return loss.value, grad


def gcvo_eval_static(grid: Grid, src_xyz, src_cov, src_feat, T, stream=None):
    """gcvo_eval_static: the same evaluation as gcvo_eval without a context and
    without allocating device memory (device inputs only, at most 65536
    source points).  Returns (f, g, H)."""
    L = lib()
    if not getattr(L, "_static_ready", False):
        P = ctypes.c_void_p
        L.gcvo_eval_static.argtypes = [P, P, P, P, ctypes.c_int64, P, P, P, P, P]
        L._static_ready = True
    raw = 0
    if stream is None:
        import torch
        raw = torch.cuda.current_stream().cuda_stream
    elif isinstance(stream, int):
        raw = stream
    else:
        raw = stream.cuda_stream
    T = _pose(T)
    f = ctypes.c_double()
    g = np.zeros(6)
    H = np.zeros(36)
    _check(L.gcvo_eval_static(grid.handle, _ptr(src_xyz), _ptr(src_cov), _ptr(src_feat), _n(src_xyz), T.ctypes.data,
                              ctypes.c_void_p(raw) if raw else None, ctypes.byref(f), g.ctypes.data, H.ctypes.data),
           "gcvo_eval_static")
    return f.value, g, H.reshape(6, 6)
