"""FP64 CPU oracle for G-CVO -- TEST INFRASTRUCTURE ONLY.

Plain, slow, brute-force restatement of the paper's method used to check the
CUDA library.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it; the library never does.

Heavy all-pairs loops live in ``gcvo_oracle.c`` (double precision, every pair
visited); the small dense steps (exp map, connection, 6x6 solve, Alg. 1) are
written here with NumPy in double precision.

Parity status of each function (what pins it, see tests/test_oracle_pins.py):
  knn_cov / eig_clamp : brute force vs scipy cKDTree neighbour sets, closed
                        forms on lines and planes, numpy.linalg.eigh.
  evaluate (f, g, M)  : central finite differences of the frozen-Sigma
                        objective; isotropic case vs a scipy cdist sum;
                        invariance under a common rigid motion.
  gamma_matrix        : torsion-free and metric-compatibility identities and
                        the closed form of Eq. (12).
  exp_se3             : scipy.linalg.expm of the 4x4 twist matrix.
  register            : exact recovery in the isotropic and sphere cases.
  linesearch          : polynomial vs direct evaluation of G(t) to O(t^5).
                        The printed-coefficient variant (literal=True) is
                        parity unpinned: it is kept only to show the printed
                        form, and nothing on the CUDA side follows it.
  f_near / g_near     : one pair placed just inside, just outside and well
                        inside the cutoff.
  grad_derivative     : central finite differences of g; its fourth term is
                        -M; isotropic D(g) + Gamma is self-adjoint; Newton on
                        it reaches the G-CVO-2 stationary point.
  grad_derivative_c   : the same D(g) as C loops, equal to grad_derivative
                        and to finite differences of g.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gcvo_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the C part of the oracle (gcc, OpenMP when available)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-shared", "-fPIC", "-std=c11", _SRC, "-o", tmp, "-lm"]
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:
        r = subprocess.run(base, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [("kernel_mode", ctypes.c_int), ("sigma2", ctypes.c_double), ("cutoff", ctypes.c_double),
                ("iso_ell", ctypes.c_double), ("feat_dim", ctypes.c_int), ("rho", ctypes.c_double)]


class _EvalOut(ctypes.Structure):
    _fields_ = [("f", ctypes.c_double), ("g", ctypes.c_double * 6), ("M", ctypes.c_double * 36),
                ("gabs", ctypes.c_double * 6), ("n_pairs_kept", ctypes.c_double),
                ("n_pairs_rho", ctypes.c_double), ("n_near_cut", ctypes.c_double),
                ("f_near", ctypes.c_double), ("g_near", ctypes.c_double * 6)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        _lib.orc_knn_cov.argtypes = [P, ctypes.c_int64, ctypes.c_int, P, P, P]
        _lib.orc_sym3_eig.argtypes = [P, P, P]
        _lib.orc_eig_clamp.argtypes = [P, ctypes.c_int64, ctypes.c_double, ctypes.c_double]
        _lib.orc_eval.argtypes = [P, P, P, ctypes.c_int64, P, P, P, ctypes.c_int64, P,
                                  ctypes.POINTER(_Params), ctypes.POINTER(_EvalOut), P]
        _lib.orc_linesearch_coeffs.argtypes = [P, P, P, ctypes.c_int64, P, P, P, ctypes.c_int64, P, P,
                                               ctypes.POINTER(_Params), ctypes.c_int, P]
        _lib.orc_grad_derivative.argtypes = [P, P, P, ctypes.c_int64, P, P, P, ctypes.c_int64, P,
                                             ctypes.POINTER(_Params), P]
        _lib.orc_num_threads.restype = ctypes.c_int
        _lib.orc_set_threads.argtypes = [ctypes.c_int]
    return _lib


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return lib().orc_num_threads()


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


# ---------------------------------------------------------------------------
# Covariances, Eq. (7b) and the eigenvalue bound of the Remark after Eq. (7).
# ---------------------------------------------------------------------------

def knn_cov(xyz, knn: int = 10):
    """Per-point covariance from the knn nearest points (self included).
    Returns (cov n x 6, neighbour indices n x knn, [d2 of knn-th, d2 of
    (knn+1)-th] n x 2)."""
    x = _d(xyz)
    n = len(x)
    cov = np.zeros((n, 6))
    nbr = np.zeros((n, knn), dtype=np.int64)
    kth = np.zeros((n, 2))
    rc = lib().orc_knn_cov(_ptr(x), n, int(knn), _ptr(cov), _ptr(nbr), _ptr(kth))
    if rc != 0:
        raise ValueError("knn_cov: bad arguments")
    return cov, nbr, kth


def sym3_eig(s):
    s = _d(s)
    lam = np.zeros(3)
    V = np.zeros(9)
    lib().orc_sym3_eig(_ptr(s), _ptr(lam), _ptr(V))
    return lam, V.reshape(3, 3)


def eig_clamp(cov, eig_max: float, eig_ratio: float) -> np.ndarray:
    c = _d(cov).copy()
    lib().orc_eig_clamp(_ptr(c), len(c), float(eig_max), float(eig_ratio))
    return c


def covariances(xyz, knn: int = 10, eig_max: float = 0.0, eig_ratio: float = 100.0) -> np.ndarray:
    cov, _, _ = knn_cov(xyz, knn)
    return eig_clamp(cov, eig_max, eig_ratio) if eig_max > 0 else cov


def max_eig(cov) -> float:
    return float(max(sym3_eig(c)[0].max() for c in _d(cov)))


# ---------------------------------------------------------------------------
# Lie-group helpers (Sec. 2.1, Eq. 3-4).
# ---------------------------------------------------------------------------

def hat3(w) -> np.ndarray:
    w = np.asarray(w, dtype=np.float64)
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


def hat6(xi) -> np.ndarray:
    """4x4 twist matrix of xi = (omega, v)."""
    X = np.zeros((4, 4))
    X[:3, :3] = hat3(xi[:3])
    X[:3, 3] = xi[3:]
    return X


def exp_se3(xi) -> np.ndarray:
    """exp of a twist: Rodrigues for the rotation and the V matrix for the
    translation (standard closed form; the paper does not print one)."""
    xi = np.asarray(xi, dtype=np.float64)
    w, v = xi[:3], xi[3:]
    th = float(np.linalg.norm(w))
    W = hat3(w)
    if th < 1e-4:
        A = 1.0 - th ** 2 / 6.0 + th ** 4 / 120.0
        B = 0.5 - th ** 2 / 24.0 + th ** 4 / 720.0
        C = 1.0 / 6.0 - th ** 2 / 120.0 + th ** 4 / 5040.0
    else:
        A = np.sin(th) / th
        B = (1.0 - np.cos(th)) / th ** 2
        C = (th - np.sin(th)) / th ** 3
    R = np.eye(3) + A * W + B * W @ W
    V = np.eye(3) + B * W + C * W @ W
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = V @ v
    return T


def exp_se3_series(xi, terms: int = 30) -> np.ndarray:
    X = hat6(xi)
    T = np.eye(4)
    P = np.eye(4)
    for k in range(1, terms):
        P = P @ X / k
        T = T + P
    return T


def ad(xi) -> np.ndarray:
    """Eq. (4): ad_xi = [[omega^, 0], [v^, omega^]]."""
    A = np.zeros((6, 6))
    W = hat3(xi[:3])
    A[:3, :3] = W
    A[3:, 3:] = W
    A[3:, :3] = hat3(xi[3:])
    return A


def ad_star(xi) -> np.ndarray:
    """Eq. (4): ad*_xi = [[-omega^, -v^], [0, -omega^]]."""
    A = np.zeros((6, 6))
    W = hat3(xi[:3])
    A[:3, :3] = -W
    A[3:, 3:] = -W
    A[:3, 3:] = -hat3(xi[3:])
    return A


def gamma_vec(u, g) -> np.ndarray:
    """Eq. (3) in vector form: Gamma(U, grad f)^vee =
    1/2 (ad_U g - ad*_U g - ad*_g U)."""
    u = np.asarray(u, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    return 0.5 * (ad(u) @ g - ad_star(u) @ g - ad_star(g) @ u)


def gamma_matrix(g) -> np.ndarray:
    """The 6x6 matrix with Gamma(xi, grad f)^vee = Gamma @ xi, assembled by
    applying the ad / ad* formula of Eq. (3) to the unit vectors."""
    return np.stack([gamma_vec(e, g) for e in np.eye(6)], axis=1)


# ---------------------------------------------------------------------------
# The objective and its derivatives at a pose.
# ---------------------------------------------------------------------------

@dataclass
class KernelParams:
    kernel_mode: int = 0          # 0 anisotropic (Eq. 7), 1 isotropic CVO (Remark 3)
    sigma2: float = 1.0           # amplitude sigma^2 (not given in the paper)
    cutoff: float = 3.0           # keep pairs with d^2 <= cutoff^2; <= 0 keeps all
    iso_ell: float = 0.1
    rho: float = 0.0              # Euclidean radius used only to count pair-evals


@dataclass
class Problem:
    tgt: np.ndarray
    tgt_cov: np.ndarray | None
    tgt_feat: np.ndarray
    src: np.ndarray
    src_cov: np.ndarray | None
    src_feat: np.ndarray

    @staticmethod
    def make(tgt, tgt_cov, tgt_feat, src, src_cov, src_feat) -> "Problem":
        tf = _d(tgt_feat)
        sf = _d(src_feat)
        if tf.ndim == 1:
            tf = tf[:, None]
        if sf.ndim == 1:
            sf = sf[:, None]
        return Problem(_d(tgt), None if tgt_cov is None else _d(tgt_cov), tf,
                       _d(src), None if src_cov is None else _d(src_cov), sf)


@dataclass
class EvalResult:
    f: float
    g: np.ndarray
    M: np.ndarray
    Gamma: np.ndarray
    H: np.ndarray
    gabs: np.ndarray
    n_kept: float
    n_rho: float
    n_near_cut: float
    per_src: np.ndarray | None = None
    f_near: float = 0.0                  # |f| and |g| terms of the pairs within 1e-4 c^2 of the
    g_near: np.ndarray | None = None     # cutoff (Eq. 7), kept or not: a lower-precision cutoff
                                         # test may decide those pairs the other way


def _params(kp: KernelParams, feat_dim: int) -> _Params:
    return _Params(kp.kernel_mode, kp.sigma2, kp.cutoff, kp.iso_ell, feat_dim, kp.rho)


def evaluate(prob: Problem, T, kp: KernelParams, per_src: bool = False) -> EvalResult:
    """f (Eq. 5), g (Lemma 1, Eq. 8), M, Gamma (Eq. 12) and
    H_GN = -M + Gamma (Eq. 11) at pose T, by visiting every pair."""
    T = _d(T)
    P = _params(kp, prob.tgt_feat.shape[1])
    out = _EvalOut()
    ps = np.zeros((len(prob.src), 7)) if per_src else None
    if kp.kernel_mode == 0 and (prob.tgt_cov is None or prob.src_cov is None):
        raise ValueError("anisotropic mode needs covariances")
    rc = lib().orc_eval(_ptr(prob.tgt), _ptr(prob.tgt_cov), _ptr(prob.tgt_feat), len(prob.tgt),
                        _ptr(prob.src), _ptr(prob.src_cov), _ptr(prob.src_feat), len(prob.src),
                        _ptr(T), ctypes.byref(P), ctypes.byref(out), _ptr(ps))
    if rc != 0:
        raise MemoryError("orc_eval")
    g = np.array(out.g[:])
    M = np.array(out.M[:]).reshape(6, 6)
    G = gamma_matrix(g)
    return EvalResult(out.f, g, M, G, -M + G, np.array(out.gabs[:]), out.n_pairs_kept,
                      out.n_pairs_rho, out.n_near_cut, ps, out.f_near, np.array(out.g_near[:]))


def gn_step(res: EvalResult) -> np.ndarray:
    """Eq. (13): xi = -H_GN^{-1} g = (M - Gamma)^{-1} g, by LU with partial
    pivoting (LAPACK gesv)."""
    return np.linalg.solve(-res.H, res.g)


def _sym6_mats(c: np.ndarray) -> np.ndarray:
    """(n, 6) covariances (xx, xy, xz, yy, yz, zz) as (n, 3, 3) matrices."""
    m = np.empty((len(c), 3, 3))
    m[:, 0, 0], m[:, 0, 1], m[:, 0, 2] = c[:, 0], c[:, 1], c[:, 2]
    m[:, 1, 0], m[:, 1, 1], m[:, 1, 2] = c[:, 1], c[:, 3], c[:, 4]
    m[:, 2, 0], m[:, 2, 1], m[:, 2, 2] = c[:, 2], c[:, 4], c[:, 5]
    return m


def grad_derivative(prob: Problem, T, kp: KernelParams, terms: bool = False):
    """G-CVO-E (Sec. 3.4, the directional derivative of Eq. (10) with all
    four terms): the 6x6 matrix D with D @ xi = D(g)[xi], g the gradient of
    Lemma 1, under the right perturbation T exp(xi^).  Per pair, with
    p = R^T (z - t), r = x - p, Sigma' = R^T Sigma_z R, A = (Sigma_x +
    Sigma')^-1, y = A r, w = c_ij sigma^2 exp(-r^T A r / 2) and g = -sum w
    J^T y, J = [-p^, I]:
        dp = -(omega x p + v),  dr = -dp,
        dSigma' = Sigma' omega^ - omega^ Sigma',  dA = -A dSigma' A,
        dw = -w (y . dr + r . dA r / 2),
        D(g) = -sum [dw J^T y + w (dp x y, 0) + w J^T dA r + w J^T A dr].
    The last term alone is -M (the Gauss-Newton part).  Pairs beyond the
    cutoff contribute nothing.  All pairs at once in NumPy (small clouds).
    With terms=True also returns the four terms' matrices."""
    T = _d(T)
    R, t = T[:3, :3], T[:3, 3]
    p = (prob.src - t) @ R                               # rows R^T (z - t)
    r = prob.tgt[:, None, :] - p[None, :, :]             # (nt, ns, 3)
    nt, ns = len(prob.tgt), len(prob.src)
    if kp.kernel_mode == 1:
        Szr = np.zeros((ns, 3, 3))
        Sig = np.broadcast_to(np.eye(3) * kp.iso_ell ** 2, (nt, ns, 3, 3))
    else:
        Szr = np.einsum("ba,nbc,cd->nad", R, _sym6_mats(prob.src_cov), R)
        Sig = _sym6_mats(prob.tgt_cov)[:, None] + Szr[None]
    A = np.linalg.inv(Sig)
    y = np.einsum("ijab,ijb->ija", A, r)
    d2 = np.einsum("ija,ija->ij", r, y)
    cij = prob.tgt_feat @ prob.src_feat.T
    w = cij * kp.sigma2 * np.exp(-0.5 * d2)
    if kp.cutoff > 0:
        w = np.where(d2 <= kp.cutoff ** 2, w, 0.0)
    Jty = np.concatenate([np.cross(p[None], y), y], axis=-1)          # J^T y
    parts = np.zeros((4, 6, 6))
    for k in range(6):
        xi = np.eye(6)[k]
        om, v = xi[:3], xi[3:]
        dp = -(np.cross(om, p) + v)                                   # (ns, 3)
        dr = -dp
        W = hat3(om)
        dS = Szr @ W - W @ Szr                                        # (ns, 3, 3)
        dA = -np.einsum("ijab,jbc,ijcd->ijad", A, dS, A)
        dAr = np.einsum("ijab,ijb->ija", dA, r)
        dw = -w * (np.einsum("ija,ja->ij", y, dr) + 0.5 * np.einsum("ija,ija->ij", r, dAr))
        Adr = np.einsum("ijab,jb->ija", A, dr)
        t1 = dw[..., None] * Jty
        t2 = w[..., None] * np.concatenate([np.cross(dp[None], y), np.zeros_like(y)], axis=-1)
        t3 = w[..., None] * np.concatenate([np.cross(p[None], dAr), dAr], axis=-1)
        t4 = w[..., None] * np.concatenate([np.cross(p[None], Adr), Adr], axis=-1)
        for q, tq in enumerate((t1, t2, t3, t4)):
            parts[q, :, k] = -tq.sum(axis=(0, 1))
    D = parts.sum(axis=0)
    return (D, parts) if terms else D


def grad_derivative_c(prob: Problem, T, kp: KernelParams) -> np.ndarray:
    """The D(g) of grad_derivative (same four terms per pair and unit
    direction), as plain FP64 loops over every pair in gcvo_oracle.c, for
    clouds too large for grad_derivative's (n_t, n_s, 3, 3) arrays."""
    if kp.kernel_mode == 0 and (prob.tgt_cov is None or prob.src_cov is None):
        raise ValueError("anisotropic mode needs covariances")
    P = _params(kp, prob.tgt_feat.shape[1])
    out = np.zeros(36)
    rc = lib().orc_grad_derivative(_ptr(prob.tgt), _ptr(prob.tgt_cov), _ptr(prob.tgt_feat), len(prob.tgt),
                                   _ptr(prob.src), _ptr(prob.src_cov), _ptr(prob.src_feat), len(prob.src),
                                   _ptr(_d(T)), ctypes.byref(P), _ptr(out))
    if rc != 0:
        raise MemoryError("orc_grad_derivative")
    return out.reshape(6, 6)


def exact_step(prob: Problem, T, kp: KernelParams, res: EvalResult) -> np.ndarray:
    """G-CVO-E step: Newton with the exact Riemannian Hessian
    H_E = D(g) + Gamma (Eq. 12), xi = -H_E^-1 g.  D(g) from the C loops
    (pinned equal to grad_derivative's NumPy restatement)."""
    H = grad_derivative_c(prob, T, kp) + res.Gamma
    return np.linalg.solve(-H, res.g)


def linesearch_poly(prob: Problem, T, xi, kp: KernelParams, literal: bool = False) -> np.ndarray:
    """c_k = sum_ij f_ij g^k_ij, k = 0..4, so that G(t) ~ sum_k c_k t^k."""
    P = _params(kp, prob.tgt_feat.shape[1])
    out = np.zeros(5)
    lib().orc_linesearch_coeffs(_ptr(prob.tgt), _ptr(prob.tgt_cov), _ptr(prob.tgt_feat), len(prob.tgt),
                                _ptr(prob.src), _ptr(prob.src_cov), _ptr(prob.src_feat), len(prob.src),
                                _ptr(_d(T)), _ptr(_d(xi)), ctypes.byref(P), int(literal), _ptr(out))
    return out


def linesearch_step(c: np.ndarray, mu0: float) -> float:
    """Eq. (9): t* = the smallest positive real root of G'(t); mu = max(mu0, t*),
    and mu0 when G' has no positive real root."""
    dc = np.array([4.0 * c[4], 3.0 * c[3], 2.0 * c[2], c[1]])   # highest power first
    while len(dc) > 1 and dc[0] == 0.0:
        dc = dc[1:]
    roots = np.roots(dc) if len(dc) > 1 else np.array([])
    real = [r.real for r in roots if abs(r.imag) <= 1e-12 * max(1.0, abs(r.real)) and r.real > 0]
    if not real:
        return mu0
    return max(mu0, min(real))


# ---------------------------------------------------------------------------
# Algorithm 1.
# ---------------------------------------------------------------------------

@dataclass
class IterLog:
    f: float
    g: np.ndarray
    xi: np.ndarray
    xi_l1: float
    T: np.ndarray           # pose at which f and g were evaluated


@dataclass
class RegisterResult:
    T: np.ndarray
    log: list = field(default_factory=list)
    converged: bool = False


def register(prob: Problem, T0, kp: KernelParams, order: int = 2, k_max: int = 200,
             eps_tol: float = 1e-8, mu0: float = 1e-10, literal_ls: bool = False) -> RegisterResult:
    """Alg. 1: repeat {evaluate f, grad f (and H_GN) at T^(k); step xi^(k);
    T^(k+1) = T^(k) exp(xi^(k))} while ||xi^(k)||_1 >= eps_tol and k < k_max.
    order 2: G-CVO-2 (Eq. 13); 1: G-CVO-1 (Eq. 9); 3: G-CVO-E (Newton with
    the exact Hessian).  The first iteration always runs."""
    T = _d(T0).copy()
    out = RegisterResult(T)
    xi_l1 = np.inf
    k = 0
    while xi_l1 >= eps_tol and k < k_max:
        res = evaluate(prob, T, kp)
        if order == 2:
            xi = gn_step(res)
        elif order == 3:
            xi = exact_step(prob, T, kp, res)
        else:
            c = linesearch_poly(prob, T, res.g, kp, literal_ls)
            xi = linesearch_step(c, mu0) * res.g
        xi_l1 = float(np.abs(xi).sum())
        out.log.append(IterLog(res.f, res.g.copy(), xi.copy(), xi_l1, T.copy()))
        T = T @ exp_se3(xi)
        k += 1
    out.T = T
    out.converged = xi_l1 < eps_tol
    return out


# ---------------------------------------------------------------------------
# Comparison helpers used by the parity tests.
# ---------------------------------------------------------------------------

def rot_angle(Ra, Rb) -> float:
    c = (np.trace(np.asarray(Ra) @ np.asarray(Rb).T) - 1.0) / 2.0
    return float(np.arccos(np.clip(c, -1.0, 1.0)))


def pose_error(Ta, Tb):
    Ta, Tb = np.asarray(Ta), np.asarray(Tb)
    return rot_angle(Ta[:3, :3], Tb[:3, :3]), float(np.linalg.norm(Ta[:3, 3] - Tb[:3, 3]))


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
