"""Pins for the FP64 oracle against facts fixed outside it: library routines
(scipy cKDTree, numpy eigh, scipy expm, scipy cdist), closed forms,
finite differences, invariances and exact recovery of a known transform.

Each test states the passage of the paper it follows.  None of these needs a
GPU.
"""
import math

import numpy as np
import pytest
from scipy.linalg import expm
from scipy.spatial import cKDTree
from scipy.spatial.distance import cdist
from scipy.spatial.transform import Rotation

from paper_2606_10019_gb300 import datagen as D


def _rand_rot(rng, deg):
    return Rotation.from_rotvec(math.radians(deg) * D.random_unit(rng)).as_matrix()


def _small_problem(O, n_t=60, n_s=50, seed=3, aniso=True, feat_dim=1):
    rng = np.random.default_rng(seed)
    tgt = rng.uniform(-0.3, 0.3, size=(n_t, 3))
    src = rng.uniform(-0.3, 0.3, size=(n_s, 3))
    tf = rng.uniform(0.2, 1.0, size=(n_t, feat_dim))
    sf = rng.uniform(0.2, 1.0, size=(n_s, feat_dim))
    tc = sc = None
    if aniso:
        def rand_cov(n):
            out = np.zeros((n, 6))
            for k in range(n):
                Q = _rand_rot(rng, rng.uniform(0, 180))
                L = np.diag(rng.uniform(0.005, 0.05, size=3))
                S = Q @ L @ Q.T
                out[k] = [S[0, 0], S[0, 1], S[0, 2], S[1, 1], S[1, 2], S[2, 2]]
            return out
        tc, sc = rand_cov(n_t), rand_cov(n_s)
    return O.Problem.make(tgt, tc, tf, src, sc, sf)


def _sym(m):
    return np.array([m[0, 0], m[0, 1], m[0, 2], m[1, 1], m[1, 2], m[2, 2]])


def _mat(s):
    return np.array([[s[0], s[1], s[2]], [s[1], s[3], s[4]], [s[2], s[4], s[5]]])


def _frozen_problem(O, prob, T_ref, T_new):
    """The same problem with source covariances re-expressed so that the
    combined Sigma_ij of Eq. (7c) evaluated at T_new equals its value at
    T_ref (the frozen-Sigma convention of Remark 2)."""
    R0, R1 = T_ref[:3, :3], T_new[:3, :3]
    Q = R1 @ R0.T
    sc = np.array([_sym(Q @ _mat(s) @ Q.T) for s in prob.src_cov])
    return O.Problem(prob.tgt, prob.tgt_cov, prob.tgt_feat, prob.src, sc, prob.src_feat)


# --------------------------------------------------------------------------
# Covariances, Eq. (7b) and the Remark after Eq. (7)
# --------------------------------------------------------------------------

def test_knn_sets_match_ckdtree(oracle_mod):
    O = oracle_mod
    rng = np.random.default_rng(0)
    x = rng.normal(size=(400, 3))
    _, nbr, kth = O.knn_cov(x, 10)
    d, idx = cKDTree(x).query(x, k=11)
    ok = 0
    for i in range(len(x)):
        if d[i, 10] - d[i, 9] < 1e-9:      # near-tie at the boundary: skip
            continue
        assert set(nbr[i]) == set(idx[i, :10]), i
        assert abs(kth[i, 0] - d[i, 9] ** 2) < 1e-12
        ok += 1
    assert ok > 390


def test_knn_cov_line_closed_form(oracle_mod):
    """Points k*d*e, k = 0..N-1, on a line: for the end point, N_n = the first
    n points, so Sigma = d^2 n (2n - 1) / 6 e e^T (rank one)."""
    O = oracle_mod
    e = np.array([1.0, 2.0, -2.0]) / 3.0
    d, n = 0.05, 10
    x = np.arange(40)[:, None] * d * e[None, :] + np.array([0.3, -0.1, 2.0])
    cov, _, _ = O.knn_cov(x, n)
    expect = d * d * n * (2 * n - 1) / 6.0 * np.outer(e, e)
    assert np.allclose(_mat(cov[0]), expect, rtol=1e-12, atol=1e-15)


def test_knn_cov_plane_normal(oracle_mod):
    O = oracle_mod
    rng = np.random.default_rng(1)
    R = _rand_rot(rng, 40)
    uv = rng.uniform(-1, 1, size=(300, 2))
    x = np.c_[uv, np.zeros(300)] @ R.T
    cov, _, _ = O.knn_cov(x, 10)
    for s in cov[:50]:
        lam, V = np.linalg.eigh(_mat(s))
        assert lam[0] < 1e-14
        assert abs(abs(V[:, 0] @ R[:, 2]) - 1.0) < 1e-9


def test_knn_cov_rigid_equivariance(oracle_mod):
    O = oracle_mod
    rng = np.random.default_rng(2)
    x = rng.normal(size=(300, 3))
    R = _rand_rot(rng, 70)
    t = rng.normal(size=3)
    c0, _, _ = O.knn_cov(x, 10)
    c1, _, _ = O.knn_cov(x @ R.T + t, 10)
    for a, b in zip(c0, c1):
        assert np.allclose(R @ _mat(a) @ R.T, _mat(b), atol=1e-12)


def test_sym3_eig_vs_numpy(oracle_mod):
    O = oracle_mod
    rng = np.random.default_rng(4)
    for _ in range(50):
        A = rng.normal(size=(3, 3))
        A = A @ A.T
        lam, V = O.sym3_eig(_sym(A))
        lam_ref = np.linalg.eigvalsh(A)
        assert np.allclose(np.sort(lam), lam_ref, rtol=1e-12, atol=1e-13)
        assert np.allclose(V @ np.diag(lam) @ V.T, A, atol=1e-12)
        assert np.allclose(V.T @ V, np.eye(3), atol=1e-12)


def test_eig_clamp(oracle_mod):
    O = oracle_mod
    rng = np.random.default_rng(5)
    covs = []
    for _ in range(30):
        Q = _rand_rot(rng, 120)
        covs.append(_sym(Q @ np.diag(10 ** rng.uniform(-6, 0, size=3)) @ Q.T))
    covs = np.array(covs)
    out = O.eig_clamp(covs, 0.01, 100.0)
    for a, b in zip(covs, out):
        la, Va = np.linalg.eigh(_mat(a))
        lb = np.linalg.eigvalsh(_mat(b))
        assert np.allclose(lb, np.clip(la, 1e-4, 0.01), rtol=1e-10)
        # eigenvectors are kept: the clamped matrix commutes with the original
        assert np.allclose(_mat(a) @ _mat(b), _mat(b) @ _mat(a), atol=1e-12)
    inside = O.eig_clamp(np.array([_sym(np.diag([0.001, 0.002, 0.005]))]), 0.01, 100.0)
    assert np.allclose(inside[0], _sym(np.diag([0.001, 0.002, 0.005])))


# --------------------------------------------------------------------------
# Lie-group pieces: exp (Sec. 2.1) and the connection (Eq. 3, 4, 12)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("scale", [0.0, 1e-9, 1e-5, 1e-2, 0.5, 2.5])
def test_exp_matches_expm(oracle_mod, scale):
    O = oracle_mod
    rng = np.random.default_rng(int(scale * 1e6) % 1000)
    xi = rng.normal(size=6) * scale
    xi[3:] = rng.normal(size=3)
    assert np.allclose(O.exp_se3(xi), expm(O.hat6(xi)), atol=1e-13, rtol=1e-12)
    assert np.allclose(O.exp_se3_series(xi, 40), expm(O.hat6(xi)), atol=1e-12)


def test_gamma_is_levi_civita(oracle_mod):
    """For left-invariant fields the Levi-Civita connection of Eq. (3) is
    torsion free (Gamma(U,V) - Gamma(V,U) = [U,V], the 4x4 matrix
    commutator) and compatible with the metric of Eq. (2)."""
    O = oracle_mod
    rng = np.random.default_rng(6)
    for _ in range(20):
        U, V, W = rng.normal(size=(3, 6))
        C = O.hat6(U) @ O.hat6(V) - O.hat6(V) @ O.hat6(U)
        br = np.r_[C[2, 1], C[0, 2], C[1, 0], C[:3, 3]]
        assert np.allclose(O.gamma_vec(U, V) - O.gamma_vec(V, U), br, atol=1e-12)
        assert abs(O.gamma_vec(U, V) @ W + V @ O.gamma_vec(U, W)) < 1e-12


def test_gamma_closed_form_eq12(oracle_mod):
    O = oracle_mod
    rng = np.random.default_rng(7)
    g = rng.normal(size=6)
    G = O.gamma_matrix(g)
    ref = np.zeros((6, 6))
    ref[:3, :3] = -0.5 * O.hat3(g[:3])
    ref[3:, :3] = -O.hat3(g[3:])
    assert np.allclose(G, ref, atol=1e-14)


# --------------------------------------------------------------------------
# Objective (Eq. 5, 7) and derivatives (Lemma 1, Eq. 10-11)
# --------------------------------------------------------------------------

def test_isotropic_objective_vs_cdist(oracle_mod):
    """Remark 3: with Sigma_ij = ell^2 I the objective is a plain Gaussian
    kernel sum weighted by <l_i, l_j>."""
    O = oracle_mod
    prob = _small_problem(O, aniso=False, feat_dim=3)
    rng = np.random.default_rng(8)
    T = D.rigid(_rand_rot(rng, 20), rng.normal(size=3) * 0.1)
    for cutoff in (0.0, 3.0):
        kp = O.KernelParams(kernel_mode=1, sigma2=1.7, cutoff=cutoff, iso_ell=0.15)
        res = O.evaluate(prob, T, kp)
        p = (prob.src - T[:3, 3]) @ T[:3, :3]
        d2 = cdist(prob.tgt, p, "sqeuclidean") / 0.15 ** 2
        K = 1.7 * np.exp(-0.5 * d2) * (prob.tgt_feat @ prob.src_feat.T)
        if cutoff > 0:
            K = K * (d2 <= 9.0)
        assert res.f == pytest.approx(K.sum(), rel=1e-12)


def test_aniso_reduces_to_isotropic(oracle_mod):
    """Eq. (7c) with Sigma_x = Sigma_z = ell^2/2 I gives Sigma_ij = ell^2 I."""
    O = oracle_mod
    prob = _small_problem(O, aniso=False)
    ell = 0.2
    half = np.tile(_sym(np.eye(3) * ell * ell / 2), (len(prob.tgt), 1))
    halfz = np.tile(_sym(np.eye(3) * ell * ell / 2), (len(prob.src), 1))
    pa = O.Problem(prob.tgt, half, prob.tgt_feat, prob.src, halfz, prob.src_feat)
    rng = np.random.default_rng(9)
    T = D.rigid(_rand_rot(rng, 30), rng.normal(size=3) * 0.1)
    r_iso = O.evaluate(prob, T, O.KernelParams(kernel_mode=1, cutoff=0, iso_ell=ell))
    r_an = O.evaluate(pa, T, O.KernelParams(kernel_mode=0, cutoff=0))
    assert r_an.f == pytest.approx(r_iso.f, rel=1e-12)
    assert np.allclose(r_an.g, r_iso.g, rtol=1e-10, atol=1e-12)
    assert np.allclose(r_an.M, r_iso.M, rtol=1e-10, atol=1e-12)


def test_rigid_invariance(oracle_mod):
    """f is unchanged when both clouds move by a common G, with
    T' = G T G^-1 and covariances recomputed by kNN on the moved clouds."""
    O = oracle_mod
    pair = D.make_corner_pair(n_src=300, n_tgt=300)
    rng = np.random.default_rng(10)
    G = D.rigid(_rand_rot(rng, 50), rng.normal(size=3))
    kp = O.KernelParams(cutoff=3.0)
    tc = O.covariances(pair.tgt_xyz, 10, 0.01, 100)
    sc = O.covariances(pair.src_xyz, 10, 0.01, 100)
    p0 = O.Problem.make(pair.tgt_xyz, tc, pair.tgt_feat, pair.src_xyz, sc, pair.src_feat)
    tg, sg = D.apply(G, pair.tgt_xyz.astype(np.float64)), D.apply(G, pair.src_xyz.astype(np.float64))
    p1 = O.Problem.make(tg, O.covariances(tg, 10, 0.01, 100), pair.tgt_feat,
                        sg, O.covariances(sg, 10, 0.01, 100), pair.src_feat)
    T = D.rigid(_rand_rot(rng, 3), rng.normal(size=3) * 0.05)
    a = O.evaluate(p0, T, kp)
    b = O.evaluate(p1, G @ T @ D.inv_rigid(G), kp)
    assert b.f == pytest.approx(a.f, rel=1e-9)
    assert a.n_kept == b.n_kept


def test_permutation_invariance(oracle_mod):
    O = oracle_mod
    prob = _small_problem(O)
    rng = np.random.default_rng(11)
    pt, ps = rng.permutation(len(prob.tgt)), rng.permutation(len(prob.src))
    q = O.Problem(prob.tgt[pt], prob.tgt_cov[pt], prob.tgt_feat[pt], prob.src[ps], prob.src_cov[ps],
                  prob.src_feat[ps])
    T = D.rigid(_rand_rot(rng, 10), rng.normal(size=3) * 0.05)
    kp = O.KernelParams(cutoff=3.0)
    a, b = O.evaluate(prob, T, kp), O.evaluate(q, T, kp)
    assert b.f == pytest.approx(a.f, rel=1e-12)
    assert np.allclose(a.g, b.g, rtol=1e-10, atol=1e-13)
    assert np.allclose(a.M, b.M, rtol=1e-10, atol=1e-13)


def _fd_grad(O, prob, T, kp, h=1e-6, frozen=True):
    g = np.zeros(6)
    for k in range(6):
        e = np.zeros(6)
        e[k] = h
        Tp, Tm = T @ O.exp_se3(e), T @ O.exp_se3(-e)
        pp = _frozen_problem(O, prob, T, Tp) if frozen else prob
        pm = _frozen_problem(O, prob, T, Tm) if frozen else prob
        g[k] = (O.evaluate(pp, Tp, kp).f - O.evaluate(pm, Tm, kp).f) / (2 * h)
    return g


def test_gradient_matches_fd_frozen_sigma(oracle_mod):
    """Lemma 1 is the gradient of the objective with Sigma_ij held at its
    value for the current T (Remark 2); central differences of that frozen
    objective along T exp(t e_k) must reproduce g."""
    O = oracle_mod
    prob = _small_problem(O)
    rng = np.random.default_rng(12)
    T = D.rigid(_rand_rot(rng, 15), rng.normal(size=3) * 0.05)
    kp = O.KernelParams(cutoff=0.0, sigma2=1.3)
    res = O.evaluate(prob, T, kp)
    fd = _fd_grad(O, prob, T, kp)
    assert np.allclose(res.g, fd, rtol=1e-6, atol=1e-7 * np.abs(res.g).max())


def test_isotropic_gradient_is_true_gradient(oracle_mod):
    O = oracle_mod
    prob = _small_problem(O, aniso=False)
    rng = np.random.default_rng(13)
    T = D.rigid(_rand_rot(rng, 15), rng.normal(size=3) * 0.05)
    kp = O.KernelParams(kernel_mode=1, cutoff=0.0, iso_ell=0.2)
    res = O.evaluate(prob, T, kp)
    fd = _fd_grad(O, prob, T, kp, frozen=False)
    assert np.allclose(res.g, fd, rtol=1e-6, atol=1e-7 * np.abs(res.g).max())


def test_gn_matrix_from_fd_of_gradient(oracle_mod):
    """Eq. (10): with Sigma frozen, D(g)[xi] = -(T1 + T2 + M xi) where
    T1 = sum J^T A r D(f_ij)[xi], T2 = sum f_ij D(J^T)[xi] A r.  The two
    terms the Gauss-Newton matrix drops are written out here from their
    definitions; the finite difference of g checks the oracle's M."""
    O = oracle_mod
    prob = _small_problem(O, n_t=25, n_s=20)
    rng = np.random.default_rng(14)
    T = D.rigid(_rand_rot(rng, 10), rng.normal(size=3) * 0.05)
    kp = O.KernelParams(cutoff=0.0)
    res = O.evaluate(prob, T, kp)
    R, t = T[:3, :3], T[:3, 3]
    for trial in range(3):
        xi = rng.normal(size=6)
        h = 1e-6
        Tp, Tm = T @ O.exp_se3(h * xi), T @ O.exp_se3(-h * xi)
        # gradient at the perturbed poses with Sigma_ij frozen at T
        gp = O.evaluate(_frozen_problem(O, prob, T, Tp), Tp, kp).g
        gm = O.evaluate(_frozen_problem(O, prob, T, Tm), Tm, kp).g
        Dg = (gp - gm) / (2 * h)
        T1 = np.zeros(6)
        T2 = np.zeros(6)
        for j in range(len(prob.src)):
            p = R.T @ (prob.src[j] - t)
            J = np.c_[-O.hat3(p), np.eye(3)]
            Jxi = J @ xi
            DJt = np.zeros((6, 3))
            DJt[:3, :] = -O.hat3(Jxi)
            for i in range(len(prob.tgt)):
                Sig = _mat(prob.tgt_cov[i]) + R.T @ _mat(prob.src_cov[j]) @ R
                A = np.linalg.inv(Sig)
                r = prob.tgt[i] - p
                fij = float(prob.tgt_feat[i] @ prob.src_feat[j]) * np.exp(-0.5 * r @ A @ r)
                T1 += J.T @ A @ r * (-fij * r @ A @ Jxi)
                T2 += fij * DJt @ A @ r
        ref = -(T1 + T2 + res.M @ xi)
        assert np.allclose(Dg, ref, rtol=1e-5, atol=1e-6 * np.abs(ref).max())


def test_gn_step_invariant_to_sigma2(oracle_mod):
    """M, g and Gamma all scale with sigma^2 (and a common scale of c_ij), so
    the step of Eq. (13) does not."""
    O = oracle_mod
    prob = _small_problem(O)
    T = np.eye(4)
    a = O.gn_step(O.evaluate(prob, T, O.KernelParams(sigma2=1.0)))
    b = O.gn_step(O.evaluate(prob, T, O.KernelParams(sigma2=37.0)))
    assert np.allclose(a, b, rtol=1e-10, atol=1e-14)


# --------------------------------------------------------------------------
# Algorithm 1: exact recovery where the frozen-Sigma bias vanishes
# --------------------------------------------------------------------------

def test_exact_recovery_isotropic(oracle_mod):
    """With Z = G X (same points and features) and an isotropic kernel, the
    RKHS inner product of Eq. (4) is maximal at T = G (Cauchy-Schwarz), and
    G-CVO-2 must converge there."""
    O = oracle_mod
    pair = D.make_corner_pair(n_src=300, n_tgt=300, noise=0.0)
    rng = np.random.default_rng(15)
    G = D.rigid(_rand_rot(rng, 5), D.random_unit(rng) * 0.1)
    tgt = pair.tgt_xyz.astype(np.float64)
    src = D.apply(G, tgt)
    prob = O.Problem.make(tgt, None, pair.tgt_feat, src, None, pair.tgt_feat)
    kp = O.KernelParams(kernel_mode=1, cutoff=0.0, iso_ell=0.2)
    out = O.register(prob, np.eye(4), kp, order=2, eps_tol=1e-12, k_max=100)
    ang, dt = O.pose_error(out.T, G)
    assert out.converged
    assert ang < 1e-9 and dt < 1e-9


def _spheres(rng, n_per=150):
    pts, covs = [], []
    for c, rad in (([0, 0, 0], 1.0), ([4, 0, 0], 1.4), ([0, 4, 1.5], 0.8)):
        d = rng.normal(size=(n_per, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        pts.append(np.asarray(c) + rad * d)
        for n in d:
            covs.append(_sym(0.002 * np.outer(n, n) + 0.02 * (np.eye(3) - np.outer(n, n))))
    return np.concatenate(pts), np.array(covs)


def test_exact_recovery_spheres_anisotropic(oracle_mod):
    """Points on spheres with covariances built from the exact normals: for a
    pair on one sphere the reflection through their bisecting plane swaps the
    two covariances, so r_ij is an eigenvector of Sigma_ij, the frozen-Sigma
    gradient vanishes at the truth, and G-CVO-2 recovers G exactly."""
    O = oracle_mod
    rng = np.random.default_rng(16)
    tgt, tc = _spheres(rng)
    G = D.rigid(_rand_rot(rng, 3), D.random_unit(rng) * 0.08)
    R = G[:3, :3]
    src = D.apply(G, tgt)
    sc = np.array([_sym(R @ _mat(s) @ R.T) for s in tc])
    feat = np.ones((len(tgt), 1))
    prob = O.Problem.make(tgt, tc, feat, src, sc, feat)
    kp = O.KernelParams(cutoff=3.0)
    assert np.abs(O.evaluate(prob, G, kp).g).max() < 1e-12 * O.evaluate(prob, G, kp).gabs.max()
    out = O.register(prob, np.eye(4), kp, order=2, eps_tol=1e-12, k_max=100)
    ang, dt = O.pose_error(out.T, G)
    assert ang < 1e-9 and dt < 1e-9


def test_loss_slices_single_maximum(oracle_mod):
    """Appendix C: along 1-D slices of the pose around the truth, the
    objective has one maximum, at the truth (isotropic identical-cloud case)."""
    O = oracle_mod
    pair = D.make_corner_pair(n_src=200, n_tgt=200, noise=0.0)
    tgt = pair.tgt_xyz.astype(np.float64)
    G = D.rigid(np.eye(3), np.zeros(3))
    prob = O.Problem.make(tgt, None, pair.tgt_feat, tgt, None, pair.tgt_feat)
    kp = O.KernelParams(kernel_mode=1, cutoff=0.0, iso_ell=0.15)
    for axis in (1, 3, 5):
        ts = np.linspace(-0.5, 0.5, 41) if axis < 3 else np.linspace(-1.0, 1.0, 41)
        fs = []
        for s in ts:
            xi = np.zeros(6)
            xi[axis] = s
            fs.append(O.evaluate(prob, G @ O.exp_se3(xi), kp).f)
        fs = np.array(fs)
        k = int(np.argmax(fs))
        assert k == 20
        assert np.all(np.diff(fs[:k + 1]) > 0) and np.all(np.diff(fs[k:]) < 0)


# --------------------------------------------------------------------------
# G-CVO-1 line search (Eq. 9, Appendix B)
# --------------------------------------------------------------------------

def test_linesearch_polynomial_is_fourth_order(oracle_mod):
    """sum_k c_k t^k must agree with G(t) = f(T exp(t xi)) (Sigma frozen) to
    O(t^5): halving t divides the error by about 32.  The coefficients as
    printed in Appendix B do not (their error is O(t^2))."""
    O = oracle_mod
    prob = _small_problem(O)
    rng = np.random.default_rng(17)
    T = D.rigid(_rand_rot(rng, 5), rng.normal(size=3) * 0.03)
    kp = O.KernelParams(cutoff=0.0)
    xi = rng.normal(size=6)
    xi /= np.linalg.norm(xi)
    c = O.linesearch_poly(prob, T, xi, kp)
    c_lit = O.linesearch_poly(prob, T, xi, kp, literal=True)
    res = O.evaluate(prob, T, kp)
    assert c[0] == pytest.approx(res.f, rel=1e-12)
    assert c[1] == pytest.approx(res.g @ xi, rel=1e-10)

    def G(t):
        Tt = T @ O.exp_se3(t * xi)
        return O.evaluate(_frozen_problem(O, prob, T, Tt), Tt, kp).f

    errs, errs_lit = [], []
    for t in (0.02, 0.01, 0.005):
        poly = sum(c[k] * t ** k for k in range(5))
        poly_l = sum(c_lit[k] * t ** k for k in range(5))
        errs.append(abs(G(t) - poly))
        errs_lit.append(abs(G(t) - poly_l))
    assert 20 < errs[0] / errs[1] < 45 and 20 < errs[1] / errs[2] < 45
    assert errs_lit[1] > 100 * errs[1]


def test_linesearch_root_rule(oracle_mod):
    O = oracle_mod
    # G'(t) = 1 - t^2 (c1 = 1, c3 = -1/3): smallest positive root 1
    assert O.linesearch_step(np.array([0, 1.0, 0, -1.0 / 3.0, 0]), 1e-4) == pytest.approx(1.0)
    # G'(t) = 1 + t^2 > 0: no real root, fall back to mu0
    assert O.linesearch_step(np.array([0, 1.0, 0, 1.0 / 3.0, 0]), 1e-4) == 1e-4
    # G'(t) = (t - 2)(t - 3)(t + 1): smallest positive root 2
    d = np.poly1d([1, -4, 1, 6])
    c = np.array([0, d.c[3], d.c[2] / 2, d.c[1] / 3, d.c[0] / 4])
    assert O.linesearch_step(c, 1e-4) == pytest.approx(2.0)


@pytest.mark.slow
def test_second_order_needs_fewer_iterations(oracle_mod):
    """Sec. 5.4: G-CVO-2 converges in tens of iterations where G-CVO-1 needs
    many more."""
    O = oracle_mod
    pair = D.make_corner_pair(n_src=250, n_tgt=250, noise=0.0)
    tgt = pair.tgt_xyz.astype(np.float64)
    rng = np.random.default_rng(18)
    G = D.rigid(_rand_rot(rng, 5), D.random_unit(rng) * 0.1)
    prob = O.Problem.make(tgt, None, pair.tgt_feat, D.apply(G, tgt), None, pair.tgt_feat)
    kp = O.KernelParams(kernel_mode=1, cutoff=0.0, iso_ell=0.2)
    o2 = O.register(prob, np.eye(4), kp, order=2, eps_tol=1e-7, k_max=200)
    o1 = O.register(prob, np.eye(4), kp, order=1, eps_tol=1e-7, k_max=200, mu0=1e-10)
    e2 = O.pose_error(o2.T, G)
    e1 = O.pose_error(o1.T, G)
    assert o2.converged and len(o2.log) < 50
    assert len(o1.log) > 3 * len(o2.log)
    assert sum(e2) < 1e-6 and sum(e1) < 1e-5


def test_first_order_minimum_step_must_be_small(oracle_mod):
    """Eq. (9) takes mu = max(mu0, t*).  At a fixed point t* ~ 1/lambda of the
    curvature along g, so a minimum step mu0 above about 2/lambda forces an
    overshoot that grows every iteration; a small mu0 keeps G-CVO-1 at the
    fixed point it shares with G-CVO-2 (g = 0)."""
    O = oracle_mod
    pair = D.make_corner_pair(n_src=300, n_tgt=300, frame=2)
    tc = O.covariances(pair.tgt_xyz, 10, 0.01, 100.0)
    sc = O.covariances(pair.src_xyz, 10, 0.01, 100.0)
    prob = O.Problem.make(pair.tgt_xyz, tc, pair.tgt_feat, pair.src_xyz, sc, pair.src_feat)
    kp = O.KernelParams(cutoff=3.0)
    ref = O.register(prob, np.eye(4), kp, order=2, k_max=100, eps_tol=1e-11)
    stay = O.register(prob, ref.T, kp, order=1, k_max=20, eps_tol=0.0, mu0=1e-10)
    assert sum(O.pose_error(stay.T, ref.T)) < 1e-9
    leave = O.register(prob, ref.T, kp, order=1, k_max=20, eps_tol=0.0, mu0=1e-4)
    assert sum(O.pose_error(leave.T, ref.T)) > 1e-3


def _e_problem(O, seed, n_t=70, n_s=60, iso=False):
    rng = np.random.default_rng(seed)
    pair = D.make_corner_pair(frame=900 + seed, n_src=n_s, n_tgt=n_t)
    if iso:
        return O.Problem.make(pair.tgt_xyz, None, pair.tgt_feat, pair.src_xyz, None, pair.src_feat), pair, rng
    tc = O.covariances(pair.tgt_xyz, 10, 0.05, 20.0)
    sc = O.covariances(pair.src_xyz, 10, 0.05, 20.0)
    return O.Problem.make(pair.tgt_xyz, tc, pair.tgt_feat, pair.src_xyz, sc, pair.src_feat), pair, rng


@pytest.mark.parametrize("iso", [False, True])
def test_exact_hessian_matches_fd_of_gradient(oracle_mod, iso):
    """G-CVO-E: D(g)[e_k] against central differences of the Lemma-1
    gradient along T exp(+-h e_k) (dense objective, so no pair crosses a
    cutoff; Sigma' follows the rotation in both), for both restatements of
    D(g): the NumPy one and the C loops."""
    O = oracle_mod
    prob, pair, rng = _e_problem(O, 3, iso=iso)
    kp = O.KernelParams(cutoff=0.0, kernel_mode=1 if iso else 0, iso_ell=0.15)
    T = pair.T_true @ O.exp_se3(rng.normal(size=6) * 0.05)
    h = 1e-5
    for Dg in (O.grad_derivative(prob, T, kp), O.grad_derivative_c(prob, T, kp)):
        for k in range(6):
            e = np.eye(6)[k] * h
            gp = O.evaluate(prob, T @ O.exp_se3(e), kp).g
            gm = O.evaluate(prob, T @ O.exp_se3(-e), kp).g
            fd = (gp - gm) / (2 * h)
            assert np.abs(Dg[:, k] - fd).max() <= 1e-6 * np.abs(Dg).max(), (k, Dg[:, k], fd)


def test_exact_hessian_last_term_is_gauss_newton(oracle_mod):
    """Of the four terms of D(g), the one in D(r) alone is -M of Eq. (11)
    (computed independently by the C oracle); the others are not zero for an
    anisotropic kernel away from the optimum."""
    O = oracle_mod
    prob, pair, rng = _e_problem(O, 4)
    kp = O.KernelParams(cutoff=3.0)
    T = pair.T_true @ O.exp_se3(rng.normal(size=6) * 0.05)
    D, parts = O.grad_derivative(prob, T, kp, terms=True)
    M = O.evaluate(prob, T, kp).M
    assert np.allclose(parts[3], -M, rtol=1e-10, atol=1e-12 * np.abs(M).max())
    assert np.abs(parts[0] + parts[1] + parts[2]).max() > 1e-3 * np.abs(M).max()


def test_gcvo_e_reaches_the_gcvo2_solution(oracle_mod):
    """Sec. 5.4: G-CVO-E (exact Hessian) and G-CVO-2 (Gauss-Newton) share the
    stationary point; started near it, Newton with the exact Hessian
    converges there in a few iterations."""
    O = oracle_mod
    prob, pair, rng = _e_problem(O, 5, n_t=120, n_s=110)
    kp = O.KernelParams(cutoff=0.0)
    ref = O.register(prob, np.eye(4), kp, order=2, k_max=200, eps_tol=1e-12)
    start = ref.T @ O.exp_se3(rng.normal(size=6) * 0.01)
    e = O.register(prob, start, kp, order=3, k_max=30, eps_tol=1e-12)
    # compare the matrices: an arccos angle cannot resolve below ~1e-8 rad
    assert np.abs(e.T - ref.T).max() < 1e-9, (np.abs(e.T - ref.T).max(), len(e.log))
    assert len(e.log) < 15


def test_exact_hessian_isotropic_is_self_adjoint(oracle_mod):
    """Sec. 2 / Eq. (12): the Riemannian Hessian of the Levi-Civita
    connection is self-adjoint, so in the orthonormal left-invariant
    coordinates D(g) + Gamma is symmetric at every pose, not only at a
    critical point.  With the isotropic kernel Lemma 1's g is the true
    gradient of f, and the identity holds to rounding; with Gamma's sign
    flipped, or Gamma left out, it fails.  (With the anisotropic kernel g
    freezes Sigma_ij (Remark 2), is not a gradient field, and the identity
    does not apply.)"""
    O = oracle_mod
    prob, pair, rng = _e_problem(O, 6, iso=True)
    kp = O.KernelParams(cutoff=0.0, kernel_mode=1, iso_ell=0.15)
    for T in (np.eye(4), pair.T_true @ O.exp_se3(rng.normal(size=6) * 0.2)):
        Dg = O.grad_derivative(prob, T, kp)
        G = O.evaluate(prob, T, kp).Gamma
        H = Dg + G
        n = np.abs(H).max()
        assert np.abs(H - H.T).max() <= 1e-12 * n
        for wrong in (Dg - G, Dg):
            assert np.abs(wrong - wrong.T).max() > 1e-3 * n


@pytest.mark.parametrize("mode", ["aniso_cutoff", "aniso_dense", "iso_cutoff"])
def test_exact_hessian_c_loops_equal_numpy(oracle_mod, mode):
    """The C restatement of D(g) (for full-size clouds) equals the NumPy one
    to rounding, with and without the cutoff and for both kernels."""
    O = oracle_mod
    iso = mode.startswith("iso")
    prob, pair, rng = _e_problem(O, 7, iso=iso)
    kp = O.KernelParams(cutoff=0.0 if mode.endswith("dense") else 3.0, kernel_mode=1 if iso else 0, iso_ell=0.15)
    for T in (np.eye(4), pair.T_true @ O.exp_se3(rng.normal(size=6) * 0.05)):
        a = O.grad_derivative(prob, T, kp)
        b = O.grad_derivative_c(prob, T, kp)
        assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def test_label_features_are_a_sum_over_classes(oracle_mod):
    """Eq. (5) with label features (SemanticCVO, Remark 3): c_ij = <l_i, l_j>
    over l channels.  With one-hot labels over 6 classes, c_ij is 1 for
    pairs of the same class and 0 otherwise, so f, g and M equal the sums of
    the one-channel problems restricted to each class's points (a plausible
    slip -- reading one channel, or the channels of the wrong point --
    breaks this)."""
    O = oracle_mod
    rng = np.random.default_rng(11)
    base = _small_problem(O, n_t=90, n_s=80, seed=5)
    L = 6
    lt = rng.integers(0, L, size=90)
    ls = rng.integers(0, L, size=80)
    onehot = lambda lab: np.eye(L)[lab]
    prob = O.Problem.make(base.tgt, base.tgt_cov, onehot(lt), base.src, base.src_cov, onehot(ls))
    T = D.rigid(_rand_rot(rng, 4.0), rng.normal(size=3) * 0.02)
    kp = O.KernelParams(cutoff=3.0)
    full = O.evaluate(prob, T, kp)
    f = 0.0
    g = np.zeros(6)
    M = np.zeros((6, 6))
    for c in range(L):
        it, js = lt == c, ls == c
        if not it.any() or not js.any():
            continue
        sub = O.Problem.make(base.tgt[it], base.tgt_cov[it], np.ones((it.sum(), 1)), base.src[js], base.src_cov[js],
                             np.ones((js.sum(), 1)))
        r = O.evaluate(sub, T, kp)
        f += r.f
        g += r.g
        M += r.M
    assert full.f == pytest.approx(f, rel=1e-12)
    assert np.allclose(full.g, g, rtol=1e-11, atol=1e-12 * np.abs(g).max())
    assert np.allclose(full.M, M, rtol=1e-11, atol=1e-12 * np.abs(M).max())
    # soft labels: the channels add, c_ij of the sum is the sum of the c_ij
    pt = rng.dirichlet(np.ones(L), size=90)
    ps = rng.dirichlet(np.ones(L), size=80)
    soft = O.evaluate(O.Problem.make(base.tgt, base.tgt_cov, pt, base.src, base.src_cov, ps), T, kp)
    parts = [O.evaluate(O.Problem.make(base.tgt, base.tgt_cov, pt[:, [c]], base.src, base.src_cov, ps[:, [c]]), T, kp)
             for c in range(L)]
    assert soft.f == pytest.approx(sum(p.f for p in parts), rel=1e-12)
    assert np.allclose(soft.g, sum(p.g for p in parts), rtol=1e-11, atol=1e-12 * np.abs(soft.g).max())


def test_near_cutoff_terms_single_pair(oracle_mod):
    """The near-cutoff report on one isotropic pair (Remark 3: Sigma_ij =
    ell^2 I, so d^2 = |r|^2 / ell^2), placed just inside, just outside and
    well inside the cutoff c = 3 (Eq. 7: the pair is kept iff d^2 <= c^2):
    f_near and g_near are that pair's own |f_ij| and |g^(ij)| whenever
    |d^2 - c^2| < 1e-4 c^2, kept or not, and zero otherwise; f and g are the
    pair's terms only when it is kept."""
    O = oracle_mod
    ell, c, s2 = 0.5, 3.0, 1.3
    kp = O.KernelParams(kernel_mode=1, sigma2=s2, cutoff=c, iso_ell=ell)
    u = np.array([2.0, -1.0, 2.0]) / 3.0            # unit direction
    p = np.array([[0.4, 0.1, -0.2]])
    lf = np.array([[0.6, 0.8, 0.0]])
    for rel, near, kept in ((-5e-5, True, True), (5e-5, True, False), (-3e-4, False, True)):
        d2 = c * c * (1.0 + rel)
        x = p + ell * np.sqrt(d2) * u
        prob = O.Problem.make(x, None, lf, p, None, lf)
        r = O.evaluate(prob, np.eye(4), kp)
        fij = s2 * 1.0 * np.exp(-0.5 * d2)           # c_ij = <l, l> = 1
        w = (x - p)[0] / ell ** 2                     # Sigma^-1 r
        g_terms = np.r_[-fij * np.cross(p[0], w), -fij * w]
        assert r.n_near_cut == (1 if near else 0)
        assert r.n_kept == (1 if kept else 0)
        assert r.f == pytest.approx(fij if kept else 0.0, rel=1e-12, abs=1e-300)
        assert np.allclose(r.g, g_terms if kept else 0.0, rtol=1e-12, atol=1e-300)
        assert r.f_near == pytest.approx(fij if near else 0.0, rel=1e-12, abs=1e-300)
        assert np.allclose(r.g_near, np.abs(g_terms) if near else 0.0, rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("aniso", [False, True])
def test_pair_counts_brute_force(oracle_mod, aniso):
    """The pair-eval unit: n_rho counts the pairs with |r_ij| <= rho (the
    Euclidean gate before the Mahalanobis test of Eq. 7), for any rho; with
    the isotropic kernel (Remark 3, d^2 = |r|^2 / ell^2) n_kept counts
    |r| <= c ell, and the dense objective (cutoff 0) keeps every pair.
    Counted here by scipy cdist over the source moved by T^-1, so a wrong
    transform direction, a strict inequality or a dropped rho would show."""
    O = oracle_mod
    prob = _small_problem(O, n_t=70, n_s=65, seed=13, aniso=aniso)
    rng = np.random.default_rng(14)
    T = D.rigid(_rand_rot(rng, 25), rng.normal(size=3) * 0.1)
    p = (prob.src - T[:3, 3]) @ T[:3, :3]
    dist = cdist(prob.tgt, p)
    for rho in (0.05, 0.2, float(np.quantile(dist, 0.3)), 2.0):
        mode = dict(kernel_mode=0) if aniso else dict(kernel_mode=1, iso_ell=0.07)
        r = O.evaluate(prob, T, O.KernelParams(cutoff=3.0, rho=rho, **mode))
        assert r.n_rho == np.count_nonzero(dist <= rho)
        if not aniso:
            assert r.n_kept == np.count_nonzero(dist <= 3.0 * 0.07)
        dense = O.evaluate(prob, T, O.KernelParams(cutoff=0.0, rho=rho, **mode))
        assert dense.n_kept == 70 * 65
        assert dense.n_rho == r.n_rho
