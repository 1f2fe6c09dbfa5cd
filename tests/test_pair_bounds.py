"""The bounds the pair kernel relies on to skip work, checked on random
covariances in the clamped range of the Remark after Eq. (7) (eigenvalues in
[lam_hi / kappa, lam_hi]).  No GPU: these are the inequalities themselves.

- rho: a pair with d^2 <= c^2 (Eq. 7) has |r|^2 <= c^2 lambda_max(Sigma_ij)
  <= c^2 (lambda_max(Sigma_i) + lambda_max(Sigma'_j)), so the Euclidean
  radius rho^2 = c^2 (lam_max,X + lam_max,Z) misses no kept pair.
- the per-pair bound: lambda_max(Sigma_ij) <= |Sigma_i|_F + |Sigma'_j|_F, so
  a pair with |r|^2 > c^2 (|Sigma_i|_F + |Sigma'_j|_F) cannot be kept; a
  sub-tile may use the largest |Sigma_i|_F of its points and the distance
  from its bounding box, both of which only loosen the test.
- double-float r: moving x and p by up to u = 2^-24 R each (FP32 rounding at
  distance R) moves d^2 by at most about 4 c u / sigma_min for a pair near
  the cutoff, sigma_min^2 the smallest eigenvalue of Sigma_ij.
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation


def _spd(rng, n, lam_hi, kappa):
    R = Rotation.random(n, random_state=rng).as_matrix()
    lam = lam_hi / kappa * np.exp(rng.uniform(0.0, np.log(kappa), size=(n, 3)))
    # a share of the matrices sit on the clamp bounds exactly
    lam[: n // 4, 0] = lam_hi / kappa
    lam[: n // 4, 1] = lam_hi
    return np.einsum("nij,nj,nkj->nik", R, lam, R), lam


@pytest.mark.parametrize("lam_hi", [0.01, 0.09])
def test_kept_pairs_lie_within_rho(lam_hi):
    rng = np.random.default_rng(1)
    c = 3.0
    A, la = _spd(rng, 4000, lam_hi, 100.0)
    B, lb = _spd(rng, 4000, lam_hi, 100.0)
    S = A + B
    rho2 = c * c * (la.max() + lb.max())
    # the farthest kept r along the weakest direction of Sigma_ij: |r|^2 = c^2 lambda_max
    w, V = np.linalg.eigh(S)
    r = c * np.sqrt(w[:, -1])[:, None] * V[:, :, -1]
    d2 = np.einsum("ni,nij,nj->n", r, np.linalg.inv(S), r)
    assert np.allclose(d2, c * c, rtol=1e-9)
    assert np.all(np.einsum("ni,ni->n", r, r) <= rho2 * (1 + 1e-12))


@pytest.mark.parametrize("lam_hi", [0.01, 0.09])
def test_per_pair_bound_never_drops_a_kept_pair(lam_hi):
    rng = np.random.default_rng(2)
    c = 3.0
    A, _ = _spd(rng, 20000, lam_hi, 100.0)
    B, _ = _spd(rng, 20000, lam_hi, 100.0)
    S = A + B
    fro = np.linalg.norm(A, axis=(1, 2)) + np.linalg.norm(B, axis=(1, 2))
    lmax = np.linalg.eigvalsh(S)[:, -1]
    assert np.all(lmax <= fro * (1 + 1e-12))
    # random r just outside the bound are never kept
    u = rng.normal(size=(20000, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    r = u * (c * np.sqrt(fro) * (1 + 1e-6))[:, None]
    d2 = np.einsum("ni,nij,nj->n", r, np.linalg.inv(S), r)
    assert np.all(d2 > c * c)
    # the bound is tight enough to matter: on flat (surface-like) covariances
    # it is well under the largest-eigenvalue radius rho^2 / c^2
    assert np.median(fro) < 2 * lam_hi


def test_box_distance_is_a_lower_bound():
    """The sub-tile tests a target against its points' bounding box: the box
    distance is at most the distance to every point in it."""
    rng = np.random.default_rng(3)
    for _ in range(200):
        pts = rng.normal(size=(rng.integers(1, 33), 3)) * rng.uniform(0.01, 1.0)
        lo, hi = pts.min(0), pts.max(0)
        x = rng.normal(size=3) * 2.0
        db2 = np.sum(np.maximum(0.0, np.maximum(lo - x, x - hi)) ** 2)
        assert np.all(db2 <= np.sum((pts - x) ** 2, axis=1) * (1 + 1e-12))


def test_position_rounding_bound():
    """First-order change of d^2 = r^T S^-1 r when r moves by e with |e| <=
    2u: |2 e^T S^-1 r| <= 2 |e| |S^-1 r| <= 4 u c / sigma_min for d <= c,
    since |S^-1 r| <= d / sigma_min."""
    rng = np.random.default_rng(4)
    c = 3.0
    A, _ = _spd(rng, 5000, 0.09, 100.0)
    B, _ = _spd(rng, 5000, 0.09, 100.0)
    S = A + B
    w, V = np.linalg.eigh(S)
    smin = np.sqrt(w[:, 0])
    # r on the cutoff ellipsoid, in random directions
    z = rng.normal(size=(5000, 3))
    z /= np.linalg.norm(z, axis=1, keepdims=True)
    L = np.linalg.cholesky(S)
    r = c * np.einsum("nij,nj->ni", L, z)
    R = 60.0
    u = R * 2.0 ** -24
    e = rng.normal(size=(5000, 3))
    e *= (2 * u / np.linalg.norm(e, axis=1))[:, None]
    Si = np.linalg.inv(S)
    d2 = np.einsum("ni,nij,nj->n", r, Si, r)
    d2e = np.einsum("ni,nij,nj->n", r + e, Si, r + e)
    bound = 4 * c * u / smin
    assert np.all(np.abs(d2e - d2) <= bound * 1.01 + 8 * u * u / smin ** 2)
    # and the rule's threshold: at R = 60 m with sigma_min = 4 cm the shift
    # is above 3e-4, so such problems take the tails
    assert 4 * c * R * 2.0 ** -24 / 0.04 > 3e-4
