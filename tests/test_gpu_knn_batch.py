"""Batched kNN covariances (Eq. 7b and the eigenvalue bound after it) through
the C ABI: one call over clouds of very different shapes -- a corner scene,
a voxelised LiDAR frame, a dense ball (the voxel shrinks with density), a
plane with far outliers (their neighbours lie beyond the fine grid's two
shells: the coarse second pass), exact duplicates, a line, a cloud of
exactly knn points -- each compared with the brute-force FP64 oracle, and
with one call per cloud bit for bit; many tiny clouds in one call; a
non-finite point in one cloud; and gcvo_register_clouds with different
kernel parameters per pair against the same pipeline run call by call."""
import numpy as np
import pytest

from helpers import soa
from paper_2606_10019_gb300 import datagen as D

pytestmark = pytest.mark.gpu

# FP32 sums of knn outer products vs FP64, relative (Frobenius) to the raw
# covariance: the clamp of the eigenvalues to [eig_max/100, eig_max] keeps
# the absolute error of the raw sum, so a clamped result much smaller than
# its raw covariance is held to the raw one's scale
COV_TOL = 2e-5


@pytest.fixture(scope="module")
def env(oracle_mod):
    import torch
    from paper_2606_10019_gb300 import build as B
    from paper_2606_10019_gb300 import gcvo as G
    B.build()
    dev = torch.device("cuda:0")
    ctx = G.gcvo_create(0)
    yield oracle_mod, G, ctx, dev
    ctx.close()


def _clouds(knn=10):
    rng = np.random.default_rng(20261204)
    out = {}
    out["corner"] = D.make_corner_pair(n_src=2000, n_tgt=2000, frame=4).src_xyz
    lid = D.LidarSequence(n_frames=1).frame(0)[0]
    out["lidar"] = lid[rng.choice(len(lid), 4000, replace=False)]
    v = rng.normal(size=(3000, 3))
    out["ball"] = 0.04 * v / np.linalg.norm(v, axis=1, keepdims=True) * rng.uniform(0, 1, (3000, 1)) ** (1 / 3)
    plane = np.c_[rng.uniform(-1, 1, (800, 2)), 0.002 * rng.normal(size=800)]
    far = rng.uniform(-60, 60, (12, 3))
    out["plane_far"] = np.r_[plane, far]
    base = rng.uniform(-0.5, 0.5, (300, 3))
    out["triplicates"] = np.repeat(base, 3, axis=0)[rng.permutation(900)]
    t = rng.uniform(-2, 2, 500)
    out["line"] = np.outer(t, np.array([1.0, 2.0, 3.0]) / np.sqrt(14.0))
    out["n_eq_knn"] = rng.uniform(-0.3, 0.3, (knn, 3))
    return {k: np.ascontiguousarray(v, dtype=np.float32) for k, v in out.items()}


def _M(c):
    return np.stack([c[:, [0, 1, 2]], c[:, [1, 3, 4]], c[:, [2, 4, 5]]], 1)


def _norm(c):
    return np.linalg.norm(_M(c), axis=(1, 2))


def _rel_err(c_gpu, c_orc):
    return _norm(c_gpu - c_orc) / np.maximum(_norm(c_orc), 1e-30)


def _check_oracle(O, name, x, c_gpu, knn, eig):
    c_raw, _, kth = O.knn_cov(x, knn)
    c_orc = O.eig_clamp(c_raw, eig, 100.0) if eig > 0 else c_raw
    if name in ("triplicates",):
        ok = np.ones(len(x), dtype=bool)   # ties only between copies of one point
    else:
        if len(x) > knn:
            gap = (kth[:, 1] - kth[:, 0]) / np.maximum(kth[:, 1], 1e-30)
            ok = gap > 1e-5
            assert ok.mean() > 0.9, (name, ok.mean())
        else:
            ok = np.ones(len(x), dtype=bool)   # every point is everyone's neighbour
    err = _rel_err(c_gpu.astype(np.float64), c_orc)
    scale = np.maximum(1.0, _norm(c_raw) / np.maximum(_norm(c_orc), 1e-30))
    err = err / scale
    if eig <= 0:
        # unclamped: a cloud of exactly coincident neighbours has Sigma = 0
        zero = np.linalg.norm(c_orc, axis=1) == 0
        assert np.all(np.abs(c_gpu[zero]) == 0)
        ok &= ~zero
    assert err[ok].max() <= COV_TOL, (name, err[ok].max())


@pytest.mark.parametrize("knn,eig", [(10, 0.01), (16, 0.0), (5, 0.09)])
def test_batched_covariances_mixed_clouds_match_oracle(env, knn, eig):
    import torch
    O, G, ctx, dev = env
    clouds = _clouds(knn)
    names = list(clouds)
    kp = G.kernel_params(knn=knn, eig_max=eig, eig_ratio=100.0)
    xyz = [soa(clouds[k], dev) for k in names]
    cov = [torch.full((6, x.shape[1]), float("nan"), device=dev) for x in xyz]
    G.gcvo_estimate_covariances_batched(ctx, xyz, kp, cov)
    for k, name in enumerate(names):
        c = cov[k].cpu().numpy().T
        assert np.isfinite(c).all(), name
        _check_oracle(O, name, clouds[name], c, knn, eig)
        c1 = torch.full_like(cov[k], float("nan"))
        G.gcvo_estimate_covariances(ctx, xyz[k], kp, c1)
        assert torch.equal(c1, cov[k]), name


def test_batched_covariances_many_tiny_clouds(env):
    """Several hundred small clouds in one call (one grid and key range per
    cloud in one sort)."""
    import torch
    O, G, ctx, dev = env
    rng = np.random.default_rng(77)
    clouds = [np.ascontiguousarray(rng.uniform(-1, 1, (int(rng.integers(10, 80)), 3)) * rng.uniform(0.01, 5.0),
                                   dtype=np.float32) for _ in range(600)]
    kp = G.kernel_params(knn=10, eig_max=0.01)
    xyz = [soa(x, dev) for x in clouds]
    cov = [torch.full((6, x.shape[1]), float("nan"), device=dev) for x in xyz]
    G.gcvo_estimate_covariances_batched(ctx, xyz, kp, cov)
    for k in range(0, 600, 37):
        c = cov[k].cpu().numpy().T
        assert np.isfinite(c).all()
        _check_oracle(O, "tiny", clouds[k], c, 10, 0.01)
        c1 = torch.empty_like(cov[k])
        G.gcvo_estimate_covariances(ctx, xyz[k], kp, c1)
        assert torch.equal(c1, cov[k])


def test_batched_covariances_nonfinite_cloud(env):
    """A NaN in one cloud fails the whole call with GCVO_ERR_NONFINITE; the
    next call on clean clouds is unaffected."""
    import torch
    O, G, ctx, dev = env
    clouds = _clouds()
    good = clouds["corner"]
    bad = clouds["line"].copy()
    bad[123, 2] = np.nan
    kp = G.kernel_params(eig_max=0.01)
    xyz = [soa(good, dev), soa(bad, dev)]
    cov = [torch.empty((6, x.shape[1]), device=dev) for x in xyz]
    with pytest.raises(G.GcvoError) as e:
        G.gcvo_estimate_covariances_batched(ctx, xyz, kp, cov)
    assert e.value.status == G.GCVO_ERR_NONFINITE
    G.gcvo_estimate_covariances_batched(ctx, xyz[:1], kp, cov[:1])
    _check_oracle(O, "corner", good, cov[0].cpu().numpy().T, 10, 0.01)


def test_register_clouds_mixed_params_equal_call_by_call(env):
    """gcvo_register_clouds with a corner pair (knn 10, eig_max 0.01) and a
    LiDAR pair (knn 12, eig_max 0.09) in one call: the poses equal those of
    the same pipeline run call by call (covariances, grids, batched
    registration), bit for bit."""
    import torch
    O, G, ctx, dev = env
    corner = D.make_corner_pair(n_src=1500, n_tgt=1600, frame=6)
    lidar = D.LidarSequence(n_frames=2).pair(0)
    kps = [G.kernel_params(knn=10, eig_max=0.01), G.kernel_params(knn=12, eig_max=0.09)]
    T0 = [np.eye(4), np.eye(4)]
    sp = G.solver_params(k_max=30, eps_tol=1e-7)
    pairs = []
    for p, kp, t0 in zip((corner, lidar), kps, T0):
        pairs.append((soa(p.tgt_xyz, dev), soa(p.tgt_feat, dev), soa(p.src_xyz, dev), soa(p.src_feat, dev), t0, kp))
    Tc, _, nc, stc = G.gcvo_register_clouds(ctx, pairs, kps[0], sp)
    probs = []
    grids = []
    for (tx, tf, sx, sf, t0, kp) in pairs:
        tc = torch.empty((6, tx.shape[1]), device=dev)
        sc = torch.empty((6, sx.shape[1]), device=dev)
        G.gcvo_estimate_covariances(ctx, tx, kp, tc)
        G.gcvo_estimate_covariances(ctx, sx, kp, sc)
        g = G.gcvo_build_grid(ctx, tx, tc, tf, kp)
        grids.append(g)
        probs.append((g, sx, sc, sf, t0))
    Tb, _, nb, stb = G.gcvo_register_batched(ctx, probs, sp)
    assert np.array_equal(nc, nb) and np.array_equal(stc, stb)
    assert np.array_equal(Tc, Tb)
