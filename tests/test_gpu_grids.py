"""Target grids built in one batch (gcvo_build_grids_batched and the grids
of gcvo_register_clouds) through the C ABI: clouds of different kinds and
sizes (a corner scene, LiDAR frames, a single point, one more than 40000
points), each grid against the one gcvo_build_grid makes of its cloud (the
same points in the same order: evaluations bit for bit) and against the
FP64 oracle; the occupied-voxel count against a host count of the same
voxel assignment; rebuilds in place with other clouds; a non-finite point
in one cloud of the batch."""
import numpy as np
import pytest

from helpers import TOL, Case, rel_H, rel_f, rel_g, soa
from paper_2606_10019_gb300 import datagen as D

pytestmark = pytest.mark.gpu


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


def _host_cells(x, h):
    """Occupied voxels of the grid assignment: o the box centre in FP64,
    x - o rounded to float, corner = float(min - o), floor((x - corner) /
    h) in float, clamped to the box (the assignment the grid documents)."""
    mn, mx = x.min(0).astype(np.float64), x.max(0).astype(np.float64)
    o = 0.5 * (mn + mx)
    corner = (mn - o).astype(np.float32)
    inv_h = np.float32(1.0 / h)
    dims = np.floor((mx - mn) / h).astype(np.int64) + 2
    cv = (x.astype(np.float64) - o).astype(np.float32)
    q = np.floor((cv - corner) * inv_h).astype(np.int64)
    q = np.clip(q, 0, dims - 1)
    return len(np.unique(q, axis=0))


def _clouds():
    rng = np.random.default_rng(11)
    pairs = [D.make_corner_pair(n_src=900, n_tgt=1300, frame=2)]
    seq = D.LidarSequence(n_frames=3)
    for k in (0, 1):
        p = seq.pair(k)
        p.tgt_xyz, p.tgt_feat = D.subsample(rng, p.tgt_xyz, p.tgt_feat, 5000 + 1000 * k)
        p.src_xyz, p.src_feat = D.subsample(rng, p.src_xyz, p.src_feat, 3000)
        pairs.append(p)
    out = [(p.tgt_xyz, p.tgt_feat, p) for p in pairs]
    big = D.make_corner_pair(n_src=2000, n_tgt=41000, frame=7)
    out.append((big.tgt_xyz, big.tgt_feat, big))
    one = np.array([[0.1, -0.2, 0.3]], np.float32)
    out.append((one, np.ones((1, 1), np.float32), None))
    return out


def test_batched_grids_equal_single_and_oracle(env):
    import torch
    O, G, ctx, dev = env
    kp = G.kernel_params(eig_max=0.05)
    clouds = _clouds()
    xyz = [soa(x, dev) for x, _, _ in clouds]
    feat = [soa(f, dev) for _, f, _ in clouds]
    covs = []
    for x in xyz:
        c = torch.empty((6, x.shape[1]), device=dev)
        if x.shape[1] >= kp.knn:
            G.gcvo_estimate_covariances(ctx, x, kp, c)
        else:
            c.zero_()
            c[0] = c[3] = c[5] = 0.01
        covs.append(c)
    grids = G.gcvo_build_grids_batched(ctx, xyz, covs, feat, kp)
    for k, (x, f, pair) in enumerate(clouds):
        g1 = G.gcvo_build_grid(ctx, xyz[k], covs[k], feat[k], kp)
        nb, cb, hb = grids[k].info()
        n1, c1, h1 = g1.info()
        assert (nb, cb, hb) == (n1, c1, h1) and nb == len(x) and 1 <= cb <= nb
        if pair is None:
            continue
        sx, sf = soa(pair.src_xyz, dev), soa(pair.src_feat, dev)
        sc = torch.empty((6, sx.shape[1]), device=dev)
        G.gcvo_estimate_covariances(ctx, sx, kp, sc)
        rb = G.gcvo_eval(ctx, grids[k], sx, sc, sf, pair.T_true)
        r1 = G.gcvo_eval(ctx, g1, sx, sc, sf, pair.T_true)
        assert rb.f == r1.f and np.array_equal(rb.g, r1.g) and np.array_equal(rb.H, r1.H)
        prob = O.Problem.make(x, covs[k].cpu().numpy().T.astype(np.float64), f, pair.src_xyz,
                              sc.cpu().numpy().T.astype(np.float64), pair.src_feat)
        o = O.evaluate(prob, pair.T_true, O.KernelParams(cutoff=3.0))
        assert rel_f(rb.f, o.f) <= TOL and rel_g(rb.g, o.g, o.gabs) <= TOL and rel_H(rb.H, o.H) <= TOL
    # rebuild in place with the clouds rotated by one
    order = [(k + 1) % len(clouds) for k in range(len(clouds))]
    grids = G.gcvo_build_grids_batched(ctx, [xyz[k] for k in order], [covs[k] for k in order],
                                       [feat[k] for k in order], kp, grids)
    for i, k in enumerate(order):
        g1 = G.gcvo_build_grid(ctx, xyz[k], covs[k], feat[k], kp)
        assert grids[i].info() == g1.info()
    # a voxel edge that is a power of two (exact in float, and so its
    # reciprocal): the occupied voxels against the host count
    kp4 = G.kernel_params(eig_max=0.05, cell_size=0.25)
    grids = G.gcvo_build_grids_batched(ctx, xyz, covs, feat, kp4)
    for k, (x, _, _) in enumerate(clouds):
        n, c, h = grids[k].info()
        assert h == 0.25 and c == _host_cells(x, 0.25), k


def test_batched_grids_nonfinite_cloud(env):
    """A NaN coordinate in one cloud fails the call with GCVO_ERR_NONFINITE and
    returns no new grid; the next call builds normally."""
    import torch
    O, G, ctx, dev = env
    kp = G.kernel_params(kernel_mode=1, iso_ell=0.1)
    a = D.make_corner_pair(n_src=300, n_tgt=500, frame=1).tgt_xyz
    b = a.copy()
    b[42, 1] = np.nan
    xyz = [soa(a, dev), soa(b, dev)]
    feat = [torch.ones((1, 500), device=dev)] * 2
    with pytest.raises(G.GcvoError) as e:
        G.gcvo_build_grids_batched(ctx, xyz, None, feat, kp)
    assert e.value.status == G.GCVO_ERR_NONFINITE
    grids = G.gcvo_build_grids_batched(ctx, xyz[:1], None, feat[:1], kp)
    assert grids[0].info()[0] == 500
