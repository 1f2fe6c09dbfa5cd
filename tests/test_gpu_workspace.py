"""Caller-owned scratch through the C ABI (gcvo_workspace_size /
gcvo_set_workspace): with a workspace set, covariances, grid rebuilds (one
at a time and batched), evaluations and registrations make no device
allocation for their scratch,
give the same results bit for bit as a context with library-owned scratch,
and refuse calls beyond the workspace's limits."""
import numpy as np
import pytest

from helpers import soa
from paper_2606_10019_gb300 import datagen as D

pytestmark = pytest.mark.gpu


def test_workspace_backed_calls_allocate_nothing(oracle_mod):
    import torch
    from paper_2606_10019_gb300 import build as B
    from paper_2606_10019_gb300 import gcvo as G
    B.build()
    dev = torch.device("cuda:0")
    own = G.gcvo_create(0)
    ws_ctx = G.gcvo_create(0)
    N, NP, ROWS = 4000, 2, 2 * 60
    ws = torch.empty(G.gcvo_workspace_size(N, NP, ROWS), dtype=torch.uint8, device=dev)
    G.gcvo_set_workspace(ws_ctx, ws, N, NP, ROWS)
    kp = G.kernel_params(eig_max=0.01)
    sp = G.solver_params(k_max=60, eps_tol=1e-7)
    pairs = [D.make_corner_pair(n_src=1500, n_tgt=1700, frame=f) for f in (1, 2)]
    res = {}
    for name, ctx in (("own", own), ("ws", ws_ctx)):
        G.gcvo_pair_schedule(ctx, 8)
        clouds = []
        for p in pairs:
            tx, sx = soa(p.tgt_xyz, dev), soa(p.src_xyz, dev)
            tf, sf = soa(p.tgt_feat, dev), soa(p.src_feat, dev)
            tc = torch.empty((6, tx.shape[1]), device=dev)
            sc = torch.empty((6, sx.shape[1]), device=dev)
            clouds.append([tx, tc, tf, sx, sc, sf])
        grids = []
        for c in clouds:   # a grid owns its storage: built before the counted calls
            G.gcvo_estimate_covariances(ctx, c[0], kp, c[1])
            grids.append(G.gcvo_build_grid(ctx, c[0], c[1], c[2], kp))
        torch.cuda.synchronize(dev)
        G.gcvo_profile_enable(ctx, True)
        for c, g in zip(clouds, grids):
            G.gcvo_estimate_covariances(ctx, c[0], kp, c[1])
            G.gcvo_estimate_covariances(ctx, c[3], kp, c[4])
            G.gcvo_rebuild_grid(ctx, g, c[0], c[1], c[2], kp)
        # the batched forms: both target clouds (3400 points) in one call each
        G.gcvo_estimate_covariances_batched(ctx, [c[0] for c in clouds], kp, [c[1] for c in clouds])
        G.gcvo_build_grids_batched(ctx, [c[0] for c in clouds], [c[1] for c in clouds], [c[2] for c in clouds],
                                   kp, grids)
        ev = [G.gcvo_eval(ctx, g, c[3], c[4], c[5], np.eye(4)) for c, g in zip(clouds, grids)]
        ex = G.gcvo_eval_exact(ctx, grids[0], clouds[0][3], clouds[0][4], clouds[0][5], np.eye(4))
        one = G.gcvo_register(ctx, grids[0], clouds[0][3], clouds[0][4], clouds[0][5], np.eye(4), sp)
        bat = G.gcvo_register_batched(ctx, [(g, c[3], c[4], c[5], np.eye(4)) for c, g in zip(clouds, grids)], sp,
                                      want_log=True)
        prof = G.gcvo_profile_read(ctx)
        G.gcvo_profile_enable(ctx, False)
        res[name] = (ev, ex, one, bat, prof, grids, clouds)
    assert res["ws"][4]["n_device_allocs"] == 0, res["ws"][4]
    for a, b in zip(res["own"][0], res["ws"][0]):
        assert a.f == b.f and np.array_equal(a.g, b.g) and np.array_equal(a.H, b.H)
    assert np.array_equal(res["own"][1].H, res["ws"][1].H)
    assert np.array_equal(res["own"][2][0], res["ws"][2][0]) and res["own"][2][2] == res["ws"][2][2]
    assert np.array_equal(res["own"][3][0], res["ws"][3][0])
    # beyond the limits: more source points than the workspace was sized for
    big = D.make_corner_pair(n_src=N + 500, n_tgt=800, frame=3)
    grids, clouds = res["ws"][5], res["ws"][6]
    sx = soa(big.src_xyz, dev)
    sc = torch.empty((6, sx.shape[1]), device=dev)
    with pytest.raises(G.GcvoError) as e:
        G.gcvo_estimate_covariances(ws_ctx, sx, kp, sc)
    assert e.value.status == G.GCVO_ERR_WORKSPACE
    # a batched call whose clouds together exceed the limit
    with pytest.raises(G.GcvoError) as e:
        G.gcvo_estimate_covariances_batched(ws_ctx, [clouds[0][0], clouds[1][0], clouds[0][3]], kp,
                                            [clouds[0][1], clouds[1][1], clouds[0][4]])
    assert e.value.status == G.GCVO_ERR_WORKSPACE
    # library-owned scratch again: the same call runs
    G.gcvo_set_workspace(ws_ctx, None)
    G.gcvo_estimate_covariances(ws_ctx, sx, kp, sc)
    r = G.gcvo_eval(ws_ctx, grids[0], sx, sc, soa(big.src_feat, dev), np.eye(4))
    assert np.isfinite(r.f)
    for name in ("own", "ws"):
        for g in res[name][5]:
            g.close()
    ws_ctx.close()
    own.close()
