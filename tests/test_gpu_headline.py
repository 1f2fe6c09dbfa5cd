"""The headline workload in the launch configuration the benchmark times: the
256-problem uneven batch (corner scenes and LiDAR frame pairs of 1k to 40k
points, perturbed starts), one gcvo_register_clouds call with the
autotuned schedule.  Sampled problems -- the largest corner problem, the
largest LiDAR problem and two more -- are checked against the FP64 oracle
at the GPU's own first two iterates: f and g within 1e-5 (allowing for the
pairs within 1e-4 c^2 of the cutoff, which an FP32 and an FP64 cutoff test
may decide differently), with the oracle fed the covariances the GPU
computed for the same clouds."""
import os
import sys

import numpy as np
import pytest

from helpers import TOL, rel_f_near, rel_g_near

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_headline_batch_sampled_against_oracle(oracle_mod):
    import torch
    sys.path.insert(0, ROOT)
    import bench
    from paper_2606_10019_gb300 import build as B
    from paper_2606_10019_gb300 import gcvo as G
    O = oracle_mod
    B.build()
    dev = torch.device("cuda:0")
    ctx = G.gcvo_create(0)
    frames, T_true = bench.make_frames(100, 0)
    batch = bench.batch_problems(frames, T_true, n_problems=256)
    kp_c = G.kernel_params(eig_max=0.01, eig_ratio=100.0, knn=bench.KNN)
    kp_l = G.kernel_params(eig_max=bench.EIG_MAX, eig_ratio=100.0, knn=bench.KNN)
    clouds = [tuple(torch.from_numpy(bench._soa(q[k])).to(dev) for k in ("tx", "tf", "sx", "sf")) for q in batch]
    kps = [kp_c if q["kind"] == "corner" else kp_l for q in batch]
    pairs = [(*c, q["T0"], kp) for c, q, kp in zip(clouds, batch, kps)]
    T, logs, n_iter, st = G.gcvo_register_clouds(ctx, pairs, kp_l, G.solver_params(k_max=2, eps_tol=1e-8),
                                                 want_log=True)
    assert np.all(n_iter == 2)
    size = [q["sx"].shape[0] + q["tx"].shape[0] for q in batch]
    corner = [k for k, q in enumerate(batch) if q["kind"] == "corner"]
    lidar = [k for k, q in enumerate(batch) if q["kind"] != "corner"]
    sample = {max(corner, key=lambda k: size[k]), max(lidar, key=lambda k: size[k]), corner[3], lidar[5]}
    assert max(size[k] for k in sample) > 60000   # the 40k end of the size range is in the sample
    for k in sorted(sample):
        q = batch[k]
        tx, tf, sx, sf = clouds[k]
        tc = torch.empty((6, tx.shape[1]), device=dev)
        sc = torch.empty((6, sx.shape[1]), device=dev)
        # the single-cloud calls give the batch's covariances bit for bit
        G.gcvo_estimate_covariances(ctx, tx, kps[k], tc)
        G.gcvo_estimate_covariances(ctx, sx, kps[k], sc)
        prob = O.Problem.make(q["tx"], tc.cpu().numpy().T.astype(np.float64), q["tf"],
                              q["sx"], sc.cpu().numpy().T.astype(np.float64), q["sf"])
        for it in range(2):
            o = O.evaluate(prob, logs[k][it]["T"], O.KernelParams(cutoff=3.0))
            assert rel_f_near(logs[k][it]["f"], o) <= TOL, (k, it)
            assert rel_g_near(logs[k][it]["g"], o) <= TOL, (k, it, o.n_near_cut)
    ctx.close()
