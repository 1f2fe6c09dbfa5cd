"""G-CVO-E parity cases added after the exact pass was first run on a GPU:
the dense objective, and full-size LiDAR frame pairs (one pair element by
element, and the bench's batched launch on sampled problems), against the
FP64 oracle through the C ABI.  Tolerances as in test_gpu_exact.py: 1e-5
relative on f, g, D(g) and H_E.  The file name makes pytest collect it after
the other GPU suites except the allocation-free one."""
import numpy as np
import pytest

from helpers import TOL, Case, rel_H, rel_f, rel_g, soa
from paper_2606_10019_gb300 import datagen as D
from test_gpu_exact import _check_exact, _poses

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


def test_eval_exact_dense_no_cutoff(env):
    """The exact pass on the paper's dense objective (cutoff 0: every pair,
    Sec. 5.4), anisotropic and isotropic, against the oracle without a
    cutoff; every pair is a pair-eval."""
    O, G, ctx, dev = env
    pair = D.make_corner_pair(n_src=700, n_tgt=900, frame=11)
    aniso = Case(O, pair, O.KernelParams(cutoff=0.0)).gpu(G, ctx, dev, G.kernel_params(eig_max=0.01, cutoff=0.0))
    iso = Case(O, pair, O.KernelParams(kernel_mode=1, iso_ell=0.08, cutoff=0.0), iso=True)
    iso.gpu(G, ctx, dev, G.kernel_params(kernel_mode=1, iso_ell=0.08, cutoff=0.0))
    for key, c in (("aniso_dense", aniso), ("iso_dense", iso)):
        for T in _poses(pair):
            r = _check_exact(O, G, ctx, key, c, T)
            assert r.n_pairs == 700 * 900


@pytest.mark.slow
def test_exact_lidar_frame_pair_full_size(env):
    """Full size: one voxelised LiDAR frame pair of the bench's trajectory
    (about 22k points each, anisotropic, cutoff 3).  f, g, D(g) and H_E of
    the exact pass against the oracle's C loops over every pair, at the
    identity and at the true pose."""
    O, G, ctx, dev = env
    pair = D.LidarSequence(n_frames=2).pair(0)
    case = Case(O, pair, O.KernelParams(cutoff=3.0), eig_max=0.09).gpu(G, ctx, dev, G.kernel_params(eig_max=0.09))
    for T in (np.eye(4), pair.T_true):
        r = G.gcvo_eval_exact(ctx, case.grid, *case.src, T)
        o = O.evaluate(case.prob, T, case.kp_o)
        Dm = O.grad_derivative_c(case.prob, T, case.kp_o)
        errs = (rel_f(r.f, o.f), rel_g(r.g, o.g, o.gabs), rel_H(r.D, Dm), rel_H(r.H, Dm + o.Gamma))
        assert max(errs) <= TOL, errs


@pytest.mark.slow
def test_exact_batched_lidar_launch_configuration_sampled(env):
    """The benchmark's G-CVO-E launch configuration -- several full-size
    LiDAR frame pairs in one batched call, schedule left to the autotuner --
    on sampled problems: at the GPU's own iterates, f and g against the
    oracle, and the step against the oracle's Newton system through its
    backward error |H_E xi + g| / (|H_E| |xi| + |g|_abs) (the step itself is
    ill-conditioned along the weakly constrained driving direction)."""
    O, G, ctx, dev = env
    seq = D.LidarSequence(n_frames=5)
    frames = [seq.frame(k) for k in range(5)]
    covs = [O.covariances(x, 10, 0.09, 100.0).astype(np.float32) for x, _ in frames]
    kp = G.kernel_params(eig_max=0.09)
    xyz = [soa(x, dev) for x, _ in frames]
    feat = [soa(f, dev) for _, f in frames]
    cv = [soa(c, dev) for c in covs]
    grids = G.gcvo_build_grids_batched(ctx, xyz[:-1], cv[:-1], feat[:-1], kp)
    probs = [(grids[k], xyz[k + 1], cv[k + 1], feat[k + 1], np.eye(4)) for k in range(4)]
    sp = G.solver_params(order=3, k_max=2, eps_tol=1e-8)
    T, logs, n_iter, st = G.gcvo_register_batched(ctx, probs, sp, want_log=True)
    kp_o = O.KernelParams(cutoff=3.0)
    for k in (0, 3):
        prob = O.Problem.make(frames[k][0], covs[k], frames[k][1], frames[k + 1][0], covs[k + 1], frames[k + 1][1])
        assert n_iter[k] >= 1
        for it in range(min(2, int(n_iter[k]))):
            Tk, xi = logs[k][it]["T"], logs[k][it]["xi"]
            o = O.evaluate(prob, Tk, kp_o)
            assert rel_f(logs[k][it]["f"], o.f) <= TOL
            assert rel_g(logs[k][it]["g"], o.g, o.gabs) <= TOL
            He = O.grad_derivative_c(prob, Tk, kp_o) + o.Gamma
            eta = np.linalg.norm(He @ xi + o.g) / (np.linalg.norm(He) * np.linalg.norm(xi) + np.linalg.norm(o.gabs))
            assert eta <= TOL, (k, it, eta)
