"""gcvo_eval_static -- the evaluation for callers that must not allocate
device memory (an application whose pool owns every device byte, a
real-time loop, a plug-in without a context) -- called through the C ABI
and compared with gcvo_eval and the oracle on the same inputs, on calls in a
row (the static scratch keeps the previous call's contents, which must not
leak into the next call): the anisotropic kernel, the isotropic kernel, the
dense objective without a cutoff, a non-finite input and the size limit.

The file name makes pytest collect it last."""
import numpy as np
import pytest

from helpers import TOL, Case, rel_H, rel_f, rel_g
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


def _check(O, G, ctx, case, T):
    ref = G.gcvo_eval(ctx, case.grid, *case.src, T)
    o = O.evaluate(case.prob, T, case.kp_o)
    f, g, H = G.gcvo_eval_static(case.grid, *case.src, T)
    for ff, gg, HH in ((ref.f, ref.g, ref.H), (o.f, o.g, o.H)):
        errs = rel_f(f, ff), rel_g(g, gg, o.gabs), rel_H(H, HH)
        assert max(errs) <= TOL, errs


def test_eval_static_matches_eval_on_calls_in_a_row(env):
    O, G, ctx, dev = env
    big = D.make_corner_pair(n_src=2000, n_tgt=2000)
    small = D.make_corner_pair(n_src=333, n_tgt=1500, frame=5)
    cb = Case(O, big, O.KernelParams(cutoff=3.0)).gpu(G, ctx, dev, G.kernel_params(eig_max=0.01))
    cs = Case(O, small, O.KernelParams(cutoff=3.0)).gpu(G, ctx, dev, G.kernel_params(eig_max=0.01))
    T1 = D.rigid(np.eye(3), np.array([0.03, -0.02, 0.01]))
    # big, then small (stale items of the big call lie beyond the small
    # call's range), then big again at another pose
    for case, T in ((cb, np.eye(4)), (cs, T1), (cb, big.T_true)):
        _check(O, G, ctx, case, T)
    # more source points than the static scratch holds: a clear refusal
    n = 70000
    with pytest.raises(G.GcvoError) as e:
        G.gcvo_eval_static(cb.grid, torch_zeros(dev, 3, n), torch_zeros(dev, 6, n), torch_zeros(dev, 1, n),
                           np.eye(4))
    assert e.value.status == G.GCVO_ERR_CAPACITY


def torch_zeros(dev, r, n):
    import torch
    return torch.zeros((r, n), device=dev)


def test_eval_static_isotropic_and_dense(env):
    """The isotropic kernel (no covariances, Remark 3) and the dense
    objective (cutoff 0: every pair), each twice in a row."""
    O, G, ctx, dev = env
    pair = D.make_corner_pair(n_src=700, n_tgt=800, frame=2)
    iso = Case(O, pair, O.KernelParams(kernel_mode=1, iso_ell=0.08, cutoff=3.0), iso=True)
    iso.gpu(G, ctx, dev, G.kernel_params(kernel_mode=1, iso_ell=0.08))
    dense = Case(O, pair, O.KernelParams(cutoff=0.0)).gpu(G, ctx, dev, G.kernel_params(eig_max=0.01, cutoff=0.0))
    T1 = D.rigid(np.eye(3), np.array([0.01, 0.02, -0.01]))
    for case in (iso, dense, iso, dense):
        for T in (np.eye(4), T1):
            _check(O, G, ctx, case, T)


def test_eval_static_nonfinite_input(env):
    """A NaN coordinate is refused with GCVO_ERR_NONFINITE, and the next call
    on clean inputs is unaffected."""
    O, G, ctx, dev = env
    pair = D.make_corner_pair(n_src=500, n_tgt=500, frame=3)
    case = Case(O, pair, O.KernelParams(cutoff=3.0)).gpu(G, ctx, dev, G.kernel_params(eig_max=0.01))
    bad = case.src[0].clone()
    bad[1, 17] = float("nan")
    with pytest.raises(G.GcvoError) as e:
        G.gcvo_eval_static(case.grid, bad, case.src[1], case.src[2], np.eye(4))
    assert e.value.status == G.GCVO_ERR_NONFINITE
    _check(O, G, ctx, case, np.eye(4))
