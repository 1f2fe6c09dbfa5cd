"""gcvo_eval_static -- the evaluation for callers that cannot allocate
device memory (a stream another framework is capturing, pool-owned memory,
real-time loops, plug-ins without a context) -- called through the C ABI and
compared with gcvo_eval and the oracle on the same inputs, on calls in a row
(the static scratch keeps the previous call's contents, which must not leak
into the next call).

The file name makes pytest collect it last."""
import numpy as np
import pytest

from helpers import TOL, Case, rel_H, rel_f, rel_g
from paper_2606_10019_gb300 import datagen as D

pytestmark = pytest.mark.gpu


def test_eval_static_matches_eval_on_calls_in_a_row(oracle_mod):
    import torch
    from paper_2606_10019_gb300 import build as B
    from paper_2606_10019_gb300 import gcvo as G
    B.build()
    O = oracle_mod
    dev = torch.device("cuda:0")
    ctx = G.gcvo_create(0)
    big = D.make_corner_pair(n_src=2000, n_tgt=2000)
    small = D.make_corner_pair(n_src=333, n_tgt=1500, frame=5)
    cb = Case(O, big, O.KernelParams(cutoff=3.0)).gpu(G, ctx, dev, G.kernel_params(eig_max=0.01))
    cs = Case(O, small, O.KernelParams(cutoff=3.0)).gpu(G, ctx, dev, G.kernel_params(eig_max=0.01))
    T1 = D.rigid(np.eye(3), np.array([0.03, -0.02, 0.01]))
    # big, then small (stale items of the big call lie beyond the small
    # call's range), then big again at another pose
    for case, T in ((cb, np.eye(4)), (cs, T1), (cb, big.T_true)):
        ref = G.gcvo_eval(ctx, case.grid, *case.src, T)
        o = O.evaluate(case.prob, T, case.kp_o)
        f, g, H = G.gcvo_eval_static(case.grid, *case.src, T)
        for ff, gg, HH in ((ref.f, ref.g, ref.H), (o.f, o.g, o.H)):
            errs = rel_f(f, ff), rel_g(g, gg, o.gabs), rel_H(H, HH)
            assert max(errs) <= TOL, errs
    # more source points than the static scratch holds: a clear refusal
    n = 70000
    with pytest.raises(G.GcvoError) as e:
        G.gcvo_eval_static(cb.grid, torch.zeros((3, n), device=dev), torch.zeros((6, n), device=dev),
                           torch.zeros((1, n), device=dev), np.eye(4))
    assert e.value.status == G.GCVO_ERR_CAPACITY
    ctx.close()
