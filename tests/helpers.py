"""Shared helpers of the GPU tests: problem construction from the seeded
generators and the parity measures (relative error definitions)."""
from __future__ import annotations

import numpy as np

TOL = 1e-5   # relative tolerance on f, g, H per evaluation (FP32 pair kernel)
POSE_TOL = 1e-5  # final pose: rad and m


def soa(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32).T)).to(dev)


def rel_f(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def rel_g(g, go, gabs):
    """max |dg| over the largest of |g| and the absolute-sum scale: g cancels
    towards zero at the optimum, its per-pair terms do not."""
    return float(np.abs(np.asarray(g) - go).max() / max(np.abs(go).max(), np.asarray(gabs).max(), 1e-300))


def rel_f_near(f, o):
    """rel_f after taking off the terms of the pairs within 1e-4 c^2 of the
    cutoff (the FP32 cutoff test of the kernel may decide them the other way
    than the FP64 one of the oracle)."""
    return max(0.0, abs(f - o.f) - o.f_near) / max(abs(o.f), 1e-300)


def rel_g_near(g, o):
    """rel_g after taking off, per component, the terms of the pairs within
    1e-4 c^2 of the cutoff."""
    d = np.maximum(np.abs(np.asarray(g) - o.g) - o.g_near, 0.0)
    return float(d.max() / max(np.abs(o.g).max(), np.asarray(o.gabs).max(), 1e-300))


def rel_H(H, Ho):
    return float(np.linalg.norm(np.asarray(H) - Ho) / max(np.linalg.norm(Ho), 1e-300))


class Case:
    """One problem with covariances from the oracle (rounded to float32 and
    fed to both sides, so input rounding is not charged to the kernel)."""

    def __init__(self, O, pair, kp_o, knn=10, eig_max=0.01, eig_ratio=100.0, iso=False):
        self.pair = pair
        self.kp_o = kp_o
        self.iso = iso
        if iso:
            self.tc = np.zeros((len(pair.tgt_xyz), 6), np.float32)
            self.sc = np.zeros((len(pair.src_xyz), 6), np.float32)
        else:
            self.tc = O.covariances(pair.tgt_xyz, knn, eig_max, eig_ratio).astype(np.float32)
            self.sc = O.covariances(pair.src_xyz, knn, eig_max, eig_ratio).astype(np.float32)
        self.prob = O.Problem.make(pair.tgt_xyz, None if iso else self.tc, pair.tgt_feat, pair.src_xyz,
                                   None if iso else self.sc, pair.src_feat)

    def gpu(self, G, ctx, dev, kp):
        p = self.pair
        self.grid = G.gcvo_build_grid(ctx, soa(p.tgt_xyz, dev), None if self.iso else soa(self.tc, dev),
                                      soa(p.tgt_feat, dev), kp)
        self.src = (soa(p.src_xyz, dev), None if self.iso else soa(self.sc, dev), soa(p.src_feat, dev))
        return self
