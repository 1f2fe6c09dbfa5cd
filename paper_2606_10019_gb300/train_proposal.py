"""Train the learned initial-pose proposal on pairs labelled by plain G-CVO.

  python -m paper_2606_10019_gb300.train_proposal --pairs 4096 --steps 4000 \
      --out proposal.npz [--lidar-frames 0]

Writes the FP32 master parameters (and the training settings) to an .npz
checkpoint; gcvo_proposal_set_params restores them.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def init_params(n_params: int, seed: int) -> np.ndarray:
    """He-uniform weights and zero biases in the library's flat order."""
    rows = [64, 64, 128, 128, 256, 256, 256, 256, 128, 128, 6, 6]
    cols = [4, 1, 64, 1, 128, 1, 512, 1, 256, 1, 128, 1]
    rng = np.random.default_rng(seed)
    out = []
    for k, (r, c) in enumerate(zip(rows, cols)):
        if k % 2 == 0:
            lim = np.sqrt(6.0 / c)
            out.append(rng.uniform(-lim, lim, size=r * c))
        else:
            out.append(np.zeros(r))
    v = np.concatenate(out).astype(np.float32)
    assert v.size == n_params
    return v


def label(G, ctx, kp, pairs, batch, dev, k_max=100, eps=1e-7):
    from . import proposal_data as PD
    probs, keep = PD.problems(G, ctx, kp, batch, [p[4] for p in pairs], dev)
    T, _, n_iter, status = G.gcvo_register_batched(ctx, probs, G.solver_params(k_max=k_max, eps_tol=eps))
    return T, n_iter, status


def train(G, ctx, net, pairs, dev, steps, batch_size=64, lr=1e-3, seed=0, kp=None, log=None):
    """Label the pairs with G-CVO, then run Adam steps on random minibatches
    (learning rate divided by 10 for the last 30 %)."""
    from . import proposal_data as PD
    import torch
    kp = kp or G.kernel_params(eig_max=0.01, eig_ratio=100.0)
    batch = PD.to_device(pairs, dev)
    T_lab, _, _ = label(G, ctx, kp, pairs, batch, dev)
    rng = np.random.default_rng(seed)
    losses = []
    for it in range(steps):
        idx = rng.choice(len(pairs), min(batch_size, len(pairs)), replace=False)
        ti = torch.tensor(idx, device=dev)
        b = [x.index_select(0, ti).contiguous() for x in batch]
        loss, _ = net.train_step(*b, T_lab[idx], lr=lr if it < 0.7 * steps else 0.1 * lr)
        losses.append(loss)
        if log and (it % 500 == 0 or it == steps - 1):
            log(f"step {it} loss {loss:.5f}")
    return losses


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--pairs", type=int, default=4096)
    ap.add_argument("--lidar-frames", type=int, default=0, help="also draw pairs from this many LiDAR frames")
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--out", default="proposal.npz")
    args = ap.parse_args()
    import torch
    from . import build as B
    from . import datagen as D
    from . import gcvo as G
    from . import proposal_data as PD
    B.build()
    dev = torch.device("cuda:0")
    ctx = G.gcvo_create(0)
    net = G.Proposal(ctx)
    net.set_params(init_params(net.n_params, args.seed))
    t0 = time.time()
    pairs = PD.corner_pairs(args.pairs, args.seed)
    if args.lidar_frames > 1:
        seq = D.LidarSequence(n_frames=args.lidar_frames)
        lp = PD.lidar_pairs(seq, args.pairs // 2, args.seed + 1, n=2000)
        pairs = pairs + lp
    losses = train(G, ctx, net, pairs, dev, args.steps, lr=args.lr, seed=args.seed, log=print)
    meta = dict(pairs=len(pairs), steps=args.steps, lr=args.lr, seed=args.seed, seconds=time.time() - t0,
                final_loss=float(np.mean(losses[-50:])))
    np.savez(args.out, params=net.get_params(), meta=json.dumps(meta))
    print(json.dumps(meta))


if __name__ == "__main__":
    main()
