"""Training and evaluation pairs for the learned initial-pose proposal.

Pairs are drawn from the seeded scene generators (the synthetic corner scene
and, optionally, voxelised frames of the synthetic 64-beam LiDAR trajectory), misaligned by
a random rigid motion (rotation up to max_deg about a random axis,
translation up to max_t), and labelled with the pose plain G-CVO-2 converges
to when started from the true pose (the library does the labelling).
"""
from __future__ import annotations

import numpy as np

from . import datagen as D


def corner_pairs(n_pairs: int, seed: int, n: int = 2000, max_deg: float = 30.0, max_t: float = 0.5):
    """(tgt_xyz, tgt_l, src_xyz, src_l, T_true) per pair; T^-1 z ~ x."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(n_pairs):
        pair = D.make_corner_pair(frame=100000 * seed + b, n_src=n, n_tgt=n)
        G = D.perturb(rng, max_deg, max_t)
        src = D.apply(G, pair.src_xyz.astype(np.float64)).astype(np.float32)
        out.append((pair.tgt_xyz, pair.tgt_feat[:, 0].copy(), src, pair.src_feat[:, 0].copy(), G @ pair.T_true))
    return out


def lidar_pairs(seq: "D.LidarSequence", n_pairs: int, seed: int, n: int = 4096, max_deg: float = 30.0,
                max_t: float = 0.5):
    """Consecutive-frame pairs of a LiDAR sequence, subsampled to n points,
    with an extra random misalignment."""
    rng = np.random.default_rng(seed)
    out = []
    nf = len(seq.poses) - 1
    for b in range(n_pairs):
        k = int(rng.integers(0, nf))
        pair = seq.pair(k)
        tx, tf = D.subsample(rng, pair.tgt_xyz, pair.tgt_feat, n)
        sx, sf = D.subsample(rng, pair.src_xyz, pair.src_feat, n)
        if len(tx) < n or len(sx) < n:
            continue
        G = D.perturb(rng, max_deg, max_t)
        sx = D.apply(G, sx.astype(np.float64)).astype(np.float32)
        out.append((tx, tf[:, 0].copy(), sx, sf[:, 0].copy(), G @ pair.T_true))
    return out


def to_device(pairs, dev):
    """Batched tensors: src xyz (B, 3, n), src l (B, n), tgt xyz, tgt l."""
    import torch
    sx = torch.tensor(np.stack([p[2].T for p in pairs]), dtype=torch.float32, device=dev).contiguous()
    sf = torch.tensor(np.stack([p[3] for p in pairs]), dtype=torch.float32, device=dev).contiguous()
    tx = torch.tensor(np.stack([p[0].T for p in pairs]), dtype=torch.float32, device=dev).contiguous()
    tf = torch.tensor(np.stack([p[1] for p in pairs]), dtype=torch.float32, device=dev).contiguous()
    return sx, sf, tx, tf


def problems(G, ctx, kp, batch, T0s, dev):
    """gcvo_problem tuples (covariances and target grids built on the GPU)
    for a batch from to_device; the returned list keeps the buffers alive."""
    import torch
    sx, sf, tx, tf = batch
    n = sx.shape[2]
    probs, keep = [], []
    for k in range(sx.shape[0]):
        tc = torch.empty((6, n), device=dev)
        sc = torch.empty((6, n), device=dev)
        G.gcvo_estimate_covariances(ctx, tx[k], kp, tc)
        G.gcvo_estimate_covariances(ctx, sx[k], kp, sc)
        g = G.gcvo_build_grid(ctx, tx[k], tc, tf[k:k + 1], kp)
        probs.append((g, sx[k], sc, sf[k:k + 1], T0s[k]))
        keep.append((tc, sc, g))
    return probs, keep


def pose_errors(Ts, T_true):
    """Rotation (degrees) and translation (m) error of each pose."""
    from scipy.spatial.transform import Rotation
    e = []
    for T, Tt in zip(Ts, T_true):
        Dm = np.linalg.inv(Tt) @ T
        e.append((np.degrees(np.linalg.norm(Rotation.from_matrix(Dm[:3, :3]).as_rotvec())),
                  float(np.linalg.norm(Dm[:3, 3]))))
    return np.array(e)


def _corner_job(args):
    seed, b0, b1, n, max_deg, max_t = args
    rng = np.random.default_rng([seed, b0])
    out = []
    for b in range(b0, b1):
        pair = D.make_corner_pair(frame=100000 * seed + b, n_src=n, n_tgt=n)
        G = D.perturb(rng, max_deg, max_t)
        src = D.apply(G, pair.src_xyz.astype(np.float64)).astype(np.float32)
        out.append((pair.tgt_xyz, pair.tgt_feat[:, 0].copy(), src, pair.src_feat[:, 0].copy(), G @ pair.T_true))
    return out


_FRAMES = None


def set_frames(frames, T_true_frames):
    """Pool initialiser: the LiDAR frames the LiDAR jobs draw from."""
    global _FRAMES
    _FRAMES = (frames, T_true_frames)


def _lidar_job(args):
    seed, b0, b1, n, max_deg, max_t = args
    frames, T_true_frames = _FRAMES
    rng = np.random.default_rng([seed, b0, 1])
    out = []
    while len(out) < b1 - b0:
        j = int(rng.integers(0, len(frames) - 1))
        tx, tf = D.subsample(rng, frames[j][0], frames[j][1], n)
        sx, sf = D.subsample(rng, frames[j + 1][0], frames[j + 1][1], n)
        if len(tx) < n or len(sx) < n:
            continue
        G = D.perturb(rng, max_deg, max_t)
        sx = D.apply(G, sx.astype(np.float64)).astype(np.float32)
        out.append((tx, tf[:, 0].copy(), sx, sf[:, 0].copy(), G @ T_true_frames[j]))
    return out


def mixed_pairs(frames, T_true_frames, n_pairs: int, seed: int, n: int = 4096, max_deg: float = 30.0,
                max_t: float = 0.5, pool=None):
    """The proposal training data: n_pairs pairs of n points, alternately a corner
    scene and a consecutive LiDAR frame pair (frames: list of (xyz, l) with
    the true relative poses T_true_frames) subsampled to n points, each
    misaligned by a random motion up to max_deg / max_t.  Returns (pairs,
    kinds) with pairs as in corner_pairs and kinds 0 (corner) / 1 (LiDAR).
    The work runs in chunks on `pool` when given (a process pool whose
    initialiser is set_frames(frames, T_true_frames))."""
    n_c = (n_pairs + 1) // 2
    n_l = n_pairs - n_c
    cj = [(seed, b, min(b + 512, n_c), n, max_deg, max_t) for b in range(0, n_c, 512)]
    lj = [(seed, b, min(b + 512, n_l), n, max_deg, max_t) for b in range(0, n_l, 512)]
    if pool is not None:
        corner = [p for c in pool.map(_corner_job, cj) for p in c]
        lidar = [p for c in pool.map(_lidar_job, lj) for p in c]
    else:
        set_frames(frames, T_true_frames)
        corner = [p for j in cj for p in _corner_job(j)]
        lidar = [p for j in lj for p in _lidar_job(j)]
    pairs = [None] * n_pairs
    kinds = np.zeros(n_pairs, dtype=np.int32)
    pairs[0::2] = corner
    pairs[1::2] = lidar
    kinds[1::2] = 1
    return pairs, kinds


def mixed_pair_chunks(n_pairs: int, seed: int, n: int = 4096, chunk: int = 512, max_deg: float = 30.0,
                      max_t: float = 0.5, pool=None):
    """mixed_pairs in chunks, in order: yields (pairs, kinds) of up to
    `chunk` pairs, alternately corner and LiDAR pairs, drawn on `pool` (a
    process pool initialised with set_frames) so that no more than a few
    chunks are ever held on the host."""
    jobs = []
    for c0 in range(0, n_pairs, chunk):
        m = min(chunk, n_pairs - c0)
        nc = (m + 1) // 2
        # corner and LiDAR draws numbered by their position in the whole set
        jobs.append((("c", (seed, c0 // 2, c0 // 2 + nc, n, max_deg, max_t)),
                     ("l", (seed, c0 // 2, c0 // 2 + m - nc, n, max_deg, max_t))))
    flat = [j for pair in jobs for j in pair]
    run = lambda j: _corner_job(j[1]) if j[0] == "c" else _lidar_job(j[1])
    it = pool.imap(_run_job, flat) if pool is not None else map(run, flat)
    for _ in jobs:
        corner, lidar = next(it), next(it)
        m = len(corner) + len(lidar)
        pairs = [None] * m
        pairs[0::2] = corner
        pairs[1::2] = lidar
        kinds = np.zeros(m, dtype=np.int32)
        kinds[1::2] = 1
        yield pairs, kinds


def _run_job(j):
    return _corner_job(j[1]) if j[0] == "c" else _lidar_job(j[1])
