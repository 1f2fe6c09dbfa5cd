"""FP64 CPU oracle of the learned initial-pose proposal -- TEST
INFRASTRUCTURE ONLY (tests and the CPU baseline may import it; the library
never does).

The network (a point-set regressor; the paper has no counterpart, it is the
learned-proposal extension of the registration path):
  per point p = (x', y', z', l) of a cloud, with xyz' = (xyz - c) / s where c
  and s are the target cloud's centroid and RMS radius:
      h1 = relu(W1 p + b1)      64
      h2 = relu(W2 h1 + b2)     128
      h3 = W3 h2 + b3           256
  feature of a cloud = max over its points of h3 (per channel);
  u = [feat_src, feat_tgt] (512)
      z1 = relu(H1 u + c1)      256
      z2 = relu(H2 z1 + c2)     128
      out = H3 z2 + c3          6  = normalised twist (omega, v / s)
  loss = mean over the batch of sum_k (out_k - label_k)^2.
Parity status: pinned by central finite differences of the loss
(tests/test_proposal_oracle.py)."""
from __future__ import annotations

import numpy as np

SHAPES = [("W1", (64, 4)), ("b1", (64,)), ("W2", (128, 64)), ("b2", (128,)), ("W3", (256, 128)), ("b3", (256,)),
          ("H1", (256, 512)), ("c1", (256,)), ("H2", (128, 256)), ("c2", (128,)), ("H3", (6, 128)), ("c3", (6,))]


def init_params(seed: int = 0) -> dict:
    """He-uniform weights, zero biases (seeded NumPy generator)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in SHAPES:
        if name[0] in "WH":
            lim = np.sqrt(6.0 / shp[1])
            p[name] = rng.uniform(-lim, lim, size=shp)
        else:
            p[name] = np.zeros(shp)
    return p


def normalise(tgt_xyz, tgt_feat, src_xyz, src_feat):
    """Point tensors (n, 4) of both clouds in the target's normalised frame,
    and (c, s)."""
    tx = np.asarray(tgt_xyz, dtype=np.float64)
    c = tx.mean(axis=0)
    s = np.sqrt(((tx - c) ** 2).sum(axis=1).mean()) + 1e-6
    pt = np.c_[(tx - c) / s, np.asarray(tgt_feat, dtype=np.float64)[:, :1]]
    ps = np.c_[(np.asarray(src_xyz, dtype=np.float64) - c) / s, np.asarray(src_feat, dtype=np.float64)[:, :1]]
    return pt, ps, c, s


def cloud_feature(p, P):
    """Max-pooled per-point MLP feature (256) and the cache for backward."""
    a1 = P @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    h3 = h2 @ p["W3"].T + p["b3"]
    arg = np.argmax(h3, axis=0)            # ties: lowest point index
    feat = h3[arg, np.arange(h3.shape[1])]
    return feat, (P, a1, h1, a2, h2, arg)


def forward(p, batch):
    """batch: list of (P_src (n,4), P_tgt (n,4)).  Returns out (B, 6) and
    the caches."""
    outs, caches = [], []
    for Ps, Pt in batch:
        fs, cs = cloud_feature(p, Ps)
        ft, ct = cloud_feature(p, Pt)
        u = np.r_[fs, ft]
        y1 = p["H1"] @ u + p["c1"]
        z1 = np.maximum(y1, 0.0)
        y2 = p["H2"] @ z1 + p["c2"]
        z2 = np.maximum(y2, 0.0)
        out = p["H3"] @ z2 + p["c3"]
        outs.append(out)
        caches.append((cs, ct, u, y1, z1, y2, z2))
    return np.array(outs), caches


def loss_and_grad(p, batch, labels):
    out, caches = forward(p, batch)
    B = len(batch)
    diff = out - labels
    loss = float((diff ** 2).sum() / B)
    g = {k: np.zeros_like(v) for k, v in p.items()}
    for b in range(B):
        cs, ct, u, y1, z1, y2, z2 = caches[b]
        d_out = 2.0 * diff[b] / B
        g["H3"] += np.outer(d_out, z2)
        g["c3"] += d_out
        d_z2 = p["H3"].T @ d_out
        d_y2 = d_z2 * (y2 > 0)
        g["H2"] += np.outer(d_y2, z1)
        g["c2"] += d_y2
        d_z1 = p["H2"].T @ d_y2
        d_y1 = d_z1 * (y1 > 0)
        g["H1"] += np.outer(d_y1, u)
        g["c1"] += d_y1
        d_u = p["H1"].T @ d_y1
        for cache, d_feat in ((cs, d_u[:256]), (ct, d_u[256:])):
            P, a1, h1, a2, h2, arg = cache
            # max-pool: the gradient of channel c goes to its argmax point
            d_h3 = np.zeros((P.shape[0], 256))
            d_h3[arg, np.arange(256)] = d_feat
            g["W3"] += d_h3.T @ h2
            g["b3"] += d_h3.sum(axis=0)
            d_a2 = (d_h3 @ p["W3"]) * (a2 > 0)
            g["W2"] += d_a2.T @ h1
            g["b2"] += d_a2.sum(axis=0)
            d_a1 = (d_a2 @ p["W2"]) * (a1 > 0)
            g["W1"] += d_a1.T @ P
            g["b1"] += d_a1.sum(axis=0)
    return loss, g


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) in place; t is the 1-based step."""
    for k in p:
        m[k] = b1 * m[k] + (1 - b1) * g[k]
        v[k] = b2 * v[k] + (1 - b2) * g[k] ** 2
        mh = m[k] / (1 - b1 ** t)
        vh = v[k] / (1 - b2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)


def flat(p) -> np.ndarray:
    """Parameters in the library's flat order."""
    return np.concatenate([np.asarray(p[name]).ravel() for name, _ in SHAPES])


def unflat(v) -> dict:
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(v[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


def se3_log(T) -> np.ndarray:
    """Twist (omega, v) of a rigid transform: rotation vector by scipy, v by
    solving V v = t with V the left Jacobian of SO(3)."""
    from scipy.spatial.transform import Rotation
    w = Rotation.from_matrix(T[:3, :3]).as_rotvec()
    th = np.linalg.norm(w)
    W = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
    if th < 1e-8:
        V = np.eye(3) + 0.5 * W
    else:
        V = np.eye(3) + (1 - np.cos(th)) / th ** 2 * W + (th - np.sin(th)) / th ** 3 * W @ W
    return np.r_[w, np.linalg.solve(V, T[:3, 3])]


def label_twist(T, c, s) -> np.ndarray:
    """Normalised twist of S T S^-1 (S the shift by -c), translation / s."""
    Tc = np.array(T, dtype=np.float64)
    Tc[:3, 3] = T[:3, 3] - c + T[:3, :3] @ c
    xi = se3_log(Tc)
    xi[3:] /= s
    return xi
