"""Seeded synthetic inputs for the G-CVO registration path.

This module holds none of the registration method's arithmetic: it only draws
scenes, sensor scans, ground-truth rigid motions and voxel-downsampled clouds.
Both the FP64 oracle (``oracle/``) and the CUDA path consume what it returns,
so it is the one module the two sides share.

Conventions (Sec. 2.1 of the paper): X is the target cloud, Z the new (source)
cloud, and a pose T acts as T x = R x + t.  The registration objective (Eq. 5)
is maximised when T^{-1} z_j lands on the target surface, so every generator
returns ``T_true`` with ``T_true^{-1} z ~ x``.

Seeds: NumPy PCG64, seed = 20260601 + 1000 * stream + frame, with one seed
stream per workload: 1 corner scenes, 2 LiDAR street, 3 RGB-D room, 4 uneven
batches (rank r of a multi-rank run adds 100 r).

The scenes stand in for the paper's datasets (KITTI LiDAR, ETH3D RGB-D,
ModelNet40 and a private racing set), none of which is available here; no item
of any of those datasets is reproduced.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.spatial.transform import Rotation

SEED_BASE = 20260601


def rng_for(stream: int, frame: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + 1000 * stream + frame))


def rigid(R: np.ndarray, t: np.ndarray) -> np.ndarray:
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = t
    return T


def inv_rigid(T: np.ndarray) -> np.ndarray:
    R = T[:3, :3]
    return rigid(R.T, -R.T @ T[:3, 3])


def apply(T: np.ndarray, xyz: np.ndarray) -> np.ndarray:
    return xyz @ T[:3, :3].T + T[:3, 3]


def random_unit(rng: np.random.Generator) -> np.ndarray:
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def random_motion(rng, angle_deg: float, trans: float, exact: bool = True) -> np.ndarray:
    """A rigid motion with a rotation of ``angle_deg`` (or up to it) about a
    random axis and a translation of ``trans`` m (or up to it) along a random
    direction."""
    a = angle_deg if exact else rng.uniform(0.0, angle_deg)
    d = trans if exact else rng.uniform(0.0, trans)
    R = Rotation.from_rotvec(math.radians(a) * random_unit(rng)).as_matrix()
    return rigid(R, d * random_unit(rng))


@dataclass
class Pair:
    """One registration problem: target X, source Z, and T_true (T^-1 z ~ x)."""
    tgt_xyz: np.ndarray          # (N_X, 3) float32
    tgt_feat: np.ndarray         # (N_X, l) float32
    src_xyz: np.ndarray          # (N_Z, 3) float32
    src_feat: np.ndarray         # (N_Z, l) float32
    T_true: np.ndarray           # (4, 4) float64
    meta: dict = field(default_factory=dict)


# ----------------------------------------------------------------------------
# Corner scene: three orthogonal 2 m x 2 m planes forming a corner plus a sphere.
# ----------------------------------------------------------------------------

def sample_corner_scene(rng, n: int, scale: float = 1.0) -> np.ndarray:
    """Area-proportional uniform samples on the planes x=0, y=0, z=0 over
    [0,2]^2 and on a sphere of radius 0.5 centred at (1,1,1); ``scale`` scales
    the whole scene."""
    area = np.array([4.0, 4.0, 4.0, math.pi])
    which = rng.choice(4, size=n, p=area / area.sum())
    u = rng.uniform(0.0, 2.0, size=n)
    v = rng.uniform(0.0, 2.0, size=n)
    out = np.zeros((n, 3))
    m = which == 0
    out[m] = np.stack([np.zeros(m.sum()), u[m], v[m]], 1)
    m = which == 1
    out[m] = np.stack([u[m], np.zeros(m.sum()), v[m]], 1)
    m = which == 2
    out[m] = np.stack([u[m], v[m], np.zeros(m.sum())], 1)
    m = which == 3
    d = rng.normal(size=(m.sum(), 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    out[m] = 1.0 + 0.5 * d
    return out * scale


def make_corner_pair(frame: int = 0, n_src: int = 2000, n_tgt: int = 2000,
                     noise: float = 0.01, angle_deg: float = 5.0, trans: float = 0.2,
                     stream: int = 1, scale: float = 1.0) -> Pair:
    """Corner-scene problem: source = scene sample + noise; target = G (independent
    resample) + fresh noise; T_true = G^{-1}."""
    rng = rng_for(stream, frame)
    G = random_motion(rng, angle_deg, trans)
    s_a = sample_corner_scene(rng, n_src, scale)
    s_b = sample_corner_scene(rng, n_tgt, scale)
    src = s_a + rng.normal(scale=noise, size=s_a.shape)
    tgt = apply(G, s_b) + rng.normal(scale=noise, size=s_b.shape)
    f_src = rng.uniform(0.0, 1.0, size=(n_src, 1))
    f_tgt = rng.uniform(0.0, 1.0, size=(n_tgt, 1))
    return Pair(tgt.astype(np.float32), f_tgt.astype(np.float32),
                src.astype(np.float32), f_src.astype(np.float32),
                inv_rigid(G), dict(kind="corner", G=G))


# ----------------------------------------------------------------------------
# Voxel downsampling (preprocessing the paper counts as IO).
# ----------------------------------------------------------------------------

def voxel_downsample(xyz: np.ndarray, feat: np.ndarray, voxel: float):
    """Centroid of the points (and mean of their features) in each occupied
    voxel of edge ``voxel``; output sorted by voxel key for determinism."""
    key = np.floor(xyz / voxel).astype(np.int64)
    key -= key.min(axis=0)
    dims = key.max(axis=0) + 1
    lin = (key[:, 0] * dims[1] + key[:, 1]) * dims[2] + key[:, 2]
    uniq, inv, cnt = np.unique(lin, return_inverse=True, return_counts=True)
    out = np.zeros((len(uniq), 3))
    np.add.at(out, inv, xyz)
    fo = np.zeros((len(uniq), feat.shape[1]))
    np.add.at(fo, inv, feat)
    return out / cnt[:, None], fo / cnt[:, None]


# ----------------------------------------------------------------------------
# LiDAR street: 64-beam spinning LiDAR in a procedural street.
# ----------------------------------------------------------------------------

@dataclass
class Street:
    boxes_lo: np.ndarray     # (B, 3)
    boxes_hi: np.ndarray     # (B, 3)
    box_int: np.ndarray      # (B,)
    poles: np.ndarray        # (P, 2) centre xy
    crowns: np.ndarray       # (C, 4) tree crowns: centre xyz, radius
    pole_r: float = 0.15
    pole_h: float = 6.0


def make_street(rng, x_min: float = -120.0, x_max: float = 420.0) -> Street:
    """A wide boulevard: two rows of box buildings on each side, set back
    35-50 m and 55-78 m with gaps between them (walls at tens of metres
    give the upper beams returns that fall in separate 0.3 m voxels, so a
    frame keeps about 23k voxel centroids), parked cars along both kerbs,
    poles along the road and a park of porous tree crowns 20-60 m out."""
    lo, hi, it = [], [], []
    for side in (-1.0, 1.0):
        for (a, b) in ((35.0, 50.0), (55.0, 78.0)):
            x = x_min + rng.uniform(0.0, 10.0)
            while x < x_max:
                L = rng.uniform(6.0, 18.0)
                D = rng.uniform(6.0, 14.0)
                H = rng.uniform(10.0, 30.0)
                off = rng.uniform(a, b)
                y0, y1 = (off, off + D) if side > 0 else (-off - D, -off)
                lo.append([x, y0, 0.0])
                hi.append([x + L, y1, H])
                it.append(rng.uniform(0.2, 0.8))
                x += L + rng.uniform(2.0, 8.0)
    # parked cars along both kerbs
    for side in (-1.0, 1.0):
        x = x_min
        while x < x_max:
            x += rng.uniform(2.0, 12.0)
            off = rng.uniform(3.5, 5.0)
            y0, y1 = (off, off + 1.8) if side > 0 else (-off - 1.8, -off)
            lo.append([x, y0, 0.0])
            hi.append([x + 4.2, y1, 1.5])
            it.append(rng.uniform(0.4, 1.0))
            x += 4.2
    poles = []
    for side in (-1.0, 1.0):
        x = x_min + rng.uniform(0.0, 10.0)
        while x < x_max:
            poles.append([x, side * rng.uniform(6.0, 7.5)])
            x += rng.uniform(4.0, 10.0)
    # park trees: a trunk (a pole) and a porous spherical crown
    crowns = []
    for side in (-1.0, 1.0):
        x = x_min + rng.uniform(0.0, 8.0)
        while x < x_max:
            y = side * rng.uniform(20.0, 60.0)
            r = rng.uniform(2.0, 4.0)
            crowns.append([x, y, rng.uniform(2.0, 3.5) + 0.3 * r, r])
            poles.append([x, y])
            x += rng.uniform(2.0, 5.0)
    return Street(np.array(lo), np.array(hi), np.array(it), np.array(poles), np.array(crowns))


LIDAR_ELEV = np.radians(np.linspace(-25.0, 3.0, 64))
LIDAR_AZ = np.radians(np.arange(1800) * 0.2)
LIDAR_HEIGHT = 1.73
LIDAR_RANGE = 80.0


def lidar_scan(street: Street, pose: np.ndarray, rng, outlier_frac: float = 0.01,
               range_noise: float = 0.01):
    """Ray-cast one 64 x 1800 scan from the sensor pose ``pose`` (sensor to
    world, sensor at its origin).  Returns sensor-frame points and intensity
    (per-surface base plus an incidence-angle term, in [0, 1])."""
    el, az = np.meshgrid(LIDAR_ELEV, LIDAR_AZ, indexing="ij")
    d_s = np.stack([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)], -1).reshape(-1, 3)
    R, o = pose[:3, :3], pose[:3, 3]
    d = d_s @ R.T
    n_ray = d.shape[0]
    t_best = np.full(n_ray, np.inf)
    base = np.zeros(n_ray)
    nrm = np.zeros((n_ray, 3))
    # ground plane z = 0
    with np.errstate(divide="ignore", invalid="ignore"):
        tg = np.where(d[:, 2] < -1e-9, -o[2] / d[:, 2], np.inf)
    hit = tg < t_best
    t_best[hit] = tg[hit]
    base[hit] = 0.3
    nrm[hit] = [0.0, 0.0, 1.0]
    # boxes (slab test), only those near the sensor
    near = (street.boxes_lo[:, 0] < o[0] + LIDAR_RANGE) & (street.boxes_hi[:, 0] > o[0] - LIDAR_RANGE)
    inv = np.where(np.abs(d) > 1e-12, 1.0 / np.where(np.abs(d) > 1e-12, d, 1.0), 1e12)
    for b in np.nonzero(near)[0]:
        t0 = (street.boxes_lo[b] - o) * inv
        t1 = (street.boxes_hi[b] - o) * inv
        tmin = np.minimum(t0, t1)
        tmax = np.maximum(t0, t1)
        tn = tmin.max(axis=1)
        tf = tmax.min(axis=1)
        ok = (tn <= tf) & (tn > 1e-6) & (tn < t_best)
        if not ok.any():
            continue
        t_best[ok] = tn[ok]
        base[ok] = street.box_int[b]
        ax = tmin[ok].argmax(axis=1)
        n = np.zeros((ok.sum(), 3))
        n[np.arange(len(ax)), ax] = 1.0
        nrm[ok] = n
    # vertical poles
    near_p = np.abs(street.poles[:, 0] - o[0]) < LIDAR_RANGE
    a = d[:, 0] ** 2 + d[:, 1] ** 2
    for c in street.poles[near_p]:
        ox, oy = o[0] - c[0], o[1] - c[1]
        bq = 2.0 * (ox * d[:, 0] + oy * d[:, 1])
        cq = ox * ox + oy * oy - street.pole_r ** 2
        disc = bq * bq - 4.0 * a * cq
        ok = (disc >= 0) & (a > 1e-12)
        with np.errstate(invalid="ignore", divide="ignore"):
            tc = (-bq - np.sqrt(np.maximum(disc, 0.0))) / (2.0 * np.maximum(a, 1e-12))
        z = o[2] + tc * d[:, 2]
        ok &= (tc > 1e-6) & (tc < t_best) & (z >= 0.0) & (z <= street.pole_h)
        if not ok.any():
            continue
        t_best[ok] = tc[ok]
        base[ok] = 0.9
        p = o + tc[ok, None] * d[ok]
        n = np.stack([p[:, 0] - c[0], p[:, 1] - c[1], np.zeros(ok.sum())], 1) / street.pole_r
        nrm[ok] = n
    # porous crowns: a ray that enters a crown stops at an exponentially
    # distributed depth (mean 0.7 m) if that depth is inside the crown
    near_c = np.abs(street.crowns[:, 0] - o[0]) < LIDAR_RANGE + 5.0
    for c in street.crowns[near_c]:
        oc = o - c[:3]
        bq = d @ oc
        cq = oc @ oc - c[3] ** 2
        disc = bq * bq - cq
        ok = disc > 0
        if not ok.any():
            continue
        sq = np.sqrt(np.maximum(disc, 0.0))
        t_in = np.maximum(-bq - sq, 1e-6)
        t_out = -bq + sq
        th = t_in + rng.exponential(0.7, size=n_ray)
        ok &= (th < t_out) & (th < t_best)
        if not ok.any():
            continue
        t_best[ok] = th[ok]
        base[ok] = 0.15
        nrm[ok] = random_dirs = rng.normal(size=(ok.sum(), 3))
        nrm[ok] /= np.linalg.norm(random_dirs, axis=1, keepdims=True)
    keep = t_best <= LIDAR_RANGE
    t = t_best[keep] + rng.normal(scale=range_noise, size=keep.sum())
    cos_inc = np.abs(np.sum(d[keep] * nrm[keep], axis=1))
    inten = np.clip(0.75 * base[keep] + 0.25 * cos_inc, 0.0, 1.0)
    pts_s = d_s[keep] * t[:, None]
    n_out = int(round(outlier_frac * len(pts_s)))
    lo, hi = pts_s.min(axis=0), pts_s.max(axis=0)
    out = rng.uniform(lo, hi, size=(n_out, 3))
    pts = np.concatenate([pts_s, out], 0)
    inten = np.concatenate([inten, rng.uniform(0.0, 1.0, size=n_out)], 0)
    return pts, inten[:, None]


def lidar_trajectory(rng, n_frames: int) -> list[np.ndarray]:
    """Sensor poses: 1-2 m forward and up to 3 degrees of yaw per frame,
    kept on the street (|y| <= 3 m, |yaw| <= 12 degrees)."""
    x, y, yaw = 0.0, 0.0, 0.0
    poses = []
    for _ in range(n_frames):
        R = Rotation.from_euler("z", yaw).as_matrix()
        poses.append(rigid(R, np.array([x, y, LIDAR_HEIGHT])))
        step = rng.uniform(1.0, 2.0)
        dyaw = math.radians(rng.uniform(-3.0, 3.0))
        if abs(yaw + dyaw) > math.radians(12.0) or abs(y) > 3.0:
            dyaw = -math.copysign(abs(dyaw), yaw if abs(y) <= 3.0 else y)
        yaw += dyaw
        x += step * math.cos(yaw)
        y += step * math.sin(yaw)
    return poses


class LidarSequence:
    """A seeded street and a 100-frame trajectory; frames are
    ray-cast and voxel-downsampled (0.3 m) on demand and cached."""

    def __init__(self, n_frames: int = 100, voxel: float = 0.3, stream: int = 2):
        rng = rng_for(stream, 0)
        self.street = make_street(rng)
        self.poses = lidar_trajectory(rng, n_frames)
        self.voxel = voxel
        self.stream = stream
        self._cache: dict[int, tuple[np.ndarray, np.ndarray]] = {}

    def frame(self, k: int):
        if k not in self._cache:
            rng = rng_for(self.stream, 1 + k)
            pts, inten = lidar_scan(self.street, self.poses[k], rng)
            xyz, f = voxel_downsample(pts, inten, self.voxel)
            self._cache[k] = (xyz.astype(np.float32), f.astype(np.float32))
        return self._cache[k]

    def pair(self, k: int) -> Pair:
        """Target = frame k, source = frame k+1; T_true = W_{k+1}^{-1} W_k."""
        xt, ft = self.frame(k)
        xs, fs = self.frame(k + 1)
        T = inv_rigid(self.poses[k + 1]) @ self.poses[k]
        return Pair(xt, ft, xs, fs, T, dict(kind="lidar", frame=k))


# ----------------------------------------------------------------------------
# RGB-D room: RGB-D frames of a procedural room.
# ----------------------------------------------------------------------------

@dataclass
class Room:
    lo: np.ndarray           # (B, 3) boxes (walls are thin boxes too)
    hi: np.ndarray
    rgb: np.ndarray          # (B, 3)


def make_room(rng) -> Room:
    W, D, H, th = 5.0, 4.0, 2.6, 0.05
    lo = [[-th, -th, -th], [-th, -th, -th], [-th, -th, -th], [W, -th, -th], [-th, D, -th], [-th, -th, H]]
    hi = [[W + th, D + th, 0.0], [0.0, D + th, H + th], [W + th, 0.0, H + th], [W + th, D + th, H + th],
          [W + th, D + th, H + th], [W + th, D + th, H + th]]
    for _ in range(int(rng.integers(6, 11))):
        s = rng.uniform([0.3, 0.3, 0.3], [1.2, 1.2, 1.5])
        c = rng.uniform([0.5, 0.5, 0.0], [W - 0.5, D - 0.5, 0.0])
        lo.append([c[0] - s[0] / 2, c[1] - s[1] / 2, 0.0])
        hi.append([c[0] + s[0] / 2, c[1] + s[1] / 2, s[2]])
    return Room(np.array(lo), np.array(hi), rng.uniform(0.0, 1.0, size=(len(lo), 3)))


def depth_frame(room: Room, pose: np.ndarray, rng, w: int = 640, h: int = 480,
                fx: float = 525.0, cx: float = 319.5, cy: float = 239.5):
    """Render depth and colour (per-surface RGB) by ray casting the room's
    boxes from camera pose ``pose`` (camera to world; camera looks along +z
    with y down), add depth noise N(0, (0.0012 z^2)^2) and back-project."""
    u, v = np.meshgrid(np.arange(w), np.arange(h))
    d_c = np.stack([(u - cx) / fx, (v - cy) / fx, np.ones_like(u, dtype=float)], -1).reshape(-1, 3)
    R, o = pose[:3, :3], pose[:3, 3]
    d = d_c @ R.T
    inv = np.where(np.abs(d) > 1e-12, 1.0 / np.where(np.abs(d) > 1e-12, d, 1.0), 1e12)
    t_best = np.full(len(d), np.inf)
    col = np.zeros((len(d), 3))
    for b in range(len(room.lo)):
        t0 = (room.lo[b] - o) * inv
        t1 = (room.hi[b] - o) * inv
        tn = np.minimum(t0, t1).max(axis=1)
        tf = np.maximum(t0, t1).min(axis=1)
        ok = (tn <= tf) & (tn > 1e-6) & (tn < t_best)
        t_best[ok] = tn[ok]
        col[ok] = room.rgb[b]
    keep = np.isfinite(t_best) & (t_best < 8.0)
    z = t_best[keep]                       # depth along the optical axis (d_c.z = 1)
    z = z + rng.normal(size=z.shape) * 0.0012 * z ** 2
    pts = d_c[keep] * z[:, None]
    return pts, col[keep]


class RgbdSequence:
    """Camera inside the room moving <= 5 cm and <= 4 degrees per
    frame; 2 cm voxel downsampling."""

    def __init__(self, n_frames: int = 20, voxel: float = 0.02, stream: int = 3):
        rng = rng_for(stream, 0)
        self.room = make_room(rng)
        self.voxel = voxel
        self.stream = stream
        yaw = 0.0
        pos = np.array([1.0, 1.2, 1.4])
        R0 = Rotation.from_euler("xyz", [-math.pi / 2 - 0.3, 0.0, -math.pi / 2 + 0.5]).as_matrix()
        self.poses = []
        for _ in range(n_frames):
            Ry = Rotation.from_euler("z", yaw).as_matrix()
            self.poses.append(rigid(Ry @ R0, pos.copy()))
            yaw += math.radians(rng.uniform(-4.0, 4.0)) * 0.9
            step = random_unit(rng) * rng.uniform(0.0, 0.05)
            step[2] *= 0.3
            pos = np.clip(pos + step, [0.6, 0.6, 1.0], [4.4, 3.4, 1.8])
        self._cache = {}

    def frame(self, k: int):
        if k not in self._cache:
            rng = rng_for(self.stream, 1 + k)
            pts, col = depth_frame(self.room, self.poses[k], rng)
            xyz, f = voxel_downsample(pts, col, self.voxel)
            self._cache[k] = (xyz.astype(np.float32), f.astype(np.float32))
        return self._cache[k]

    def pair(self, k: int) -> Pair:
        xt, ft = self.frame(k)
        xs, fs = self.frame(k + 1)
        T = inv_rigid(self.poses[k + 1]) @ self.poses[k]
        return Pair(xt, ft, xs, fs, T, dict(kind="rgbd", frame=k))


# ----------------------------------------------------------------------------
# Batches of problems of uneven size with large perturbations.
# ----------------------------------------------------------------------------

def perturb(rng, max_deg: float = 30.0, max_trans: float = 0.5) -> np.ndarray:
    return random_motion(rng, max_deg, max_trans, exact=False)


def subsample(rng, xyz, feat, n):
    if len(xyz) <= n:
        return xyz, feat
    idx = np.sort(rng.choice(len(xyz), size=n, replace=False))
    return xyz[idx], feat[idx]
