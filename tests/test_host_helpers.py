"""Host-side helpers that the tests and the benchmark rely on, checked on the
CPU: the pose-error measure, the generators' pose convention (T_true^-1 z
lands on the target surface, Sec. 2.1), and the uneven batch recipe (sizes,
mix and perturbation bounds)."""
import math
import os
import sys

import numpy as np
import pytest
from scipy.spatial import cKDTree
from scipy.spatial.transform import Rotation

from paper_2606_10019_gb300 import datagen as D
from paper_2606_10019_gb300 import proposal_data as PD

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_pose_errors_known_offsets():
    rng = np.random.default_rng(0)
    Ts, Tt, want = [], [], []
    for deg, d in ((0.0, 0.0), (1.5, 0.02), (30.0, 0.5), (179.0, 3.0)):
        T_true = D.rigid(Rotation.from_rotvec(rng.normal(size=3)).as_matrix(), rng.normal(size=3))
        axis = D.random_unit(rng)
        delta = D.rigid(Rotation.from_rotvec(math.radians(deg) * axis).as_matrix(), d * D.random_unit(rng))
        Ts.append(T_true @ delta)
        Tt.append(T_true)
        want.append((deg, d))
    e = PD.pose_errors(Ts, Tt)
    assert np.allclose(e, np.array(want), atol=1e-9)


def _median_nn(src_in_tgt, tgt):
    return float(np.median(cKDTree(tgt).query(src_in_tgt)[0]))


def test_corner_pair_convention():
    pair = D.make_corner_pair(n_src=2000, n_tgt=2000)
    Ti = D.inv_rigid(pair.T_true)
    aligned = _median_nn(D.apply(Ti, pair.src_xyz.astype(np.float64)), pair.tgt_xyz)
    raw = _median_nn(pair.src_xyz.astype(np.float64), pair.tgt_xyz)
    assert aligned < 0.5 * raw
    assert aligned < 0.05


def test_lidar_pair_convention():
    seq = D.LidarSequence(n_frames=2)
    pair = seq.pair(0)
    Ti = D.inv_rigid(pair.T_true)
    aligned = _median_nn(D.apply(Ti, pair.src_xyz.astype(np.float64)), pair.tgt_xyz)
    raw = _median_nn(pair.src_xyz.astype(np.float64), pair.tgt_xyz)
    # voxel centroids of 0.3 m voxels: aligned neighbours sit within a voxel
    assert aligned < 0.3 and aligned < raw


@pytest.mark.slow
def test_uneven_batch_recipe():
    """The headline batch: sizes log-uniform in [1000, 40000] (a LiDAR
    problem is at most a whole frame), corner scenes and LiDAR pairs
    alternating, and each start a motion of at most 30 degrees and 0.5 m
    applied to the truth."""
    sys.path.insert(0, ROOT)
    import bench
    frames, T_true = bench.make_frames(3, 0)
    batch = bench.batch_problems(frames, T_true, n_problems=32)
    assert len(batch) == 32
    kinds = [q["kind"] for q in batch]
    assert kinds[0::2] == ["corner"] * 16 and kinds[1::2] == ["lidar"] * 16
    frame_max = max(len(x) for x, _ in frames)
    for q in batch:
        n = q["sx"].shape[0]
        assert 1000 <= n <= 40000 and q["tx"].shape[0] <= 40000
        if q["kind"] == "lidar":
            assert n <= frame_max
        # T0 = P T_true with P a motion of at most 30 degrees and 0.5 m
        P = q["T0"] @ D.inv_rigid(q["T_true"])
        e = PD.pose_errors([P], [np.eye(4)])[0]
        assert e[0] <= 30.0 + 1e-9 and e[1] <= 0.5 + 1e-9
        assert q["sx"].dtype == np.float32 and q["sx"].shape[1] == 3
