"""Pins for oracle.rig and oracle.diag: distances by dense sampling, the tie
rule, pin radius by brute force, pose targets, and polar decomposition
properties."""
import numpy as np
import pytest

from oracle import rig, diag
from synth import figure_rig, figure_config, rodrigues


def test_segment_distance_against_dense_sampling(rng):
    a = rng.normal(size=3)
    b = a + rng.normal(size=3)
    P = rng.normal(size=(200, 3)) * 2
    d2 = rig._seg_dist2(P, a, b)
    ts = np.linspace(0, 1, 20001)
    S = a + ts[:, None] * (b - a)
    brute = ((P[:, None, :] - S[None]) ** 2).sum(-1).min(axis=1)
    assert np.allclose(d2, brute, atol=1e-7)


def test_nearest_bone_by_brute_force(rng):
    joints, parent = figure_rig()
    P = rng.uniform([-0.7, -0.15, 0.0], [0.7, 0.15, 1.0], size=(400, 3))
    h = rig.nearest_handle(P, joints, parent, "bone")
    bl = rig.bones(parent)
    ts = np.linspace(0, 1, 4001)
    for k in range(len(P)):
        d = [np.min(np.sum((joints[p] + ts[:, None] * (joints[j] - joints[p]) - P[k]) ** 2, 1))
             for p, j in bl]
        assert bl[int(np.argmin(d))][0] == h[k] or np.sort(d)[1] - np.min(d) < 1e-6


def test_ties_go_to_the_lowest_index():
    joints = np.array([[-1.0, 0, 0], [1.0, 0, 0], [0, 5.0, 0]])
    P = np.array([[0.0, 0, 0], [0.0, 1e-9, 0], [0.3, 0, 0]])
    h = rig.nearest_handle(P, joints, [-1, -1, -1], "joint", scale=1.0)
    assert list(h) == [0, 0, 1]
    # mirror-symmetric bones: point on the symmetry plane goes to the first bone
    joints = np.array([[0, 0, 0.0], [0.5, 0, -1], [-0.5, 0, -1]])
    h = rig.nearest_handle(np.array([[0.0, 0.0, -0.5]]), joints, [-1, 0, 0], "bone", scale=1.0)
    assert h[0] == 0


def test_pins_within_radius_by_brute_force():
    cfg = figure_config(3000, seeds=[])
    X, joints, parent = cfg["X"], cfg["joints"], cfg["parent"]
    r = cfg["pin_radius"]
    verts, hand = rig.select_pins(X, joints, parent, r)
    centres = list(joints) + [0.5 * (joints[p] + joints[j]) for p, j in rig.bones(parent)]
    want = [v for v in range(len(X)) if min(np.linalg.norm(X[v] - c) for c in centres) <= r]
    assert list(verts) == want
    assert len(verts) > 3 * len(joints)
    assert np.array_equal(hand, rig.vertex_handles(X, joints, parent)[verts])


def test_pin_targets_follow_handles(rng):
    X = rng.normal(size=(10, 3))
    Q = np.stack([rodrigues(rng.normal(size=3), 0.7), rodrigues(rng.normal(size=3), -1.2)])
    t = rng.normal(size=(2, 3))
    xf = np.concatenate([Q, t[:, :, None]], axis=2).reshape(2, 12)
    Qu, tu = rig.unpack_pose(xf)
    assert np.array_equal(Qu, Q) and np.array_equal(tu, t)
    pv = np.array([1, 4, 7])
    ph = np.array([0, 1, 1])
    xp = rig.pin_targets(X, pv, ph, Qu, tu)
    for k in range(3):
        assert np.allclose(xp[k], Q[ph[k]] @ X[pv[k]] + t[ph[k]])


@pytest.mark.parametrize("inverted", [False, True])
def test_polar_decomposition_properties(inverted, rng):
    F = rng.normal(size=(40, 3, 3)) + 2 * np.eye(3)
    if inverted:
        F[:, :, 0] *= -1
    R, P = diag.polar(F)
    assert np.allclose(np.einsum("kji,kjl->kil", R, R), np.eye(3))
    assert np.allclose(np.linalg.det(R), 1.0)
    assert np.allclose(P, np.swapaxes(P, 1, 2))
    assert np.allclose(R @ P, F)
    ev = np.linalg.eigvalsh(P)
    detF = np.linalg.det(F)
    assert np.all((ev[:, 0] < 0) == (detF < 0))
    # for a rotation times an SPD matrix the polar factors are recovered exactly
    Q = np.stack([rodrigues(rng.normal(size=3), 1.0) for _ in range(5)])
    A = rng.normal(size=(5, 3, 3))
    Sp = np.einsum("kij,klj->kil", A, A) + np.eye(3)
    R2, P2 = diag.polar(Q @ Sp)
    assert np.allclose(R2, Q) and np.allclose(P2, Sp)


def test_nearest_midpoint_by_brute_force(rng):
    joints, parent = figure_rig()
    P = rng.uniform([-0.7, -0.15, 0.0], [0.7, 0.15, 1.0], size=(300, 3))
    h = rig.nearest_handle(P, joints, parent, "midpoint")
    bl = rig.bones(parent)
    mids = np.array([0.5 * (joints[p] + joints[j]) for p, j in bl])
    d = ((P[:, None, :] - mids[None]) ** 2).sum(-1)
    want = np.array([bl[k][0] for k in d.argmin(axis=1)])
    assert np.array_equal(h, want)
