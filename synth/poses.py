"""Seeded rig poses: one rigid world-frame transform [Q | t] per handle.

A pose is an array ``xf[H, 12]`` holding each handle's 3x4 matrix row-major,
so that a point p moves to ``Q @ p + t``.  The stick-figure poses are built by
forward kinematics over the joint tree (each joint turns its subtree about its
own rest position), so bones stay connected; the root also translates.
"""
from __future__ import annotations

import numpy as np


def rodrigues(axis, angle):
    """Rotation matrix about a unit ``axis`` by ``angle`` radians."""
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0.0, -a[2], a[1]], [a[2], 0.0, -a[0]], [-a[1], a[0], 0.0]])
    return np.eye(3) + np.sin(angle) * K + (1.0 - np.cos(angle)) * (K @ K)


def _pack(Q, t):
    return np.concatenate([Q, np.asarray(t).reshape(3, 1)], axis=1).reshape(12)


def identity_pose(H):
    return np.tile(_pack(np.eye(3), np.zeros(3)), (H, 1))


def rigid_pose(H, Q, t):
    """Every handle carries the same rigid motion."""
    return np.tile(_pack(np.asarray(Q, float), np.asarray(t, float)), (H, 1))


def figure_pose(joints, parent, seed, max_angle_deg=45.0, max_root_shift=0.1):
    """Forward-kinematics pose with a random local turn at every joint.

    For each joint (``numpy.random.default_rng(seed)``): axis ~ normalised
    Gaussian, angle ~ U(-max_angle, max_angle) about the joint's rest position.
    The root additionally shifts by U(-max_root_shift, max_root_shift)^3
    (body height is 1).  Joints must be ordered parents-first.
    """
    joints = np.asarray(joints, dtype=np.float64)
    H = len(joints)
    rng = np.random.default_rng(seed)
    W = np.zeros((H, 4, 4))
    for j in range(H):
        axis = rng.normal(size=3)
        ang = np.deg2rad(rng.uniform(-max_angle_deg, max_angle_deg))
        R = rodrigues(axis, ang)
        L = np.eye(4)
        L[:3, :3] = R
        L[:3, 3] = joints[j] - R @ joints[j]          # turn about the joint
        if parent[j] < 0:
            L[:3, 3] += rng.uniform(-max_root_shift, max_root_shift, size=3)
            W[j] = L
        else:
            assert parent[j] < j, "joints must be ordered parents-first"
            W[j] = W[parent[j]] @ L
    return W[:, :3, :4].reshape(H, 12).copy()


def bar_twist_pose(nx=4, ny=4, nz=16, turn_deg=90.0, shift=0.5):
    """Two-handle bar pose: handle 0 fixed, handle 1 turned about the long axis
    through its end-face centre and shifted along +z."""
    c = np.array([nx / 2.0, ny / 2.0, float(nz)])
    Q = rodrigues([0.0, 0.0, 1.0], np.deg2rad(turn_deg))
    t = c - Q @ c + np.array([0.0, 0.0, shift])
    return np.stack([_pack(np.eye(3), np.zeros(3)), _pack(Q, t)])


def figure_animation(joints, parent, seed, frames, fps=30.0, max_angle_deg=45.0, max_root_shift=0.1):
    """A smooth pose sequence (one animated character) for warm-started solves.

    For each joint (``numpy.random.default_rng(seed)``): a fixed axis ~
    normalised Gaussian, amplitude ~ U(0, max_angle), frequency ~ U(0.3, 1) Hz
    and phase ~ U(0, 2 pi); at frame f (time f / fps) the joint turns by
    amplitude * sin(2 pi frequency t + phase) about its rest position.  The root
    also shifts by max_root_shift * sin(...) per axis with its own frequencies
    and phases.  Returns (frames, H, 12) forward-kinematics transforms.
    """
    joints = np.asarray(joints, dtype=np.float64)
    H = len(joints)
    rng = np.random.default_rng(seed)
    axis = rng.normal(size=(H, 3))
    amp = np.deg2rad(rng.uniform(0.0, max_angle_deg, size=H))
    freq = rng.uniform(0.3, 1.0, size=H)
    phase = rng.uniform(0.0, 2 * np.pi, size=H)
    rfreq = rng.uniform(0.3, 1.0, size=3)
    rphase = rng.uniform(0.0, 2 * np.pi, size=3)
    out = np.zeros((frames, H, 12))
    for f in range(frames):
        t = f / fps
        W = np.zeros((H, 4, 4))
        for j in range(H):
            R = rodrigues(axis[j], amp[j] * np.sin(2 * np.pi * freq[j] * t + phase[j]))
            L = np.eye(4)
            L[:3, :3] = R
            L[:3, 3] = joints[j] - R @ joints[j]
            if parent[j] < 0:
                L[:3, 3] += max_root_shift * np.sin(2 * np.pi * rfreq * t + rphase)
                W[j] = L
            else:
                assert parent[j] < j, "joints must be ordered parents-first"
                W[j] = W[parent[j]] @ L
        out[f] = W[:, :3, :4].reshape(H, 12)
    return out
