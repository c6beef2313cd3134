"""Checks of the seeded input generators (sizes, orientation, conformity)."""
import os

import numpy as np
import pytest

from synth import (bar_mesh, bar_twist_config, figure_pose, figure_rig, kuhn_voxel_mesh,
                   lame_from_young, SNH_E, SNH_NU)
from oracle import element

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split()
                vals[k] = float(v)
    return vals


def test_bar_counts_match_the_stated_workload():
    g = _read_golden("bar_4x4x16_counts.txt")
    X, T = bar_mesh()
    assert len(X) == g["verts"] and len(T) == g["tets"]
    # 3x3-block nonzeros of the vertex graph: diagonal plus both directions of every edge
    e = set()
    for t in T:
        for a in range(4):
            for b in range(a + 1, 4):
                e.add((min(t[a], t[b]), max(t[a], t[b])))
    # edges of the Kuhn grid: axis edges, one diagonal per square face, one per cube
    nx, ny, nz = 4, 4, 16
    axis = nx * (ny + 1) * (nz + 1) + (nx + 1) * ny * (nz + 1) + (nx + 1) * (ny + 1) * nz
    face = nx * ny * (nz + 1) + nx * (ny + 1) * nz + (nx + 1) * ny * nz
    assert len(e) == axis + face + nx * ny * nz
    assert len(X) + 2 * len(e) == 4921


def test_kuhn_mesh_is_positive_and_conforming(rng):
    occ = rng.uniform(size=(4, 3, 5)) < 0.6
    X, T = kuhn_voxel_mesh(occ)
    _, vol, _, _ = element.rest_shape(X, T)
    assert np.all(vol > 0)
    assert np.isclose(vol.sum(), occ.sum())
    faces = {}
    for t in T:
        for drop in range(4):
            f = tuple(sorted(np.delete(t, drop)))
            faces[f] = faces.get(f, 0) + 1
    assert max(faces.values()) <= 2             # a face is shared by at most two tets


def test_lame_constants_of_the_figure_material():
    g = _read_golden("snh_material.txt")
    mu, lam = lame_from_young(SNH_E, SNH_NU)
    assert abs(mu - g["mu"]) < 1e-2 and abs(lam - g["lambda"]) < 1e-2
    # the paper's printed co-rotational mu for the collision example is E/(2(1+nu))
    # of E = 7e6, nu = 0.45
    mu2, _ = lame_from_young(7.0e6, 0.45)
    assert abs(mu2 - g["collision_mu"]) / g["collision_mu"] < 1e-4


def test_figure_poses_are_rigid_and_keep_bones_connected():
    joints, parent = figure_rig()
    xf = figure_pose(joints, parent, 3)
    M = xf.reshape(-1, 3, 4)
    Q, t = M[:, :, :3], M[:, :, 3]
    assert np.allclose(np.einsum("kji,kjl->kil", Q, Q), np.eye(3))
    assert np.allclose(np.linalg.det(Q), 1.0)
    for j, p in enumerate(parent):
        if p >= 0:   # parent and child transforms agree at the child joint
            assert np.allclose(Q[p] @ joints[j] + t[p], Q[j] @ joints[j] + t[j])
    assert np.array_equal(xf, figure_pose(joints, parent, 3))


def test_bar_twist_pose():
    cfg = bar_twist_config()
    M = cfg["xfs"][0].reshape(2, 3, 4)
    c = np.array([2.0, 2.0, 16.0])
    assert np.allclose(M[0], np.concatenate([np.eye(3), np.zeros((3, 1))], 1))
    assert np.allclose(M[1][:, :3] @ c + M[1][:, 3], c + [0, 0, 0.5])
    assert np.allclose(M[1][:, :3] @ [1, 0, 0], [0, 1, 0])
    assert len(cfg["pin_verts"]) == 50


def test_character_rig_subdivides_bones():
    from synth import character_rig, figure_rig
    J, P = character_rig(40)
    J0, P0 = figure_rig()
    assert len(J) == 40 and all(P[j] < j for j in range(40)) and P[0] == -1
    # every original joint survives, and every new joint lies on an original bone
    ids = [int(np.argmin(np.linalg.norm(J - o, axis=1))) for o in J0]
    assert all(np.allclose(J[i], o) for i, o in zip(ids, J0))
    bones0 = [(J0[p], J0[j]) for j, p in enumerate(P0) if p >= 0]
    for j in set(range(40)) - set(ids):
        on = [np.linalg.norm(np.cross(J[j] - a, b - a)) / np.linalg.norm(b - a) < 1e-12 and
              0 < np.dot(J[j] - a, b - a) < np.dot(b - a, b - a) for a, b in bones0]
        assert any(on)
    # chains: the original parent of each original joint is still an ancestor
    for j, p in enumerate(P0):
        if p < 0:
            continue
        a = P[ids[j]]
        while a != ids[p]:
            assert a > ids[p]
            a = P[a]


def test_figure_animation_is_smooth_and_rigid():
    from synth import figure_animation, figure_rig
    J, P = figure_rig()
    A = figure_animation(J, P, 3, 20)
    Q = A.reshape(20, 15, 3, 4)[:, :, :, :3]
    assert np.allclose(np.einsum("fhji,fhjk->fhik", Q, Q), np.eye(3), atol=1e-12)
    assert np.allclose(np.linalg.det(Q), 1.0)
    step = np.abs(np.diff(A, axis=0)).max()
    assert 0 < step < 0.3          # frame-to-frame motion at 30 frames/s
