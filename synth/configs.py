"""Workload recipes: a mesh, its rig, its material constants and seeded poses.

Each recipe returns a plain dict of arrays.  Rigs name handles by joint index;
``cluster_rule`` says how tets pick a handle rotation ("bone": nearest bone
segment, "joint": nearest joint) and pins are either explicit (``pin_verts``,
``pin_handle``) or chosen by radius around joints and bone midpoints.
"""
from __future__ import annotations

import functools

import numpy as np

from .meshes import bar_mesh, character_rig, figure_mesh_for_tets
from .poses import bar_twist_pose, figure_pose

# Stable neo-Hookean figure material: Young's modulus (Pa) and Poisson ratio.
SNH_E = 1.0e5
SNH_NU = 0.45


def lame_from_young(E, nu):
    """Lame constants (mu, lambda) of an isotropic material."""
    mu = E / (2.0 * (1.0 + nu))
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return mu, lam


def bar_twist_config(nx=4, ny=4, nz=16):
    """The 4x4x16 bar: ARAP, handle 0 fixed at z=0, handle 1 at z=nz turned
    90 deg about the long axis and shifted 0.5 along it; every vertex of an end
    face is pinned to that face's handle; tets take the nearest handle."""
    X, T = bar_mesh(nx, ny, nz)
    joints = np.array([[nx / 2, ny / 2, 0.0], [nx / 2, ny / 2, float(nz)]])
    parent = np.array([-1, -1], dtype=np.int32)
    lo = np.where(X[:, 2] == 0.0)[0]
    hi = np.where(X[:, 2] == float(nz))[0]
    pin_verts = np.concatenate([lo, hi]).astype(np.int32)
    pin_handle = np.concatenate([np.zeros(len(lo)), np.ones(len(hi))]).astype(np.int32)
    return dict(
        name=f"bar{nx}x{ny}x{nz}", X=X, T=T, joints=joints, parent=parent,
        cluster_rule="joint", pin_verts=pin_verts, pin_handle=pin_handle, pin_radius=0.0,
        model="arap", mu=1.0, lam=0.0, xfs=bar_twist_pose(nx, ny, nz)[None],
    )


@functools.lru_cache(maxsize=8)
def _figure_mesh_cached(target_tets, scale):
    return figure_mesh_for_tets(target_tets, scale)


def figure_config(target_tets=200_000, model="snh", seeds=range(16), scale=1.0,
                  E=SNH_E, nu=SNH_NU, pin_radius_cells=1.5):
    """Capsule stick figure voxelised to ~target_tets, 15 joint handles,
    FK poses seeded by ``seeds`` (+-45 deg turns, +-0.1 root shift)."""
    X, T, joints, parent, h = _figure_mesh_cached(int(target_tets), float(scale))
    mu, lam = lame_from_young(E, nu)
    xfs = np.stack([figure_pose(joints, parent, s) for s in seeds]) if len(seeds) else \
        np.zeros((0, len(joints), 12))
    return dict(
        name=f"figure{len(T)}", X=X.copy(), T=T.copy(), joints=joints, parent=parent,
        cluster_rule="bone", pin_verts=None, pin_handle=None, pin_radius=pin_radius_cells * h,
        model=model, mu=mu, lam=lam, xfs=xfs, h=h,
    )


def character_config(target_tets=2_000_000, n_handles=40, model="snh", seeds=range(4), E=SNH_E, nu=SNH_NU,
                     max_angle_deg=20.0, pin_radius_cells=1.5):
    """The capsule character voxelised to ~target_tets with the skeleton
    subdivided to n_handles joints (``character_rig``); FK poses turn every
    joint by up to +-max_angle_deg (the subdivided chains compound it)."""
    X, T, _, _, h = _figure_mesh_cached(int(target_tets), 1.0)
    joints, parent = character_rig(n_handles)
    mu, lam = lame_from_young(E, nu)
    xfs = np.stack([figure_pose(joints, parent, s, max_angle_deg=max_angle_deg) for s in seeds]) \
        if len(seeds) else np.zeros((0, len(joints), 12))
    return dict(
        name=f"character{len(T)}h{n_handles}", X=X.copy(), T=T.copy(), joints=joints, parent=parent,
        cluster_rule="bone", pin_verts=None, pin_handle=None, pin_radius=pin_radius_cells * h,
        model=model, mu=mu, lam=lam, xfs=xfs, h=h,
    )


def face_traction_loads(X, T, on_face, traction):
    """Nodal loads of a uniform traction (force per area, 3-vector) on the
    boundary triangles whose three vertices satisfy ``on_face``: each triangle
    gives a third of traction x area to each of its vertices (the consistent
    load of linear shape functions)."""
    X = np.asarray(X, dtype=np.float64)
    f = np.zeros_like(X)
    tri = {}
    for tet in np.asarray(T):
        for skip in range(4):
            face = tuple(sorted(int(v) for i, v in enumerate(tet) if i != skip))
            tri[face] = tri.get(face, 0) + 1
    for face, count in tri.items():
        if count != 1 or not all(on_face[v] for v in face):
            continue
        a, b, c = (X[v] for v in face)
        area = 0.5 * np.linalg.norm(np.cross(b - a, c - a))
        for v in face:
            f[v] += np.asarray(traction, dtype=np.float64) * area / 3.0
    return f


def bar_pull_config(nx=3, ny=3, nz=8, traction=0.05, model="arap", mu=1.0, lam=0.0):
    """A bar with its z=0 face pinned to one identity handle and a uniform
    traction along +z on its z=nz face, applied as consistent nodal loads
    ``f_ext``.  Every tet takes the single handle."""
    X, T = bar_mesh(nx, ny, nz)
    joints = np.array([[nx / 2, ny / 2, 0.0]])
    parent = np.array([-1], dtype=np.int32)
    lo = np.where(X[:, 2] == 0.0)[0].astype(np.int32)
    f_ext = face_traction_loads(X, T, X[:, 2] == float(nz), [0.0, 0.0, traction])
    return dict(
        name=f"barpull{nx}x{ny}x{nz}", X=X, T=T, joints=joints, parent=parent,
        cluster_rule="joint", pin_verts=lo, pin_handle=np.zeros(len(lo), dtype=np.int32), pin_radius=0.0,
        model=model, mu=mu, lam=lam, xfs=np.array([[1.0, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0]])[None],
        f_ext=f_ext, traction=traction,
    )
