"""Voxel tetrahedral meshes (Kuhn six-tet split) and the capsule stick figure.

The paper's character meshes (flour sack, human, turtle; Table 1) are not
available, so seeded voxel meshes of matching size stand in for them.  Every
cube is split into the six tetrahedra that share its main diagonal; using the
same diagonal in every cube makes the split conforming across faces.
"""
from __future__ import annotations

import itertools

import numpy as np

# The six axis orders of the Kuhn split.  Walking the cube from corner (0,0,0)
# to (1,1,1) one axis at a time visits four corners, which form one tetrahedron.
_PERMS = list(itertools.permutations(range(3)))


def _perm_parity(p):
    inv = 0
    for i in range(3):
        for j in range(i + 1, 3):
            inv += p[i] > p[j]
    return inv & 1


def kuhn_voxel_mesh(occ: np.ndarray, h: float = 1.0, origin=(0.0, 0.0, 0.0)):
    """Tetrahedralise the occupied cells of a boolean grid ``occ[nx,ny,nz]``.

    Returns ``X`` (n,3) float64 corner positions and ``T`` (m,4) int32 tets,
    every tet positively oriented.  Only corners touched by an occupied cell
    become vertices; vertices are numbered in (i, j, k) lexicographic order.
    """
    occ = np.asarray(occ, dtype=bool)
    nx, ny, nz = occ.shape
    cells = np.argwhere(occ)                       # (c,3) lexicographic
    used = np.zeros((nx + 1, ny + 1, nz + 1), dtype=bool)
    for off in itertools.product((0, 1), repeat=3):
        used[cells[:, 0] + off[0], cells[:, 1] + off[1], cells[:, 2] + off[2]] = True
    vid = -np.ones(used.shape, dtype=np.int64)
    corners = np.argwhere(used)
    vid[corners[:, 0], corners[:, 1], corners[:, 2]] = np.arange(len(corners))
    X = corners.astype(np.float64) * h + np.asarray(origin, dtype=np.float64)
    tets = []
    for p in _PERMS:
        e0 = np.zeros(3, dtype=np.int64); e0[p[0]] = 1
        e1 = e0.copy(); e1[p[1]] = 1
        path = [np.zeros(3, dtype=np.int64), e0, e1, np.ones(3, dtype=np.int64)]
        if _perm_parity(p):                        # odd axis order: swap to keep det > 0
            path = [path[0], path[2], path[1], path[3]]
        cols = [vid[cells[:, 0] + c[0], cells[:, 1] + c[1], cells[:, 2] + c[2]] for c in path]
        tets.append(np.stack(cols, axis=1))
    # cell-major order: the six tets of one cube are adjacent
    T = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    return X, T


def bar_mesh(nx=4, ny=4, nz=16, h=1.0):
    """Box of nx*ny*nz unit cubes (the 4x4x16 bar: 425 verts, 1536 tets)."""
    return kuhn_voxel_mesh(np.ones((nx, ny, nz), dtype=bool), h)


# ---------------------------------------------------------------------------
# Capsule stick figure: body height ~1, z up, arms along x.
# 15 joints: pelvis, neck, head; shoulder, elbow, wrist x2; hip, knee, ankle x2.
# ---------------------------------------------------------------------------
_JOINTS = np.array([
    [0.00, 0.0, 0.52],   # 0 pelvis
    [0.00, 0.0, 0.80],   # 1 neck
    [0.00, 0.0, 0.95],   # 2 head
    [0.14, 0.0, 0.78],   # 3 shoulder L
    [0.38, 0.0, 0.78],   # 4 elbow L
    [0.60, 0.0, 0.78],   # 5 wrist L
    [-0.14, 0.0, 0.78],  # 6 shoulder R
    [-0.38, 0.0, 0.78],  # 7 elbow R
    [-0.60, 0.0, 0.78],  # 8 wrist R
    [0.08, 0.0, 0.50],   # 9 hip L
    [0.09, 0.0, 0.27],   # 10 knee L
    [0.10, 0.0, 0.04],   # 11 ankle L
    [-0.08, 0.0, 0.50],  # 12 hip R
    [-0.09, 0.0, 0.27],  # 13 knee R
    [-0.10, 0.0, 0.04],  # 14 ankle R
])
_PARENT = np.array([-1, 0, 1, 1, 3, 4, 1, 6, 7, 0, 9, 10, 0, 12, 13], dtype=np.int32)
# (start, end, radius): torso, head, two arms, two legs
_CAPSULES = [
    ((0.00, 0.0, 0.50), (0.00, 0.0, 0.80), 0.100),
    ((0.00, 0.0, 0.86), (0.00, 0.0, 0.95), 0.065),
    ((0.06, 0.0, 0.78), (0.62, 0.0, 0.78), 0.038),
    ((-0.06, 0.0, 0.78), (-0.62, 0.0, 0.78), 0.038),
    ((0.08, 0.0, 0.50), (0.10, 0.0, 0.03), 0.050),
    ((-0.08, 0.0, 0.50), (-0.10, 0.0, 0.03), 0.050),
]


def figure_rig(scale: float = 1.0):
    """Joint positions (15,3) and parent links of the stick figure."""
    return _JOINTS * scale, _PARENT.copy()


def character_rig(n_handles: int = 40, scale: float = 1.0):
    """The stick figure's skeleton with extra joints inserted along its bones
    (spine, neck and limb segments), n_handles joints in all, parents first.
    The extra joints go to the bones in proportion to their lengths (largest
    remainder), evenly spaced along each bone."""
    J, P = _JOINTS * scale, _PARENT
    bones = [(int(P[j]), j) for j in range(len(J)) if P[j] >= 0]
    extra = n_handles - len(J)
    if extra < 0:
        raise ValueError("n_handles below the figure's 15 joints")
    L = np.array([np.linalg.norm(J[j] - J[p]) for p, j in bones])
    share = extra * L / L.sum()
    k = np.floor(share).astype(int)
    for i in np.argsort(-(share - k))[: extra - k.sum()]:
        k[i] += 1
    per_bone = {j: int(k[i]) for i, (_, j) in enumerate(bones)}
    joints, parent, new_id = [], [], {}
    for j in range(len(J)):
        p = int(P[j])
        up = new_id[p] if p >= 0 else -1
        for s in range(1, per_bone.get(j, 0) + 1):      # intermediate joints of bone p -> j
            t = s / (per_bone[j] + 1)
            joints.append(J[p] + t * (J[j] - J[p]))
            parent.append(up)
            up = len(joints) - 1
        joints.append(J[j])
        parent.append(up)
        new_id[j] = len(joints) - 1
    return np.array(joints), np.array(parent, dtype=np.int32)


def _capsule_occupancy(centers: np.ndarray, scale: float) -> np.ndarray:
    inside = np.zeros(len(centers), dtype=bool)
    for a, b, r in _CAPSULES:
        a = np.asarray(a) * scale
        b = np.asarray(b) * scale
        ab = b - a
        t = np.clip(((centers - a) @ ab) / (ab @ ab), 0.0, 1.0)
        d = np.linalg.norm(centers - (a + t[:, None] * ab), axis=1)
        inside |= d <= r * scale
    return inside


def figure_mesh(h: float, scale: float = 1.0):
    """Voxelise the union of the six capsules at cell edge ``h``.

    A cell is occupied when its centre lies inside a capsule.  Returns
    ``X, T, joints, parent``.
    """
    lo = np.array([-0.70, -0.15, -0.08]) * scale
    hi = np.array([0.70, 0.15, 1.05]) * scale
    dims = np.ceil((hi - lo) / h).astype(int)
    ii, jj, kk = np.meshgrid(*[np.arange(d) for d in dims], indexing="ij")
    centers = lo + (np.stack([ii, jj, kk], axis=-1).reshape(-1, 3) + 0.5) * h
    occ = _capsule_occupancy(centers, scale).reshape(dims)
    X, T = kuhn_voxel_mesh(occ, h, lo)
    joints, parent = figure_rig(scale)
    return X, T, joints, parent


def figure_mesh_for_tets(target_tets: int, scale: float = 1.0, rel_tol: float = 0.02):
    """Bisect the cell edge h until the tet count is within ``rel_tol`` of the target."""
    lo_h, hi_h = 1e-4 * scale, 0.2 * scale      # small h -> many tets
    best = None
    for it in range(60):
        h = np.sqrt(lo_h * hi_h)
        X, T, joints, parent = figure_mesh(h, scale)
        m = len(T)
        if best is None or abs(m - target_tets) < abs(best[1].shape[0] - target_tets):
            best = (X, T, joints, parent, h)
        if abs(m - target_tets) <= rel_tol * target_tets:
            break
        if m > target_tets:
            lo_h = h
        else:
            if it == 0:
                # first try already too coarse: bracket from tets ~ h^-3 instead of
                # bisecting toward the far lower end (a grid too large to build)
                lo_h = h * (m / target_tets) ** (1.0 / 3.0) * 0.8
            hi_h = h
    X, T, joints, parent, h = best
    return X, T, joints, parent, h
