"""Rig coupling: rotation clusters, pinned vertices and their pose targets.

Paper §3.1: every tet takes the rotation of the bone segment closest to its
barycenter; all tets of a cluster share that rotation.  A bone runs from a
parent joint to a child joint and carries the parent joint's handle transform.
A rig with no parent links has no segments; tets then take the nearest joint.
§4 ("Exploring different rotation clustering") also compares the nearest
joint and the nearest bone midpoint; both are available as rules.  Ties go to
the lowest bone (child-joint) index: a candidate wins only if its squared
distance is smaller by more than TIE_EPS * L^2, L the bounding-box diagonal of
the points, so mirror-symmetric geometry resolves the same way in any rounding
order.

Eq. 6 pins vertices "along the skeleton"; §4 ("comparing to standard FEM")
pins "around the handles and midpoints".  Reading: pin every vertex within
r_pin of a joint or a bone midpoint; the pin follows the handle its position
clusters to.  §3.2 ("Initial shape preservation"): pinned targets are
x_p = H x_hat_p, the handle transform applied to the pin's rest position.
"""
import numpy as np

TIE_EPS = 1.0e-10


def bones(parent):
    """(proximal joint, distal joint) for every joint with a parent, ordered
    by the distal joint's index."""
    return [(int(p), j) for j, p in enumerate(parent) if p >= 0]


def _seg_dist2(P, a, b):
    ab = b - a
    t = np.clip(((P - a) @ ab) / (ab @ ab), 0.0, 1.0)
    d = P - (a + t[:, None] * ab)
    return np.einsum("ij,ij->i", d, d)


def nearest_handle(P, joints, parent, rule="bone", scale=None):
    """Handle index for every point in P (k,3)."""
    P = np.asarray(P, dtype=np.float64)
    joints = np.asarray(joints, dtype=np.float64)
    if scale is None:
        scale = np.linalg.norm(P.max(axis=0) - P.min(axis=0)) if len(P) else 1.0
    tol = TIE_EPS * scale * scale
    bl = bones(parent)
    if rule == "bone" and bl:
        cands = [(_seg_dist2(P, joints[p], joints[j]), p) for p, j in bl]
    elif rule == "midpoint" and bl:
        cands = []
        for p, j in bl:
            d = P - 0.5 * (joints[p] + joints[j])
            cands.append((np.einsum("ij,ij->i", d, d), p))
    else:
        cands = [(np.einsum("ij,ij->i", P - joints[j], P - joints[j]), j)
                 for j in range(len(joints))]
    best_d = cands[0][0].copy()
    best_h = np.full(len(P), cands[0][1], dtype=np.int32)
    for d, h in cands[1:]:
        win = d < best_d - tol
        best_d[win] = d[win]
        best_h[win] = h
    return best_h


def cluster_tets(X, T, joints, parent, rule="bone"):
    """Rotation cluster (a handle index) of every tet, from its barycenter."""
    X = np.asarray(X, dtype=np.float64)
    scale = np.linalg.norm(X.max(axis=0) - X.min(axis=0))
    bary = X[np.asarray(T)].mean(axis=1)
    return nearest_handle(bary, joints, parent, rule, scale)


def vertex_handles(X, joints, parent, rule="bone"):
    """The handle each vertex position clusters to (used for pins and the
    rigid initial guess)."""
    X = np.asarray(X, dtype=np.float64)
    scale = np.linalg.norm(X.max(axis=0) - X.min(axis=0))
    return nearest_handle(X, joints, parent, rule, scale)


def select_pins(X, joints, parent, r_pin, rule="bone"):
    """Vertices within r_pin of any joint or bone midpoint, and their handles."""
    X = np.asarray(X, dtype=np.float64)
    joints = np.asarray(joints, dtype=np.float64)
    scale = np.linalg.norm(X.max(axis=0) - X.min(axis=0))
    centres = [joints[j] for j in range(len(joints))]
    centres += [0.5 * (joints[p] + joints[j]) for p, j in bones(parent)]
    r2 = r_pin * r_pin + TIE_EPS * scale * scale
    hit = np.zeros(len(X), dtype=bool)
    for c in centres:
        d = X - c
        hit |= np.einsum("ij,ij->i", d, d) <= r2
    verts = np.nonzero(hit)[0].astype(np.int32)
    return verts, vertex_handles(X, joints, parent, rule)[verts]


def unpack_pose(xf):
    """xf (H,12) row-major [Q | t] -> Q (H,3,3), t (H,3)."""
    M = np.asarray(xf, dtype=np.float64).reshape(-1, 3, 4)
    return M[:, :, :3].copy(), M[:, :, 3].copy()


def pin_targets(X, pin_verts, pin_handle, Q, t):
    """x_p = Q_h x_hat_p + t_h (§3.2)."""
    Xp = np.asarray(X, dtype=np.float64)[pin_verts]
    return np.einsum("kij,kj->ki", Q[pin_handle], Xp) + t[pin_handle]
