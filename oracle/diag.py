"""Per-element diagnostics: polar decomposition of F and the rotation mismatch.

The paper takes R_k from the rig (§3, Eq. 3; §3.1), not from F.  The polar
factor of F_k is therefore a diagnostic: it flags inverted tets (det F <= 0)
and measures how far the rig rotation is from the tet's own rotation, the
source of the cluster-boundary artifacts the paper reports (§5).

Polar decomposition from the SVD F = U diag(sv) V^T: R_F = U V^T and
P = V diag(sv) V^T; for det F < 0 the smallest singular value takes the sign,
so that R_F stays a rotation (det +1).
"""
import numpy as np

from . import element, rig


def polar(F):
    """Rotation R_F and symmetric P with F = R_F P, (m,3,3) each."""
    U, sv, Vt = np.linalg.svd(F)
    det = np.linalg.det(U) * np.linalg.det(Vt)
    sign = np.where(det < 0, -1.0, 1.0)
    U = U.copy()
    U[:, :, 2] *= sign[:, None]
    sv = sv.copy()
    sv[:, 2] *= sign
    R = U @ Vt
    P = np.einsum("kji,kj,kjl->kil", Vt, sv, Vt)
    return R, P


def diagnostics(st, xf, x):
    """Inverted-tet count, max |skew(R^T F)|_F / |F|_F, max angle (rad)
    between the rig rotation and the polar rotation of F."""
    Q, _ = rig.unpack_pose(xf)
    R = Q[st.cluster]
    F = element.deformation_gradient(x, st.T, st.G)
    detF = np.linalg.det(F)
    A = np.einsum("kji,kjl->kil", R, F)
    skew = 0.5 * (A - np.swapaxes(A, 1, 2))
    rel_skew = np.linalg.norm(skew, axis=(1, 2)) / np.maximum(np.linalg.norm(F, axis=(1, 2)), 1e-300)
    RF, _ = polar(F)
    c = (np.einsum("kij,kij->k", R, RF) - 1.0) * 0.5
    ang = np.arccos(np.clip(c, -1.0, 1.0))
    return dict(inverted=int(np.sum(detF <= 0)), max_rel_skew=float(rel_skew.max()),
                max_angle=float(ang.max()))
