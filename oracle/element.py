"""Per-tetrahedron kinematics, energy, gradient and condensed Hessian.

Paper §3: F = B x with B the deformation-gradient operator (text after Eq. 4);
W_k the tet volume (Eq. 5); S_k the symmetric stretch tied to F_k through the
rig rotation R_k (Eq. 3); the 9x6 map R_k of Eq. 6 applied to s_k; the
condensed system of Eq. 12, whose matrix sum_k W_k A_k^T H_s A_k uses
A_k = R_k^+ B_k, the pseudo-inverse of [R] times B (text after Eq. 12).

Reading of Eq. 9-11 (the KKT system as printed is singular: [R]H_s^-1[R]^T is
9x9 of rank 6): the constraint B_k x = R_k s_k holds in the least-squares
sense through the pseudo-inverse the paper names, s_k = R_k^+ vec(F_k), which
for a rotation R_k and symmetric S is S_k = sym(R_k^T F_k).  E(x) =
sum_k W_k Psi(S_k(x)); Eq. 12 is then the Newton system of E.
"""
import numpy as np
import scipy.sparse as sp

from . import material
from .mandel import to_mandel, from_mandel


def rest_shape(X, T):
    """Rest edge matrix D_m (columns X_a - X_0), volume W_k = det(D_m)/6,
    D_m^{-1}, and the shape-function gradients G (m,4,3): G_a = row a-1 of
    D_m^{-1} for a = 1..3 and G_0 = -(G_1 + G_2 + G_3), so that
    F = sum_a x_a G_a^T."""
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T)
    P = X[T]                                        # (m,4,3)
    Dm = np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]], axis=-1)
    vol = np.linalg.det(Dm) / 6.0
    Dminv = np.linalg.inv(Dm)
    G = np.empty((len(T), 4, 3))
    G[:, 1:, :] = Dminv
    G[:, 0, :] = -Dminv.sum(axis=1)
    return Dm, vol, Dminv, G


def deformation_gradient(x, T, G):
    """F_k = B_k x = sum_a x_{T[k,a]} G_{k,a}^T, (m,3,3)."""
    return np.einsum("kai,kaj->kij", np.asarray(x)[T], G)


def stretch(R, F):
    """S_k = sym(R_k^T F_k): the symmetric S minimising |R_k S - F_k|_F."""
    A = np.einsum("kji,kjl->kil", R, F)             # R^T F
    return 0.5 * (A + np.swapaxes(A, 1, 2))


def element_energy(x, T, G, vol, R, model, mu, lam):
    """W_k Psi(S_k), (m,)."""
    s = to_mandel(stretch(R, deformation_gradient(x, T, G)))
    return vol * material.psi(model, s, mu, lam)


def multiplier(x, T, G, R, model, mu, lam):
    """Lambda_k = R_k sigma_k with sigma_k = dPsi/dS (3x3): the multiplier that
    makes s_k stationary in Eq. 6 (R_k^T lambda_k = grad Psi, Eq. 10) and the
    first Piola stress of E with respect to F_k."""
    s = to_mandel(stretch(R, deformation_gradient(x, T, G)))
    sigma = from_mandel(material.grad(model, s, mu, lam))
    return np.einsum("kij,kjl->kil", R, sigma)


def element_forces(x, T, G, vol, R, model, mu, lam):
    """dE/dx_a per element, (m,4,3): W_k Lambda_k G_a."""
    Lam = multiplier(x, T, G, R, model, mu, lam)
    return vol[:, None, None] * np.einsum("kij,kaj->kai", Lam, G)


def gradient(x, T, G, vol, R, model, mu, lam):
    """dE/dx for every vertex, (n,3)."""
    f = element_forces(x, T, G, vol, R, model, mu, lam)
    g = np.zeros((len(x), 3))
    np.add.at(g, np.asarray(T).reshape(-1), f.reshape(-1, 3))
    return g


def condensed_map(R, G):
    """A_k = R_k^+ B_k as a (m,6,12) array: column 3a+i is the Mandel vector of
    sym(R_k^T e_i G_a^T), the stretch caused by a unit move of vertex a along i."""
    m = len(G)
    A = np.empty((m, 6, 12))
    for a in range(4):
        for i in range(3):
            M = np.einsum("kj,kl->kjl", R[:, i, :], G[:, a, :])  # (R^T e_i) G_a^T
            A[:, :, 3 * a + i] = to_mandel(0.5 * (M + np.swapaxes(M, 1, 2)))
    return A


def element_hessians(x, T, G, vol, R, model, mu, lam, project=True):
    """K_k = W_k A_k^T H_s A_k, (m,12,12); H_s projected to SPD for SNH."""
    s = to_mandel(stretch(R, deformation_gradient(x, T, G)))
    Hs = material.hess(model, s, mu, lam)
    if project and model == "snh":
        Hs = material.project_spd(Hs, mu)
    A = condensed_map(R, G)
    return vol[:, None, None] * np.einsum("kpi,kpq,kqj->kij", A, Hs, A, optimize=True)


def assemble(Ke, T, n):
    """Sum element 12x12 blocks into a sparse (3n,3n) matrix."""
    T = np.asarray(T)
    dof = (3 * T[:, :, None] + np.arange(3)).reshape(len(T), 12)
    rows = np.repeat(dof, 12, axis=1).reshape(-1)
    cols = np.tile(dof, (1, 12)).reshape(-1)
    return sp.coo_matrix((Ke.reshape(-1), (rows, cols)), shape=(3 * n, 3 * n)).tocsr()
