"""Energy densities Psi(S) of the symmetric stretch S, with gradient and Hessian
in Mandel coordinates (paper §3, Eq. 2 and Eq. 6: Psi(s_k); §4 names ARAP and
co-rotational elasticity without formulas).

Readings of the paper (it gives no formulas):
  ARAP   Psi = mu |S - I|_F^2
  corot  Psi = mu |S - I|_F^2 + (lam/2) tr(S - I)^2
  SNH    Psi = (mu/2)(|S|_F^2 - 3) - mu (J - 1) + (lam_s/2)(J - 1)^2,  J = det S,
         lam_s = lam + mu, the stable neo-Hookean of Kim and Eberle ("Dynamic
         Deformables", SIGGRAPH 2022 course), whose shift of lambda makes the rest
         Hessian equal linear (co-rotational) elasticity's.
All three vanish with zero gradient at S = I.  SNH is polynomial, so it is
defined for inverted S; its Hessian is made SPD per element by filtering its
eigenvalues: each eigenvalue is replaced by max(|eigenvalue|, eps*mu), eps = 1e-6
(absolute-value eigenvalue filtering, Chen et al., "Stabler Neo-Hookean
Simulation: Absolute Eigenvalue Filtering for Projected Newton", SIGGRAPH 2024),
applied only to elements whose smallest eigenvalue is below eps*mu.
"""
import numpy as np

from .mandel import I6, basis

MODELS = ("arap", "corot", "snh")
SPD_EPS = 1.0e-6

# Levi-Civita symbol: det S = (1/6) eps_ijk eps_lmn S_il S_jm S_kn
_EPS3 = np.zeros((3, 3, 3))
for _i, _j, _k in [(0, 1, 2), (1, 2, 0), (2, 0, 1)]:
    _EPS3[_i, _j, _k] = 1.0
    _EPS3[_i, _k, _j] = -1.0
_E6 = basis()                                  # (6,3,3)


def _det_and_derivs(s):
    """J = det S and its gradient and Hessian with respect to the 6-vector s,
    written from the Levi-Civita expansion of the determinant."""
    from .mandel import from_mandel
    S = from_mandel(s)                                            # (m,3,3)
    # W[e,i,j,l,m] = sum_kn eps_ijk eps_lmn S_kn  (second derivative of det wrt S_il, S_jm)
    W = np.einsum("ijk,lmn,ekn->eijlm", _EPS3, _EPS3, S, optimize=True)
    # first derivative: dJ/dS_il = (1/2) eps_ijk eps_lmn S_jm S_kn
    dJdS = 0.5 * np.einsum("eijlm,ejm->eil", W, S, optimize=True)
    J = np.einsum("eijlm,eil,ejm->e", W, S, S, optimize=True) / 6.0
    g = np.einsum("pil,eil->ep", _E6, dJdS)
    H = np.einsum("pil,qjm,eijlm->epq", _E6, _E6, W, optimize=True)
    return J, g, H


def psi(model, s, mu, lam):
    s = np.atleast_2d(s)
    d = s - I6
    base = np.einsum("ep,ep->e", d, d)
    if model == "arap":
        return mu * base
    if model == "corot":
        return mu * base + 0.5 * lam * (s @ I6 - 3.0) ** 2
    if model == "snh":
        J, _, _ = _det_and_derivs(s)
        lam_s = lam + mu
        return 0.5 * mu * (np.einsum("ep,ep->e", s, s) - 3.0) - mu * (J - 1.0) \
            + 0.5 * lam_s * (J - 1.0) ** 2
    raise ValueError(model)


def grad(model, s, mu, lam):
    """dPsi/ds, (m,6); as a symmetric matrix this is the stress sigma with
    dPsi = sigma : dS."""
    s = np.atleast_2d(s)
    mu = np.broadcast_to(mu, s.shape[:1])[:, None]
    lam = np.broadcast_to(lam, s.shape[:1])[:, None]
    if model == "arap":
        return 2.0 * mu * (s - I6)
    if model == "corot":
        return 2.0 * mu * (s - I6) + lam * (s @ I6 - 3.0)[:, None] * I6
    if model == "snh":
        J, gJ, _ = _det_and_derivs(s)
        lam_s = lam + mu
        return mu * s - mu * gJ + lam_s * (J - 1.0)[:, None] * gJ
    raise ValueError(model)


def hess(model, s, mu, lam):
    """d2Psi/ds2, (m,6,6), not projected."""
    s = np.atleast_2d(s)
    m = s.shape[0]
    mu = np.broadcast_to(mu, (m,))[:, None, None]
    lam = np.broadcast_to(lam, (m,))[:, None, None]
    eye = np.broadcast_to(np.eye(6), (m, 6, 6))
    if model == "arap":
        return 2.0 * mu * eye
    if model == "corot":
        return 2.0 * mu * eye + lam * np.outer(I6, I6)[None]
    if model == "snh":
        J, gJ, HJ = _det_and_derivs(s)
        lam_s = lam + mu
        return mu * eye + (lam_s * (J - 1.0)[:, None, None] - mu) * HJ \
            + lam_s * np.einsum("ep,eq->epq", gJ, gJ)
    raise ValueError(model)


def project_spd(H, mu, eps=SPD_EPS):
    """Replace every eigenvalue of each 6x6 H by max(|eigenvalue|, eps*mu);
    elements whose smallest eigenvalue is already >= eps*mu are returned unchanged."""
    H = np.array(H, dtype=np.float64, copy=True)
    floor = eps * np.broadcast_to(mu, H.shape[:1])
    lam_, V = np.linalg.eigh(H)
    bad = lam_[:, 0] < floor
    if np.any(bad):
        lc = np.maximum(np.abs(lam_[bad]), floor[bad, None])
        H[bad] = np.einsum("epi,ei,eqi->epq", V[bad], lc, V[bad])
    return H
