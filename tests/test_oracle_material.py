"""Pins for oracle.material: rest state, finite differences, library determinant,
closed forms that relate the three models."""
import numpy as np
import pytest

from oracle import material
from oracle.mandel import to_mandel, from_mandel, I6, basis

MODELS = ["arap", "corot", "snh"]


def _rand_sym(rng, k, scale=0.3, shift=1.0):
    A = rng.normal(size=(k, 3, 3)) * scale
    return shift * np.eye(3) + 0.5 * (A + np.swapaxes(A, 1, 2))


def test_mandel_is_isometric(rng):
    S = _rand_sym(rng, 20)
    T = _rand_sym(rng, 20)
    assert np.allclose(np.einsum("kij,kij->k", S, T), np.einsum("kp,kp->k", to_mandel(S), to_mandel(T)))
    assert np.allclose(from_mandel(to_mandel(S)), S)
    E = basis()
    G = np.einsum("pij,qij->pq", E, E)
    assert np.allclose(G, np.eye(6))


@pytest.mark.parametrize("model", MODELS)
def test_rest_energy_and_stress_vanish(model, rng):
    mu = rng.uniform(0.5, 5.0, size=7)
    lam = rng.uniform(0.0, 50.0, size=7)
    s = np.tile(I6, (7, 1))
    assert np.allclose(material.psi(model, s, mu, lam), 0.0, atol=1e-13)
    assert np.allclose(material.grad(model, s, mu, lam), 0.0, atol=1e-12)


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("shift", [1.0, 0.2, -0.6])   # near rest, compressed, inverted
def test_gradient_and_hessian_match_finite_differences(model, shift, rng):
    k = 6
    s = to_mandel(_rand_sym(rng, k, 0.4, shift))
    mu = rng.uniform(0.5, 3.0, size=k)
    lam = rng.uniform(0.0, 20.0, size=k)
    g = material.grad(model, s, mu, lam)
    H = material.hess(model, s, mu, lam)
    h = 1e-5
    for p in range(6):
        e = np.zeros(6); e[p] = h
        dpsi = (material.psi(model, s + e, mu, lam) - material.psi(model, s - e, mu, lam)) / (2 * h)
        assert np.allclose(dpsi, g[:, p], rtol=1e-7, atol=1e-7 * np.abs(g).max())
        dg = (material.grad(model, s + e, mu, lam) - material.grad(model, s - e, mu, lam)) / (2 * h)
        assert np.allclose(dg, H[:, :, p], rtol=1e-7, atol=1e-7 * np.abs(H).max())
    assert np.allclose(H, np.swapaxes(H, 1, 2))


def test_levi_civita_determinant_matches_library(rng):
    S = _rand_sym(rng, 50, 0.8, 0.3)
    J, gJ, _ = material._det_and_derivs(to_mandel(S))
    assert np.allclose(J, np.linalg.det(S))
    # gradient of det is the adjugate, det(S) S^{-1}, for invertible S
    adj = np.linalg.det(S)[:, None, None] * np.linalg.inv(S)
    assert np.allclose(gJ, to_mandel(adj))


def test_snh_rest_hessian_equals_corotational(rng):
    """With lam_s = lam + mu the SNH rest Hessian is linear elasticity's."""
    mu = rng.uniform(0.5, 3.0, size=4)
    lam = rng.uniform(0.0, 20.0, size=4)
    s = np.tile(I6, (4, 1))
    assert np.allclose(material.hess("snh", s, mu, lam), material.hess("corot", s, mu, lam))


def test_corot_without_lambda_is_arap(rng):
    s = to_mandel(_rand_sym(rng, 9))
    mu = rng.uniform(0.5, 3.0, size=9)
    z = np.zeros(9)
    assert np.allclose(material.psi("corot", s, mu, z), material.psi("arap", s, mu, z))
    assert np.allclose(material.grad("corot", s, mu, z), material.grad("arap", s, mu, z))


def test_quadratic_models_have_textbook_hessian(rng):
    """ARAP: 2 mu I; corot: 2 mu I + lam m m^T (m = Mandel identity)."""
    s = to_mandel(_rand_sym(rng, 3))
    H = material.hess("corot", s, 2.0, 5.0)
    assert np.allclose(H[0], 4.0 * np.eye(6) + 5.0 * np.outer(I6, I6))


def test_spd_projection(rng):
    A = rng.normal(size=(30, 6, 6))
    H = A + np.swapaxes(A, 1, 2)                       # indefinite
    mu = np.full(30, 2.0)
    P = material.project_spd(H, mu)
    lp = np.linalg.eigvalsh(P)
    lh = np.linalg.eigvalsh(H)
    assert np.all(lp >= 2.0e-6 * (1 - 1e-9))
    # eigenvalue magnitudes are kept (filtered by absolute value)
    assert np.allclose(np.sort(lp, axis=1), np.sort(np.maximum(np.abs(lh), 2e-6), axis=1))
    # already-SPD input passes through untouched
    B = np.einsum("kij,klj->kil", A, A) + np.eye(6)
    assert np.array_equal(material.project_spd(B, mu), B)
