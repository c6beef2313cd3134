"""Pins for oracle.element: volumes by the triple product, the pseudo-inverse
against library least squares, finite differences of the global energy, and the
closed-form stiffness of quadratic models."""
import numpy as np
import pytest

from oracle import element
from oracle.mandel import to_mandel, basis
from synth import bar_mesh, rodrigues

MODELS = ["arap", "corot", "snh"]


def _rand_rot(rng, k):
    return np.stack([rodrigues(rng.normal(size=3), rng.uniform(-np.pi, np.pi)) for _ in range(k)])


@pytest.fixture
def small(rng):
    X, T = bar_mesh(2, 2, 3)
    m = len(T)
    R = _rand_rot(rng, 3)[rng.integers(0, 3, size=m)]
    x = X + 0.15 * rng.normal(size=X.shape)
    mu = rng.uniform(0.5, 2.0, size=m)
    lam = rng.uniform(0.0, 10.0, size=m)
    return X, T, R, x, mu, lam


def test_rest_shape_by_triple_product(rng):
    X, T = bar_mesh(2, 3, 2)
    X = X + 0.05 * rng.normal(size=X.shape)
    _, vol, _, G = element.rest_shape(X, T)
    a, b, c, d = (X[T[:, i]] for i in range(4))
    vol_ref = np.einsum("ki,ki->k", b - a, np.cross(c - a, d - a)) / 6.0
    assert np.allclose(vol, vol_ref)
    assert np.allclose(G.sum(axis=1), 0.0)
    F = element.deformation_gradient(X, T, G)
    assert np.allclose(F, np.eye(3))
    assert np.all(vol > 0)


def test_affine_motion_gives_its_matrix(rng):
    X, T = bar_mesh(2, 2, 2)
    _, _, _, G = element.rest_shape(X, T)
    A = rng.normal(size=(3, 3))
    F = element.deformation_gradient(X @ A.T + rng.normal(size=3), T, G)
    assert np.allclose(F, A)


def test_stretch_is_least_squares_pseudo_inverse(rng):
    """s_k = R_k^+ vec(F_k) with R_k the 9x6 matrix of Eq. 6, solved by lstsq."""
    R = _rand_rot(rng, 12)
    F = rng.normal(size=(12, 3, 3))
    S = element.stretch(R, F)
    E = basis()
    for k in range(12):
        Rk = np.stack([(R[k] @ E[j]).reshape(9) for j in range(6)], axis=1)   # 9x6
        s_ls, *_ = np.linalg.lstsq(Rk, F[k].reshape(9), rcond=None)
        assert np.allclose(s_ls, to_mandel(S[k]))
        # orthonormal columns in the Mandel basis: pseudo-inverse is the transpose
        assert np.allclose(Rk.T @ Rk, np.eye(6))


@pytest.mark.parametrize("model", MODELS)
def test_gradient_matches_energy_differences(model, small):
    X, T, R, x, mu, lam = small
    _, vol, _, G = element.rest_shape(X, T)
    g = element.gradient(x, T, G, vol, R, model, mu, lam)
    h = 1e-6
    E = lambda y: element.element_energy(y, T, G, vol, R, model, mu, lam).sum()
    for v, i in [(0, 0), (5, 2), (17, 1), (len(X) - 1, 0)]:
        e = np.zeros_like(x); e[v, i] = h
        fd = (E(x + e) - E(x - e)) / (2 * h)
        assert abs(fd - g[v, i]) <= 1e-6 * (1 + abs(g[v, i]))


@pytest.mark.parametrize("model", MODELS)
def test_hessian_matches_gradient_differences(model, small):
    X, T, R, x, mu, lam = small
    _, vol, _, G = element.rest_shape(X, T)
    K = element.assemble(element.element_hessians(x, T, G, vol, R, model, mu, lam, project=False),
                         T, len(X)).toarray()
    h = 1e-6
    g = lambda y: element.gradient(y, T, G, vol, R, model, mu, lam).reshape(-1)
    for dof in [0, 7, 22, 3 * len(X) - 1]:
        e = np.zeros(3 * len(X)); e[dof] = h
        fd = (g((x.reshape(-1) + e).reshape(x.shape)) - g((x.reshape(-1) - e).reshape(x.shape))) / (2 * h)
        assert np.allclose(fd, K[:, dof], atol=1e-6 * np.abs(K).max())
    assert np.allclose(K, K.T)


@pytest.mark.parametrize("model", ["arap", "corot"])
def test_closed_form_stiffness_blocks(model, small):
    """K_ab = W [mu (G_a.G_b) I + mu h_b h_a^T + lam h_a h_b^T], h = R G (rotated
    shape gradients), for Psi = mu|S-I|^2 (+ lam/2 tr^2)."""
    X, T, R, x, mu, lam = small
    if model == "arap":
        lam = np.zeros_like(lam)
    _, vol, _, G = element.rest_shape(X, T)
    Ke = element.element_hessians(x, T, G, vol, R, model, mu, lam)
    for k in [0, 3, len(T) - 1]:
        h = G[k] @ R[k].T                 # row a = R G_a
        for a in range(4):
            for b in range(4):
                ref = vol[k] * (mu[k] * (G[k, a] @ G[k, b]) * np.eye(3)
                                + mu[k] * np.outer(h[b], h[a]) + lam[k] * np.outer(h[a], h[b]))
                assert np.allclose(Ke[k, 3 * a:3 * a + 3, 3 * b:3 * b + 3], ref)


@pytest.mark.parametrize("model", MODELS)
def test_element_forces_balance(model, small):
    """Translation invariance: the four vertex forces of a tet sum to zero."""
    X, T, R, x, mu, lam = small
    _, vol, _, G = element.rest_shape(X, T)
    f = element.element_forces(x, T, G, vol, R, model, mu, lam)
    assert np.allclose(f.sum(axis=1), 0.0, atol=1e-12 * np.abs(f).max())
