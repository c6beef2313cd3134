"""Pins for external vertex forces in the oracle (§4, "Collision response"):
the uniaxial closed form of a pulled ARAP bar, linearity and reciprocity of the
co-rotational response, SNH equilibrium, and forces on pinned vertices."""
import numpy as np
import pytest

from oracle import element, solve as S
from synth import bar_pull_config, bar_twist_config, face_traction_loads


def _solve(cfg, **kw):
    st = S.Setup.from_config(cfg)
    x, info = S.solve(st, cfg["xfs"][0], cfg["model"], newton_tol=1e-13, **kw)
    return st, x, info


def test_pulled_arap_bar_is_uniform_uniaxial_strain():
    # ARAP (lambda = 0, no lateral contraction): stress 2 mu eps along z balances
    # the traction, so every vertex moves by eps z along z, eps = t / (2 mu)
    cfg = bar_pull_config(traction=0.05, mu=1.3)
    st, x, _ = _solve(cfg, f_ext=cfg["f_ext"])
    eps = cfg["traction"] / (2 * cfg["mu"])
    X = cfg["X"]
    want = X + np.outer(X[:, 2] * eps, [0, 0, 1])
    assert np.abs(x - want).max() <= 1e-11 * st.bbox_diag
    # without the force the bar stays at rest
    _, x0, _ = _solve(cfg)
    assert np.abs(x0 - X).max() <= 1e-12 * st.bbox_diag


def test_corot_response_is_linear_and_reciprocal(rng):
    cfg = dict(bar_twist_config(3, 3, 8), model="corot", mu=1.0, lam=2.0)
    n = len(cfg["X"])
    free = np.setdiff1d(np.arange(n), cfg["pin_verts"])
    f1 = np.zeros((n, 3))
    f2 = np.zeros((n, 3))
    f1[rng.choice(free, 5, replace=False)] = rng.normal(size=(5, 3)) * 0.05
    f2[rng.choice(free, 5, replace=False)] = rng.normal(size=(5, 3)) * 0.05
    _, x0, _ = _solve(cfg)
    d1 = _solve(cfg, f_ext=f1)[1] - x0
    d2 = _solve(cfg, f_ext=f2)[1] - x0
    d12 = _solve(cfg, f_ext=2 * f1 - f2)[1] - x0
    scale = np.abs(d1).max()
    assert np.abs(d12 - (2 * d1 - d2)).max() <= 1e-9 * scale
    # Maxwell-Betti: the response matrix is symmetric
    w12, w21 = np.sum(f1 * d2), np.sum(f2 * d1)
    assert abs(w12 - w21) <= 1e-9 * (abs(w12) + abs(w21))
    # a force does positive work on its own displacement
    assert np.sum(f1 * d1) > 0 and np.sum(f2 * d2) > 0


def test_snh_equilibrium_under_load():
    cfg = bar_pull_config(traction=0.4, model="snh", mu=1.0, lam=4.0)
    st, x, info = _solve(cfg, f_ext=cfg["f_ext"])
    assert info["converged"]
    # internal forces balance the load on every free vertex
    gi = element.gradient(x, st.T, st.G, st.vol, np.repeat(np.eye(3)[None], st.m, 0), "snh", st.mu, st.lam)
    free = np.setdiff1d(np.arange(st.n), st.pin_verts)
    assert np.abs(gi[free] - cfg["f_ext"][free]).max() <= 1e-9 * np.abs(cfg["f_ext"]).max()
    # the bar lengthens and (lambda > 0) narrows at the loaded end
    top = cfg["X"][:, 2] == cfg["X"][:, 2].max()
    assert x[top, 2].min() > cfg["X"][top, 2].max()
    w0 = np.ptp(cfg["X"][top, 0])
    assert np.ptp(x[top, 0]) < w0


def test_forces_on_eliminated_pins_do_nothing(rng):
    cfg = bar_twist_config(3, 3, 8)
    n = len(cfg["X"])
    f = np.zeros((n, 3))
    f[cfg["pin_verts"]] = rng.normal(size=(len(cfg["pin_verts"]), 3))
    st, x0, _ = _solve(cfg)
    _, x1, _ = _solve(cfg, f_ext=f)
    assert np.abs(x1 - x0).max() <= 1e-12 * st.bbox_diag


def test_face_traction_loads_total():
    cfg = bar_pull_config(4, 2, 5, traction=0.3)
    assert np.allclose(cfg["f_ext"].sum(0), [0, 0, 0.3 * 4 * 2])
    top = cfg["X"][:, 2] == 5.0
    assert np.all(cfg["f_ext"][~top] == 0)
    f = face_traction_loads(cfg["X"], cfg["T"], cfg["X"][:, 0] == 0.0, [1.0, 0, 0])
    assert np.allclose(f.sum(0), [2 * 5, 0, 0])
