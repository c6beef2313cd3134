"""Pins of the oracle's per-element diagnostics (oracle/diag.py) by closed forms.

The diagnostics compare the rig rotation R_k of a tet (§3 Eq. 3, §3.1) with
the tet's own deformation F_k: the number of inverted tets (det F <= 0), the
largest |skew(R^T F)|_F / |F|_F, and the largest angle between R_k and the
rotation factor of F_k.  Each case below has a value fixed by hand:

* a rigid turn by theta about an axis with the rig at rest: R^T F = Q(theta),
  |skew| = sqrt(2) sin(theta), |F| = sqrt(3), angle = theta;
* the same turn carried by the rig: zero skew, zero angle;
* a simple shear F = I + gamma e_x e_y^T with the rig at rest:
  |skew| = gamma / sqrt(2), |F| = sqrt(3 + gamma^2), and the rotation factor of
  F turns by atan(gamma / 2) about z (the 2-D polar decomposition of a shear);
* a reflected tet (det F = -1) is counted once, an unreflected one not at all.
"""
import numpy as np
import pytest

from oracle import diag, solve as S
from synth import bar_twist_config, identity_pose, rigid_pose, rodrigues


@pytest.fixture(scope="module")
def bar():
    cfg = bar_twist_config(nx=2, ny=2, nz=4)
    return cfg, S.Setup.from_config(cfg)


def _apply(X, M, c):
    """x = M (X - c) + c for every vertex."""
    return (X - c) @ np.asarray(M).T + c


@pytest.mark.parametrize("theta", [0.05, 0.3, 1.1, 2.5])
def test_rigid_turn_with_rig_at_rest(bar, theta):
    cfg, st = bar
    axis = np.array([1.0, -2.0, 0.5])
    Qr = rodrigues(axis, theta)
    x = _apply(st.X, Qr, st.X.mean(0))
    d = diag.diagnostics(st, identity_pose(len(cfg["joints"])), x)
    assert d["inverted"] == 0
    assert d["max_rel_skew"] == pytest.approx(np.sqrt(2.0) * np.sin(theta) / np.sqrt(3.0), rel=1e-12)
    assert d["max_angle"] == pytest.approx(theta, rel=1e-10)


def test_rigid_turn_carried_by_rig(bar):
    cfg, st = bar
    Qr = rodrigues([0.3, 0.4, -1.0], 0.8)
    t = np.array([0.5, -1.0, 2.0])
    x = st.X @ Qr.T + t
    d = diag.diagnostics(st, rigid_pose(len(cfg["joints"]), Qr, t), x)
    assert d["inverted"] == 0
    assert d["max_rel_skew"] <= 1e-14
    assert d["max_angle"] <= 1e-7     # arccos near 1 loses half the digits


@pytest.mark.parametrize("gamma", [0.02, 0.2, 0.9])
def test_simple_shear(bar, gamma):
    cfg, st = bar
    M = np.eye(3)
    M[0, 1] = gamma
    x = _apply(st.X, M, np.zeros(3))
    d = diag.diagnostics(st, identity_pose(len(cfg["joints"])), x)
    assert d["inverted"] == 0
    assert d["max_rel_skew"] == pytest.approx((gamma / np.sqrt(2.0)) / np.sqrt(3.0 + gamma * gamma), rel=1e-12)
    assert d["max_angle"] == pytest.approx(np.arctan(gamma / 2.0), rel=1e-9)


def test_polar_of_shear_is_the_planar_rotation():
    g = 0.4
    F = np.eye(3)[None].copy()
    F[0, 0, 1] = g
    R, P = diag.polar(F)
    phi = np.arctan(g / 2.0)
    # F = R P with R a turn about z by -phi (maps the sheared frame back)
    expect = rodrigues([0.0, 0.0, 1.0], -phi)
    assert np.allclose(R[0], expect, atol=1e-14)
    assert np.allclose(P[0], P[0].T, atol=1e-14)
    assert np.allclose(R[0] @ P[0], F[0], atol=1e-14)


def test_inverted_count(bar):
    cfg, st = bar
    x = st.X.copy()
    x[:, 2] = -x[:, 2]       # mirror the whole mesh through z = 0: every tet flips
    d_all = diag.diagnostics(st, identity_pose(len(cfg["joints"])), x)
    assert d_all["inverted"] == st.m
    d_none = diag.diagnostics(st, identity_pose(len(cfg["joints"])), st.X)
    assert d_none["inverted"] == 0
    assert d_none["max_rel_skew"] == 0.0 and d_none["max_angle"] <= 1e-7


def test_one_flipped_tet_is_counted_once():
    # two tets sharing a face; the apex of the second is pushed through the face
    X = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [0.4, 0.4, -1.0]])
    T = np.array([[0, 1, 2, 3], [0, 2, 1, 4]])
    st = S.Setup(X, T, joints=[[0.0, 0, 0]], parent=[-1], mu=1.0, lam=0.0, cluster_rule="joint",
                 pin_verts=np.array([0]), pin_handle=np.array([0]))
    assert np.all(st.vol > 0)
    x = X.copy()
    x[4, 2] = 0.5            # apex of tet 1 crosses the shared face z = 0
    d = diag.diagnostics(st, identity_pose(1), x)
    assert d["inverted"] == 1
