"""Newton driver for one pose (paper Algorithm 1, §3 Eq. 12, §3.2).

Algorithm 1 sets x <- X, then per pose builds [R] from the rig, assembles the
condensed matrix and right-hand side of Eq. 12, and solves.  For quadratic
Psi (ARAP, co-rotational) with R fixed by the rig the Hessian is constant per
frame, so one solve reaches the minimiser (text after Eq. 12); SNH needs
Newton iterations.  This driver runs Newton on E(x) for every model:

  x <- initial guess; pinned x_v <- x_p                     (elimination mode)
  repeat up to newton_max times:
      g = dE/dx on free DOFs; stop if |g| <= newton_tol * |g(x_ref)|, where
      x_ref is the rigid initial guess (so the test does not depend on the
      start: a warm start at the solution stops at once)
      K = sum_k W_k A_k^T H_s A_k on free DOFs (Eq. 12; SNH: H_s SPD-projected)
      solve K d = -g              (sparse direct LU, or FP64 Jacobi-PCG)
      SNH: backtracking alpha in {1, 1/2, ..., 2^-ls_max} until
           E(x + alpha d) <= E(x) + c alpha g.d  (c = 1e-4); the step is taken
           untested when the predicted decrease -g.d is below 1e-10 |E(x)|
           (it is then rounding noise); if no alpha passes, the smallest is taken.
      x <- x + alpha d

Constraint C(x) (Eq. 6): "eliminate" fixes pinned vertices at x_p (k_s -> inf,
the default); "penalty" adds k_s/2 |x_v - x_p|^2 per pin as written in Eq. 6.
Rotations: "rig" (the method: R_k is the rotation of the tet's cluster handle,
§3 Eq. 3, §3.1) or "polar" (R_k = the rotation factor of F_k(x), det +1, as a
co-rotational FEM element takes it: E is then the energy of the standard FEM
model §4 compares against, coupled to the rig through the pins only).  In
"polar" mode R is re-evaluated at every iterate and line-search trial, the
Newton step uses the Hessian at fixed R, and every model is line-searched.

External forces (§4, "Collision response"): a per-vertex force field f adds
-sum_v f_v . x_v to E, so the gradient gains -f and the Hessian is unchanged.

Initial guess: "rest" (x = X, as in Algorithm 1), "rigid" (every vertex moved by
the transform of the handle its position clusters to), "corot", or an explicit
array.  "corot" (the default) starts SNH from one Newton step of the
co-rotational energy with the same mu, lambda taken at the rigid guess: that
energy is quadratic with the same rest Hessian as SNH (lambda_SNH = lambda +
mu), so the step lands near the SNH minimiser instead of on the rigid guess,
whose vertex field jumps across every cluster boundary.  The step counts as a
Newton step; for ARAP and co-rotational Psi "corot" is the rigid guess.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import diag, element, rig

LS_C = 1.0e-4
LS_MAX = 20
LS_NOISE = 1.0e-10


class Setup:
    """Everything about a mesh and rig that does not change with the pose."""

    def __init__(self, X, T, joints, parent, mu, lam, cluster_rule="bone",
                 pin_verts=None, pin_handle=None, pin_radius=0.0, tet_cluster=None):
        self.X = np.asarray(X, dtype=np.float64)
        self.T = np.asarray(T, dtype=np.int64)
        self.n, self.m = len(self.X), len(self.T)
        self.joints = np.asarray(joints, dtype=np.float64)
        self.parent = np.asarray(parent, dtype=np.int64)
        self.Dm, self.vol, self.Dminv, self.G = element.rest_shape(self.X, self.T)
        if np.any(self.vol <= 0):
            raise ValueError("rest tet with non-positive volume")
        self.mu = np.broadcast_to(np.asarray(mu, dtype=np.float64), (self.m,)).copy()
        self.lam = np.broadcast_to(np.asarray(lam, dtype=np.float64), (self.m,)).copy()
        self.rule = cluster_rule
        if tet_cluster is not None:
            self.cluster = np.asarray(tet_cluster, dtype=np.int64)
        else:
            self.cluster = rig.cluster_tets(self.X, self.T, self.joints, self.parent, cluster_rule)
        self.vhandle = rig.vertex_handles(self.X, self.joints, self.parent, cluster_rule)
        if pin_verts is not None:
            self.pin_verts = np.asarray(pin_verts, dtype=np.int64)
            self.pin_handle = np.asarray(pin_handle, dtype=np.int64)
        else:
            self.pin_verts, self.pin_handle = rig.select_pins(
                self.X, self.joints, self.parent, pin_radius, cluster_rule)
        self.bbox_diag = float(np.linalg.norm(self.X.max(axis=0) - self.X.min(axis=0)))

    @classmethod
    def from_config(cls, cfg, **over):
        kw = dict(X=cfg["X"], T=cfg["T"], joints=cfg["joints"], parent=cfg["parent"],
                  mu=cfg["mu"], lam=cfg["lam"], cluster_rule=cfg["cluster_rule"],
                  pin_verts=cfg.get("pin_verts"), pin_handle=cfg.get("pin_handle"),
                  pin_radius=cfg.get("pin_radius", 0.0))
        kw.update(over)
        return cls(**kw)


def initial_guess(st, Q, t, init):
    if isinstance(init, str):
        if init == "rest":
            return st.X.copy()
        if init in ("rigid", "corot"):
            return np.einsum("kij,kj->ki", Q[st.vhandle], st.X) + t[st.vhandle]
        raise ValueError(init)
    return np.array(init, dtype=np.float64, copy=True)


def _pcg(K, b, tol, maxit):
    """FP64 CG with Jacobi preconditioning, relative residual tol."""
    d = K.diagonal()
    x = np.zeros_like(b)
    r = b.copy()
    z = r / d
    p = z.copy()
    rz = r @ z
    bn = np.linalg.norm(b)
    it = 0
    while np.linalg.norm(r) > tol * bn and it < maxit:
        q = K @ p
        a = rz / (p @ q)
        x += a * p
        r -= a * q
        z = r / d
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
    return x, it


def solve(st, xf, model, constraint="eliminate", ks=0.0, newton_max=50, newton_tol=1e-12,
          init="corot", linear="direct", cg_tol=1e-13, cg_max=100000, f_ext=None, rotation="rig"):
    """Solve one pose.  Returns (x (n,3), info dict).  f_ext: (n,3) external
    vertex forces or None; rotation: "rig" or "polar"."""
    if rotation not in ("rig", "polar"):
        raise ValueError(rotation)
    Q, t = rig.unpack_pose(xf)
    fv = np.zeros((st.n, 3)) if f_ext is None else np.asarray(f_ext, dtype=np.float64).reshape(st.n, 3)
    R_rig = Q[st.cluster]

    def rot(y):
        if rotation == "rig":
            return R_rig
        return diag.polar(element.deformation_gradient(y, st.T, st.G))[0]

    xp = rig.pin_targets(st.X, st.pin_verts, st.pin_handle, Q, t)
    x = initial_guess(st, Q, t, init)
    x[st.pin_verts] = xp
    n = st.n
    free = np.ones((n, 3), dtype=bool)
    if constraint == "eliminate":
        free[st.pin_verts] = False
    elif constraint != "penalty":
        raise ValueError(constraint)
    fidx = np.nonzero(free.reshape(-1))[0]

    def newton_direction(y, g, mdl):
        a = (st.T, st.G, st.vol, rot(y), mdl, st.mu, st.lam)
        Ke = element.element_hessians(y, *a, project=True)
        K = element.assemble(Ke, st.T, n)
        if constraint == "penalty":
            pd = (3 * st.pin_verts[:, None] + np.arange(3)).reshape(-1)
            K = K + sp.coo_matrix((np.full(len(pd), ks), (pd, pd)), shape=K.shape).tocsr()
        Kff = K[fidx][:, fidx].tocsc()
        if linear == "direct":
            return spla.spsolve(Kff, -g), 0
        return _pcg(Kff.tocsr(), -g, cg_tol, cg_max)

    def energy(y):
        e = element.element_energy(y, st.T, st.G, st.vol, rot(y), model, st.mu, st.lam).sum() \
            - np.einsum("ij,ij->", fv, y)
        if constraint == "penalty":
            d = y[st.pin_verts] - xp
            e += 0.5 * ks * np.einsum("ij,ij->", d, d)
        return e

    def grad(y):
        g = element.gradient(y, st.T, st.G, st.vol, rot(y), model, st.mu, st.lam) - fv
        if constraint == "penalty":
            np.add.at(g, st.pin_verts, ks * (y[st.pin_verts] - xp))
        return g

    info = dict(gnorm=[], alpha=[], energy=[], cg_iters=[], converged=False)
    x_ref = initial_guess(st, Q, t, "rigid")
    x_ref[st.pin_verts] = xp
    g0 = float(np.linalg.norm(grad(x_ref).reshape(-1)[fidx]))
    n_pred = 0
    if isinstance(init, str) and init == "corot" and model == "snh" and newton_max > 0:
        gc = element.gradient(x, st.T, st.G, st.vol, rot(x), "corot", st.mu, st.lam) - fv
        if constraint == "penalty":
            np.add.at(gc, st.pin_verts, ks * (x[st.pin_verts] - xp))
        df, cit = newton_direction(x, gc.reshape(-1)[fidx], "corot")
        d = np.zeros(3 * n)
        d[fidx] = df
        x = x + d.reshape(n, 3)
        info["cg_iters"].append(cit)
        info["alpha"].append(1.0)
        n_pred = 1
    for it in range(n_pred, newton_max + 1):
        g = grad(x).reshape(-1)[fidx]
        gn = float(np.linalg.norm(g))
        info["gnorm"].append(gn)
        if gn == 0.0 or gn <= newton_tol * g0:
            info["converged"] = True
            break
        if it == newton_max:
            break
        df, cit = newton_direction(x, g, model)
        info["cg_iters"].append(cit)
        d = np.zeros(3 * n)
        d[fidx] = df
        d = d.reshape(n, 3)
        alpha = 1.0
        if model == "snh" or rotation == "polar":
            e0 = energy(x)
            slope = float(g @ df)
            if -slope > LS_NOISE * abs(e0):
                for k in range(LS_MAX + 1):
                    alpha = 0.5 ** k
                    if energy(x + alpha * d) <= e0 + LS_C * alpha * slope:
                        break
            info["energy"].append(e0)
        info["alpha"].append(alpha)
        x = x + alpha * d
    info["newton_iters"] = len(info["alpha"])
    info["g0"] = g0
    info["final_rel_grad"] = info["gnorm"][-1] / g0 if g0 else 0.0
    info["final_energy"] = energy(x)
    return x, info


def element_outputs(st, xf, model, x, rotation="rig"):
    """s_k (Mandel 6-vector) and lambda_k (3x3, row-major 9) at x (Eq. 10-11)."""
    from .mandel import to_mandel
    Q, _ = rig.unpack_pose(xf)
    F = element.deformation_gradient(x, st.T, st.G)
    R = Q[st.cluster] if rotation == "rig" else diag.polar(F)[0]
    s = to_mandel(element.stretch(R, F))
    lam = element.multiplier(x, st.T, st.G, R, model, st.mu, st.lam)
    return s, lam.reshape(-1, 9)
