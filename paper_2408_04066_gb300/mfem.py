"""Thin ctypes binding of libmfem.so (include/mfem.h), same names as the C ABI.

Argument marshalling only: every step of the pose solve runs in the CUDA
library.  Host arrays are numpy; device arrays are torch CUDA tensors (their
data pointers are passed through).  If the library is not built, loading fails
with an error -- there is no Python fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

MFEM_OK, MFEM_EINVAL, MFEM_EDEGEN, MFEM_ENOMEM, MFEM_ENOTCONV, MFEM_ETIMEOUT, MFEM_EBUSY, MFEM_ECUDA = range(8)
STATUS_NAMES = ["OK", "EINVAL", "EDEGEN", "ENOMEM", "ENOTCONV", "ETIMEOUT", "EBUSY", "ECUDA"]
MODELS = {"arap": 0, "corot": 1, "snh": 2}
PRECISIONS = {"fp64": 0, "mixed": 1}
CONSTRAINTS = {"eliminate": 0, "penalty": 1}
CLUSTER_RULES = {"bone": 0, "joint": 1, "midpoint": 2}
INITS = {"rigid": 0, "rest": 1, "warm": 2, "corot": 3}
ROTATIONS = {"rig": 0, "polar": 1}
PRECONDS = {"block_jacobi": 0, "two_level": 1}
LAUNCHES = {"graph": 0, "direct": 1}
COARSE_PRODUCTS = {"tc": 0, "fp32": 1}
MEM_HOST, MEM_DEVICE = 0, 1
ABI_VERSION = 6   # MFEM_ABI_VERSION of the header these structures follow

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


class Material(C.Structure):
    _fields_ = [("model", C.c_int32), ("mu", _dp), ("lambda_", _dp), ("mu0", C.c_double), ("lambda0", C.c_double)]


class Handles(C.Structure):
    _fields_ = [("n_handles", C.c_int32), ("joints", _dp), ("parent", _ip), ("tet_cluster", _ip),
                ("pin_verts", _ip), ("pin_handle", _ip), ("n_pins", C.c_int32), ("pin_radius", C.c_double),
                ("cluster_rule", C.c_int32)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("constraint", C.c_int32), ("k_s", C.c_double),
                ("newton_tol", C.c_double), ("cg_tol", C.c_double), ("newton_max", C.c_int32),
                ("cg_max", C.c_int32), ("init", C.c_int32), ("max_batch", C.c_int32),
                ("tile_rows", C.c_int32), ("diagnostics", C.c_int32), ("rotation", C.c_int32),
                ("precond", C.c_int32), ("launch", C.c_int32), ("coarse_agg", C.c_int32),
                ("spmv_split", C.c_int32), ("coarse_product", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("newton_iters", C.c_int32), ("pcg_iters", C.c_int32),
                ("converged", C.c_int32), ("grad0", C.c_double), ("rel_grad", C.c_double),
                ("energy", C.c_double), ("inverted", C.c_int32), ("max_rel_skew", C.c_double),
                ("max_angle", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Profile(C.Structure):
    _fields_ = [("kernel_launches", C.c_int32), ("pcg_launches", C.c_int32), ("pcg_ms", C.c_double),
                ("pcg_bytes", C.c_double), ("pcg_iters", C.c_int64), ("element_launches", C.c_int32),
                ("element_ms", C.c_double), ("element_bytes", C.c_double), ("assemble_ms", C.c_double),
                ("linesearch_ms", C.c_double), ("total_ms", C.c_double), ("tile_rows", C.c_int32),
                ("grid_blocks", C.c_int32), ("element_updates", C.c_int64), ("coarse_dof", C.c_int32),
                ("coarse_launches", C.c_int32), ("coarse_tc", C.c_int32), ("spmv_split", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None

# (name, restype, argtypes) for every function of include/mfem.h
_SIGS = [
    ("mfem_abi_version", C.c_int32, []),
    ("mfem_default_options", None, [C.POINTER(Options)]),
    ("mfem_status_string", C.c_char_p, [C.c_int32]),
    ("mfem_create", C.c_int32, [_dp, C.c_int32, _ip, C.c_int32, C.POINTER(Material), C.POINTER(Handles),
                                C.POINTER(Options), C.POINTER(C.c_void_p)]),
    ("mfem_set_stream", C.c_int32, [C.c_void_p, C.c_void_p]),
    ("mfem_set_pose", C.c_int32, [C.c_void_p, _dp, C.c_int32]),
    ("mfem_set_forces", C.c_int32, [C.c_void_p, _dp, C.c_int32]),
    ("mfem_solve", C.c_int32, [C.c_void_p, _dp, C.POINTER(Stats)]),
    ("mfem_solve_batch", C.c_int32, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_int32,
                                     C.POINTER(Stats)]),
    ("mfem_solve_multi", C.c_int32, [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(C.c_void_p), _ip,
                                     C.POINTER(C.c_void_p), C.c_int32, C.POINTER(C.c_void_p)]),
    ("mfem_get_elem", C.c_int32, [C.c_void_p, _dp, _dp]),
    ("mfem_get_elem_static", C.c_int32, [C.c_void_p, _dp, _dp]),
    ("mfem_coarse_apply", C.c_int32, [C.c_void_p, C.POINTER(C.c_float), C.c_int32, C.POINTER(C.c_float),
                                      C.c_int32]),
    ("mfem_get_state", C.c_int32, [C.c_void_p, _dp]),
    ("mfem_set_state", C.c_int32, [C.c_void_p, _dp]),
    ("mfem_get_profile", C.c_int32, [C.c_void_p, C.POINTER(Profile)]),
    ("mfem_get_info", C.c_int32, [C.c_void_p, _ip, _ip, _ip, _ip, C.POINTER(C.c_int64),
                                  C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    ("mfem_plan", C.c_int32, [_dp, C.c_int32, _ip, C.c_int32, C.POINTER(Handles), _ip, _ip, _ip]),
    ("mfem_destroy", None, [C.c_void_p]),
    ("mfem_last_error", C.c_char_p, [C.c_void_p]),
    ("mfem_server_create", C.c_int32, [C.c_size_t, C.c_int32, C.POINTER(C.c_void_p)]),
    ("mfem_server_add", C.c_int32, [C.c_void_p, C.c_void_p, _ip]),
    ("mfem_server_submit", C.c_int32, [C.c_void_p, C.c_int32, _dp, _dp, C.POINTER(C.c_uint64)]),
    ("mfem_server_wait", C.c_int32, [C.c_void_p, C.c_uint64, C.c_int32, C.POINTER(Stats),
                                     C.POINTER(C.c_double)]),
    ("mfem_server_counters", C.c_int32, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                         C.POINTER(C.c_int64), _ip, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                         C.POINTER(C.c_int64)]),
    ("mfem_server_destroy", None, [C.c_void_p]),
]


def lib_path():
    return _build.LIB


def load(path=None):
    """Load libmfem.so (raises if it is missing: build it first)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2408_04066_gb300.build.build()")
    lib = C.CDLL(path)
    for name, res, args in _SIGS:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if lib.mfem_abi_version() != ABI_VERSION:
        raise RuntimeError(f"{path} has ABI version {lib.mfem_abi_version()}, the binding expects "
                           f"{ABI_VERSION}: rebuild it")
    _lib = lib
    return lib


class MfemError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


def _check(st, ctx=None):
    if st != MFEM_OK:
        raise MfemError(st, load().mfem_last_error(ctx).decode())


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a, t=_dp):
    return None if a is None else a.ctypes.data_as(t)


def default_options(**over):
    o = Options()
    load().mfem_default_options(C.byref(o))
    for k, v in over.items():
        if k == "precision":
            v = PRECISIONS[v] if isinstance(v, str) else v
        elif k == "constraint":
            v = CONSTRAINTS[v] if isinstance(v, str) else v
        elif k == "init":
            v = INITS[v] if isinstance(v, str) else v
        elif k == "rotation":
            v = ROTATIONS[v] if isinstance(v, str) else v
        elif k == "precond":
            v = PRECONDS[v] if isinstance(v, str) else v
        elif k == "launch":
            v = LAUNCHES[v] if isinstance(v, str) else v
        elif k == "coarse_product":
            v = COARSE_PRODUCTS[v] if isinstance(v, str) else v
        setattr(o, k, v)
    return o


def _handles(n_h, joints, parent, cluster_rule, pin_verts, pin_handle, pin_radius, tet_cluster, keep):
    j = _f64(joints, (-1, 3))
    par = _i32(parent)
    keep += [j, par]
    h = Handles()
    h.n_handles = n_h
    h.joints = _p(j)
    h.parent = _p(par, _ip)
    if tet_cluster is not None:
        tc = _i32(tet_cluster)
        keep.append(tc)
        h.tet_cluster = _p(tc, _ip)
    if pin_verts is not None:
        pv, ph = _i32(pin_verts), _i32(pin_handle)
        keep += [pv, ph]
        h.pin_verts = _p(pv, _ip)
        h.pin_handle = _p(ph, _ip)
        h.n_pins = len(pv)
    h.pin_radius = float(pin_radius or 0.0)
    h.cluster_rule = CLUSTER_RULES[cluster_rule] if isinstance(cluster_rule, str) else cluster_rule
    return h


def plan(X, T, joints, parent, cluster_rule="bone", pin_verts=None, pin_handle=None, pin_radius=0.0,
         tet_cluster=None):
    """mfem_plan: host-only clusters and pins (caller order)."""
    lib = load()
    X = _f64(X, (-1, 3))
    T = _i32(T).reshape(-1, 4)
    keep = []
    h = _handles(len(_f64(joints, (-1, 3))), joints, parent, cluster_rule, pin_verts, pin_handle, pin_radius,
                 tet_cluster, keep)
    tc = np.zeros(len(T), np.int32)
    pinned = np.zeros(len(X), np.int32)
    ph = np.zeros(len(X), np.int32)
    _check(lib.mfem_plan(_p(X), len(X), _p(T, _ip), len(T), C.byref(h), _p(tc, _ip), _p(pinned, _ip),
                         _p(ph, _ip)))
    return tc, pinned.astype(bool), ph


class Context:
    """mfem_create / mfem_set_pose / mfem_solve / mfem_solve_batch ... for one mesh."""

    def __init__(self, X, T, joints, parent, model="arap", mu=1.0, lam=0.0, cluster_rule="bone",
                 pin_verts=None, pin_handle=None, pin_radius=0.0, tet_cluster=None, **options):
        lib = load()
        self._lib = lib
        X = _f64(X, (-1, 3))
        T = _i32(T).reshape(-1, 4)
        self.n, self.m = len(X), len(T)
        keep = []
        mat = Material()
        mat.model = MODELS[model] if isinstance(model, str) else model
        mu_a, lam_a = np.asarray(mu, dtype=np.float64), np.asarray(lam, dtype=np.float64)
        if mu_a.ndim:
            mu_a = _f64(mu_a)
            keep.append(mu_a)
            mat.mu = _p(mu_a)
        else:
            mat.mu0 = float(mu_a)
        if lam_a.ndim:
            lam_a = _f64(lam_a)
            keep.append(lam_a)
            mat.lambda_ = _p(lam_a)
        else:
            mat.lambda0 = float(lam_a)
        self.H = len(_f64(joints, (-1, 3)))
        h = _handles(self.H, joints, parent, cluster_rule, pin_verts, pin_handle, pin_radius, tet_cluster, keep)
        self.options = default_options(**options)
        ptr = C.c_void_p()
        st = lib.mfem_create(_p(X), self.n, _p(T, _ip), self.m, C.byref(mat), C.byref(h),
                             C.byref(self.options), C.byref(ptr))
        _check(st, None)
        self._ctx = ptr

    @classmethod
    def from_config(cls, cfg, **options):
        """Build from a workload dict with keys X, T, joints, parent, model, mu, lam,
        cluster_rule, pin_verts, pin_handle, pin_radius."""
        return cls(cfg["X"], cfg["T"], cfg["joints"], cfg["parent"], model=cfg["model"], mu=cfg["mu"],
                   lam=cfg["lam"], cluster_rule=cfg["cluster_rule"], pin_verts=cfg.get("pin_verts"),
                   pin_handle=cfg.get("pin_handle"), pin_radius=cfg.get("pin_radius", 0.0), **options)

    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.mfem_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def release(self):
        """Give up ownership (after mfem_server_add)."""
        p = self._ctx
        self._ctx = None
        return p

    def set_stream(self, stream):
        _check(self._lib.mfem_set_stream(self._ctx, C.c_void_p(int(stream) if stream else 0)), self._ctx)

    def set_pose(self, xf):
        xf = _f64(xf, (-1, 12))
        _check(self._lib.mfem_set_pose(self._ctx, _p(xf), len(xf)), self._ctx)

    def set_forces(self, f):
        """External vertex forces: (n,3) for every pose, (S,n,3) for pose b of a
        batch taking field b, or None to remove them."""
        if f is None:
            _check(self._lib.mfem_set_forces(self._ctx, None, 0), self._ctx)
            return
        f = _f64(f)
        sets = 1 if f.ndim == 2 else f.shape[0]
        f = _f64(f, (sets, self.n, 3))
        _check(self._lib.mfem_set_forces(self._ctx, _p(f), sets), self._ctx)

    def solve(self, out=None):
        out = np.empty((self.n, 3)) if out is None else out
        st = Stats()
        s = self._lib.mfem_solve(self._ctx, _p(out), C.byref(st))
        if s not in (MFEM_OK, MFEM_ENOTCONV):
            _check(s, self._ctx)
        return out, st.as_dict()

    def solve_batch(self, xfs, out=None, raise_on_notconv=False):
        """xfs: numpy (B,H,12) host array or torch CUDA tensor.  Returns (out, stats)."""
        dev = hasattr(xfs, "is_cuda") and xfs.is_cuda
        if dev:
            import torch
            B = xfs.shape[0]
            assert xfs.dtype == torch.float64 and xfs.is_contiguous()
            if out is None:
                out = torch.empty((B, self.n, 3), dtype=torch.float64, device=xfs.device)
            xp, op, mem = C.c_void_p(xfs.data_ptr()), C.c_void_p(out.data_ptr()), MEM_DEVICE
        else:
            xfs = _f64(xfs, (-1, self.H, 12))
            B = xfs.shape[0]
            if out is None:
                out = np.empty((B, self.n, 3))
            xp, op, mem = C.c_void_p(xfs.ctypes.data), C.c_void_p(out.ctypes.data), MEM_HOST
        stats = (Stats * B)()
        s = self._lib.mfem_solve_batch(self._ctx, xp, B, op, mem, stats)
        if s != MFEM_OK and (s != MFEM_ENOTCONV or raise_on_notconv):
            _check(s, self._ctx)
        return out, [st.as_dict() for st in stats]

    def get_elem(self):
        s = np.empty((self.m, 6))
        lam = np.empty((self.m, 9))
        _check(self._lib.mfem_get_elem(self._ctx, _p(s), _p(lam)), self._ctx)
        return s, lam

    def get_elem_static(self, s=None, lam=None):
        """mfem_get_elem_static: same outputs, staged through the library's
        fixed device array (no device allocation)."""
        s = np.empty((self.m, 6)) if s is None else s
        lam = np.empty((self.m, 9)) if lam is None else lam
        _check(self._lib.mfem_get_elem_static(self._ctx, _p(s), _p(lam)), self._ctx)
        return s, lam

    def coarse_apply(self, rc, product="tc"):
        """mfem_coarse_apply: e_b = A_c^{-1} rc_b as the solve computes it, rc
        (B, N) float32 in the mesh's coarse basis; product "tc" or "fp32"."""
        rc = np.ascontiguousarray(rc, dtype=np.float32)
        if rc.ndim == 1:
            rc = rc[None]
        e = np.empty_like(rc)
        fp = C.POINTER(C.c_float)
        _check(self._lib.mfem_coarse_apply(self._ctx, rc.ctypes.data_as(fp), rc.shape[0], e.ctypes.data_as(fp),
                                           COARSE_PRODUCTS[product] if isinstance(product, str) else product),
               self._ctx)
        return e

    def get_state(self):
        x = np.empty((self.n, 3))
        _check(self._lib.mfem_get_state(self._ctx, _p(x)), self._ctx)
        return x

    def set_state(self, x):
        x = _f64(x, (-1, 3))
        _check(self._lib.mfem_set_state(self._ctx, _p(x)), self._ctx)

    def profile(self):
        p = Profile()
        _check(self._lib.mfem_get_profile(self._ctx, C.byref(p)), self._ctx)
        return p.as_dict()

    def info(self):
        n, m, H, npins = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        nnz, slots, byts = C.c_int64(), C.c_int64(), C.c_int64()
        _check(self._lib.mfem_get_info(self._ctx, C.byref(n), C.byref(m), C.byref(H), C.byref(npins),
                                       C.byref(nnz), C.byref(slots), C.byref(byts)), self._ctx)
        return dict(n=n.value, m=m.value, n_handles=H.value, n_pins=npins.value, nnz_blocks=nnz.value,
                    sell_slots=slots.value, device_bytes=byts.value)


def solve_multi(ctxs, xfs, outs=None, raise_on_notconv=False):
    """mfem_solve_multi: xfs[i] (B_i,H_i,12) poses of Context ctxs[i] -- all numpy
    host arrays or all torch CUDA float64 tensors.  Returns (outs, stats)."""
    lib = load()
    k = len(ctxs)
    dev = hasattr(xfs[0], "is_cuda") and xfs[0].is_cuda
    if dev:
        import torch
        assert all(x.dtype == torch.float64 and x.is_contiguous() for x in xfs)
        if outs is None:
            outs = [torch.empty((x.shape[0], c.n, 3), dtype=torch.float64, device=x.device)
                    for c, x in zip(ctxs, xfs)]
        xp = [x.data_ptr() for x in xfs]
        op = [o.data_ptr() for o in outs]
        mem = MEM_DEVICE
    else:
        xfs = [_f64(x, (-1, c.H, 12)) for c, x in zip(ctxs, xfs)]
        if outs is None:
            outs = [np.empty((x.shape[0], c.n, 3)) for c, x in zip(ctxs, xfs)]
        xp = [x.ctypes.data for x in xfs]
        op = [o.ctypes.data for o in outs]
        mem = MEM_HOST
    Bs = (C.c_int32 * k)(*[int(x.shape[0]) for x in xfs])
    stats = [(Stats * int(x.shape[0]))() for x in xfs]
    st_ptrs = (C.c_void_p * k)(*[C.cast(s, C.c_void_p) for s in stats])
    cp = (C.c_void_p * k)(*[c._ctx.value for c in ctxs])
    s = lib.mfem_solve_multi(cp, k, (C.c_void_p * k)(*xp), Bs, (C.c_void_p * k)(*op), mem, st_ptrs)
    if s != MFEM_OK and (s != MFEM_ENOTCONV or raise_on_notconv):
        _check(s, ctxs[0]._ctx)
    return outs, [[st.as_dict() for st in ss] for ss in stats]


class Server:
    """mfem_server_*: continuous batching over resident meshes."""

    def __init__(self, device_mem_budget=0, max_slots=16):
        self._lib = load()
        p = C.c_void_p()
        _check(self._lib.mfem_server_create(device_mem_budget, max_slots, C.byref(p)))
        self._srv = p
        self._meshes = {}
        self._bufs = {}

    def add(self, ctx: Context):
        mid = C.c_int32()
        _check(self._lib.mfem_server_add(self._srv, ctx._ctx, C.byref(mid)))
        self._meshes[mid.value] = (ctx.n, ctx.H)
        ctx.release()
        return mid.value

    def submit(self, mesh_id, xf, out=None):
        if mesh_id not in self._meshes:
            raise MfemError(MFEM_EINVAL, f"unknown mesh id {mesh_id}")
        n, H = self._meshes[mesh_id]
        xf = _f64(xf, (H, 12))
        out = np.empty((n, 3)) if out is None else out
        t = C.c_uint64()
        _check(self._lib.mfem_server_submit(self._srv, mesh_id, _p(xf), _p(out), C.byref(t)))
        self._bufs[t.value] = out
        return t.value

    def wait(self, ticket, timeout_ms=-1):
        st = Stats()
        lat = C.c_double()
        s = self._lib.mfem_server_wait(self._srv, ticket, timeout_ms, C.byref(st), C.byref(lat))
        if s == MFEM_ETIMEOUT:
            return None
        out = self._bufs.pop(ticket)
        if s not in (MFEM_OK, MFEM_ENOTCONV):
            _check(s)
        return out, st.as_dict(), lat.value

    def counters(self):
        a, b, c, e, f, g = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        d = C.c_int32()
        _check(self._lib.mfem_server_counters(self._srv, C.byref(a), C.byref(b), C.byref(c), C.byref(d), C.byref(e),
                                              C.byref(f), C.byref(g)))
        return dict(completed=a.value, steps=b.value, pcg_launches=c.value, peak_slots=d.value,
                    pools_added=e.value, pools_released=f.value, device_bytes=g.value)

    def close(self):
        if getattr(self, "_srv", None):
            self._lib.mfem_server_destroy(self._srv)
            self._srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
