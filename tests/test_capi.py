"""The C-ABI library without a GPU: it builds, loads, exports every symbol the
header declares, and its host-only planning matches the oracle."""
import re
import os

import numpy as np
import pytest

from paper_2408_04066_gb300 import build as B
from paper_2408_04066_gb300 import mfem
from oracle import solve as S
from synth import bar_twist_config, figure_config, bar_mesh

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "mfem.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return mfem.load()


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mfem_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert lib.mfem_abi_version() == mfem.ABI_VERSION == 6
    # the binding declares the same set
    assert sorted(n for n, _, _ in mfem._SIGS) == names


def test_status_strings(lib):
    for s in range(8):
        assert lib.mfem_status_string(s)


@pytest.mark.parametrize("which", ["bar", "figure"])
def test_host_plan_matches_oracle(lib, which):
    cfg = bar_twist_config() if which == "bar" else figure_config(10000, seeds=[])
    tc, pinned, ph = mfem.plan(cfg["X"], cfg["T"], cfg["joints"], cfg["parent"], cfg["cluster_rule"],
                               cfg["pin_verts"], cfg["pin_handle"], cfg["pin_radius"])
    st = S.Setup.from_config(cfg)
    assert np.array_equal(tc, st.cluster)
    assert np.array_equal(np.nonzero(pinned)[0], np.sort(st.pin_verts))
    order = np.argsort(st.pin_verts)
    assert np.array_equal(ph[pinned], st.pin_handle[order])


def test_host_plan_rejects_bad_inputs(lib):
    X, T = bar_mesh(1, 1, 2)
    joints, parent = np.zeros((1, 3)), [-1]
    bad = T.copy()
    bad[3, 2] = len(X)
    with pytest.raises(mfem.MfemError) as e:
        mfem.plan(X, bad, joints, parent, pin_radius=0.5)
    assert e.value.status == mfem.MFEM_EINVAL and "out of range" in str(e.value)
    flip = T.copy()
    flip[5, [1, 2]] = flip[5, [2, 1]]            # inverted rest tet
    with pytest.raises(mfem.MfemError) as e:
        mfem.plan(X, flip, joints, parent, pin_radius=0.5)
    assert e.value.status == mfem.MFEM_EDEGEN and "tet 5" in str(e.value)
    Xn = X.copy()
    Xn[2, 1] = np.nan
    with pytest.raises(mfem.MfemError) as e:
        mfem.plan(Xn, T, joints, parent, pin_radius=0.5)
    assert e.value.status == mfem.MFEM_EINVAL
    with pytest.raises(mfem.MfemError) as e:
        mfem.plan(X, T, np.zeros((2, 3)), [-1, 1], pin_radius=0.5)     # a joint cannot parent itself
    assert "parent[1]" in str(e.value)
    with pytest.raises(mfem.MfemError):
        mfem.plan(X, T, np.zeros((1, 3)), [-1], pin_verts=[0, 0], pin_handle=[0, 0])


def test_user_clusters_override(lib):
    cfg = figure_config(3000, seeds=[])
    user = np.random.default_rng(0).integers(0, 15, size=len(cfg["T"]))
    tc, _, _ = mfem.plan(cfg["X"], cfg["T"], cfg["joints"], cfg["parent"], pin_radius=cfg["pin_radius"],
                         tet_cluster=user)
    assert np.array_equal(tc, user)


@pytest.mark.parametrize("rule", ["joint", "midpoint"])
def test_host_plan_other_cluster_rules_match_oracle(lib, rule):
    cfg = figure_config(10000, seeds=[])
    tc, pinned, ph = mfem.plan(cfg["X"], cfg["T"], cfg["joints"], cfg["parent"], rule, None, None,
                               cfg["pin_radius"])
    st = S.Setup.from_config(dict(cfg, cluster_rule=rule))
    assert np.array_equal(tc, st.cluster)
    assert np.array_equal(np.nonzero(pinned)[0], np.sort(st.pin_verts))


@pytest.mark.parametrize("rule", ["bone", "joint", "midpoint"])
@pytest.mark.parametrize("seed", range(4))
def test_host_plan_matches_oracle_on_grid_rigs_with_ties(lib, rule, seed):
    """Random voxel blobs with joints on the half-integer grid: many tet
    barycenters and vertices sit at exactly equal distances from two joints,
    bones or midpoints, so the tie rule (lowest index within the margin) is
    exercised, and the host planner must still agree with the oracle."""
    rng = np.random.default_rng(100 + seed)
    from synth.meshes import kuhn_voxel_mesh
    occ = rng.random((5, 4, 6)) < 0.6
    occ[2, 2, :] = True                                  # a spine through the blob
    X, T = kuhn_voxel_mesh(occ, 1.0)
    H = int(rng.integers(2, 7))
    joints = rng.integers(0, 11, size=(H, 3)) * 0.5
    joints[:, 0] = np.minimum(joints[:, 0], 5.0)
    joints[:, 1] = np.minimum(joints[:, 1], 4.0)
    parent = np.array([-1] + [int(rng.integers(0, j)) for j in range(1, H)], dtype=np.int32)
    for j in range(1, H):                                # no zero-length bones
        if np.allclose(joints[j], joints[parent[j]]):
            joints[j, 2] += 0.5
    cfg = dict(X=X, T=T, joints=joints, parent=parent, cluster_rule=rule, pin_verts=None, pin_handle=None,
               pin_radius=0.75, model="arap", mu=1.0, lam=0.0)
    tc, pinned, ph = mfem.plan(X, T, joints, parent, rule, None, None, cfg["pin_radius"])
    st = S.Setup.from_config(cfg)
    assert np.array_equal(tc, st.cluster)
    assert np.array_equal(np.nonzero(pinned)[0], np.sort(st.pin_verts))
    order = np.argsort(st.pin_verts)
    assert np.array_equal(ph[pinned], st.pin_handle[order])


def test_missing_library_fails_loudly(tmp_path):
    """No silent fallback: loading a library that is not there raises."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("from paper_2408_04066_gb300 import mfem\n"
            "try:\n"
            f"    mfem.load({str(tmp_path / 'libmfem.so')!r})\n"
            "except RuntimeError as e:\n"
            "    print('raised:', e)\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "raised:" in r.stdout and "is missing" in r.stdout


def test_context_without_a_gpu_is_an_error(lib):
    """Without a CUDA device, creating a context returns MFEM_ECUDA: the
    product path has no CPU fallback."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    cfg = bar_twist_config()
    with pytest.raises(mfem.MfemError) as e:
        mfem.Context.from_config(cfg, precision="fp64")
    assert e.value.status == mfem.MFEM_ECUDA


def _header_struct_fields(name):
    """Field names and C types of `typedef struct { ... } name;` in the header,
    in declaration order (comments stripped; `double a, b;` gives two fields)."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    body = re.search(r"typedef struct \{([^}]*)\}\s*" + name + r"\s*;", text).group(1)
    fields = []
    for decl in body.split(";"):
        decl = " ".join(decl.split())
        if not decl:
            continue
        m = re.match(r"((?:const )?[A-Za-z_0-9]+\s*\**)\s*(.*)", decl)
        ctype, names = m.group(1).replace(" ", ""), m.group(2)
        for n in names.split(","):
            n = n.strip()
            stars = len(n) - len(n.lstrip("*"))
            fields.append((n.lstrip("*"), ctype + "*" * stars))
    return fields


_CTYPE = {"int32_t": "c_int", "double": "c_double", "int64_t": "c_long", "size_t": "c_ulong"}


@pytest.mark.parametrize("cname,pyname", [("mfem_material", "Material"), ("mfem_handles", "Handles"),
                                          ("mfem_options", "Options"), ("mfem_stats", "Stats"),
                                          ("mfem_profile", "Profile")])
def test_binding_structs_match_the_header(cname, pyname):
    """The ctypes structures declare the header's fields in the same order with
    the same widths, so no field is read at a shifted offset."""
    import ctypes as C
    hdr = _header_struct_fields(cname)
    py = getattr(mfem, pyname)._fields_
    assert [n.rstrip("_") for n, _ in py] == [n for n, _ in hdr]   # lambda_: a Python keyword
    for (n, t), (_, pt) in zip(hdr, py):
        if t.endswith("*"):
            assert C.sizeof(pt) == C.sizeof(C.c_void_p), n
        else:
            assert C.sizeof(pt) == C.sizeof(getattr(C, _CTYPE[t])), (n, t)
