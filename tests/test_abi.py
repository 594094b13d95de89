"""C-ABI checks that need no GPU: exports, host mesh, argument validation."""
import ctypes as ct
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def g():
    import paper_2512_11590_gb300 as mod
    if not os.path.exists(mod.LIB_PATH):
        from paper_2512_11590_gb300.build import build
        build()
    mod.lib()
    return mod


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(rmat_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(g):
    names = declared_functions()
    assert len(names) >= 12
    L = ct.CDLL(g.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    assert set(g.EXPORTED) <= set(names)


def test_python_constants_match_header(g):
    """Every RMAT_* integer the binding defines has the header's value, and every
    RMAT_PARAM_* of the header has a binding constant."""
    src = open(os.path.join(ROOT, "include", "rmat.h")).read()
    defs = dict(re.findall(r"^#define\s+(RMAT_\w+)\s+\(?(-?\d+)\)?", src, flags=re.M))
    assert len(defs) > 20
    for name, val in defs.items():
        if hasattr(g, name):
            assert getattr(g, name) == int(val), name
    for name in defs:
        if name.startswith("RMAT_PARAM_"):
            assert hasattr(g, name), name


@pytest.mark.parametrize("n,a", [(1, 3.0), (4, 15.0), (50, 15.0), (100, 15.0), (60, 18.0), (137, 7.5)])
def test_library_mesh_bitwise_equals_oracle(g, n, a):
    from oracle import mesh as M
    m = g.rmat_mesh(n, a)
    o = M.lagrange_mesh(n, a)
    for k in ("x", "omx", "r", "f_a"):
        assert np.array_equal(m[k], o[k]), k
    assert np.array_equal(m["T0"], M.kinetic_bloch(n, a, o))
    np.testing.assert_allclose(m["lam"], o["lam"], rtol=1e-15)


def test_mesh_argument_errors(g):
    d = ct.POINTER(ct.c_double)()
    assert g.lib().rmat_mesh(0, 1.0, d, d, d, d, d, d) == -1
    assert g.lib().rmat_mesh(10, -1.0, d, d, d, d, d, d) == -2
    assert g.lib().rmat_mesh(10, float("nan"), d, d, d, d, d, d) == -2


def test_null_context_arguments(g):
    L = g.lib()
    assert L.rmat_create(None, 0, None) == -1
    assert L.rmat_factor(None, None) == -1
    assert L.rmat_solve(None, None, 1, 0, 0.0, None, None) == -1
    assert L.rmat_set_param(None, 1, 64) == -1
    assert L.rmat_set_param(None, g.RMAT_PARAM_METHOD, 1) == -1
    assert L.rmat_propagate(None, None, 10.0, 1, None, None, 0, 0.0, None, None, None) == -1
    assert L.rmat_destroy(None) == 0
    assert g.status_string(g.RMAT_ENOCONV).startswith("refinement")
    assert "Coulomb" in g.status_string(g.RMAT_ECHANFN)


def test_no_gpu_fails_loudly(g):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ct.c_void_p()
    assert g.lib().rmat_create(ct.byref(h), 0, None) in (g.RMAT_ENODEV, g.RMAT_ECUDA)


@pytest.mark.parametrize("n,r1,r2", [(2, 0.0, 3.0), (10, 4.0, 9.0), (60, 15.0, 30.0), (150, 5.0, 25.0)])
def test_library_sector_mesh_matches_oracle(g, n, r1, r2):
    """Host sector mesh (closed-form barycentric weights, negative-sum diagonal)
    against the oracle's (log-product weights, explicit diagonal sums)."""
    from oracle import propagation as P
    m = g.rmat_sector_mesh(n, r1, r2)
    o = P.sector_mesh(n, r1, r2)
    np.testing.assert_allclose(m["r"], o["r"], rtol=1e-15)
    np.testing.assert_allclose(m["lam"], o["lam"], rtol=1e-14)
    for k in ("fL", "fR"):
        assert np.max(np.abs(m[k] - o[k])) <= 1e-11 * np.max(np.abs(o[k])), k
    assert np.max(np.abs(m["Kf"] - o["Kf"])) <= 1e-10 * np.max(np.abs(o["Kf"]))


def test_sector_mesh_argument_errors(g):
    d = ct.POINTER(ct.c_double)()
    assert g.lib().rmat_sector_mesh(1, 0.0, 1.0, d, d, d, d, d) == -1
    assert g.lib().rmat_sector_mesh(10, 2.0, 2.0, d, d, d, d, d) == -2
    assert g.lib().rmat_sector_mesh(10, -1.0, 2.0, d, d, d, d, d) == -2
