"""The C ABI library builds, loads and exports every symbol include/mam.h
declares; argument validation happens before any device call, so the
invalid-argument paths are checked here without a GPU."""
import ctypes as C
import math
import os
import re

import numpy as np
import pytest

from paper_2309_05315_gb300 import _capi
from paper_2309_05315_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build()
    return _capi.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mam.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mam_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    # and the Python binding declares every one of them
    assert set(names) <= set(_capi.exported_names())


def make_desc(M=2, R=4, S=(3, 3), q=None, gamma=math.inf, rho=1.0, **kw):
    S = np.asarray(S, dtype=np.int32)
    n = int(S.sum())
    q = np.full(n, 1.0 / S[0]) if q is None else np.asarray(q, dtype=np.float64)
    keep = dict(S=S, q=q, zeta=np.zeros((n, 2)), alpha=np.full(M, 1.0 / M),
                xi=np.zeros((R, 2)))
    d = _capi.MamDesc()
    d.M, d.R, d.dim = M, R, 2
    d.S = keep["S"].ctypes.data_as(C.POINTER(C.c_int32))
    for k in ("q", "zeta", "alpha", "xi"):
        setattr(d, k, keep[k].ctypes.data_as(C.POINTER(C.c_double)))
    d.cost = None
    d.rho, d.gamma = rho, gamma
    d.n_bundles, d.seed, d.cost_dtype, d.theta0_mode, d.diag_mode = 0, 0, 0, 0, 0
    d.stream = None
    for k, v in kw.items():
        setattr(d, k, v)
    return d, keep


@pytest.mark.parametrize("case", [
    dict(M=0),
    dict(R=0),
    dict(R=20000),
    dict(dim=4),
    dict(rho=0.0),
    dict(rho=-1.0),
    dict(rho=1e-35),
    dict(rho=1e35),
    dict(gamma=-0.5),
    dict(cost_dtype=7),
    dict(theta0_mode=3),
    dict(n_bundles=5),
    dict(capped=2),
    dict(capped=1, eta=-1.0),
    dict(capped=1, eta=float("nan")),
    dict(capped=1, eta=float("inf")),
    dict(eta=0.5),  # eta without capped columns
])
def test_invalid_descriptor_fields(L, case):
    d, keep = make_desc()
    for k, v in case.items():
        setattr(d, k, v)
    h = C.c_void_p()
    st = L.mam_create(C.byref(d), C.byref(h))
    assert st == 1 and not h.value
    assert len(L.mam_last_error(None)) > 0


@pytest.mark.parametrize("q", [
    [0.5, 0.5, 0.0, 0.4, 0.6, float("nan")],   # NaN weight
    [0.5, 0.5, 0.0, -0.1, 0.6, 0.5],           # negative weight
    [0.0, 0.0, 0.0, 0.4, 0.6, 0.0],            # measure without mass
    [0.5, 0.5, 0.0, 0.4, 0.7, 0.0],            # unequal masses, balanced
])
def test_invalid_weights(L, q):
    d, keep = make_desc(q=q)
    h = C.c_void_p()
    assert L.mam_create(C.byref(d), C.byref(h)) == 1
    assert not h.value


def test_capped_columns_allow_unequal_masses(L):
    """Validation accepts unequal masses when the columns are capped (the
    call then fails later, on the device allocation of a GPU-less host, or
    succeeds on a GPU)."""
    q = [0.5, 0.5, 0.0, 0.4, 0.7, 0.0]
    d, keep = make_desc(q=q, capped=1, eta=0.25)
    h = C.c_void_p()
    st = L.mam_create(C.byref(d), C.byref(h))
    assert st != 1, L.mam_last_error(None)
    if h.value:
        L.mam_destroy(h)


def test_null_arguments(L):
    assert L.mam_step(None, 1) == 1
    assert L.mam_objective(None, 0, None) == 1
    assert L.mam_objective_all(None, None) == 1
    assert L.mam_create(None, None) == 1
    L.mam_destroy(None)  # allowed


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(_capi, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_capi, "_lib", None)
    with pytest.raises(ImportError):
        _capi.lib()


def test_shared_cost_layout_needs_one_support(L):
    """MAM_COST_SHARED: every measure must have the same support points, and
    the cost must be the squared Euclidean one; checked before any device
    call."""
    d, keep = make_desc(S=(3, 3), cost_layout=1)
    zeta = np.zeros((6, 2))
    zeta[4, 1] = 0.5                                  # measure 1 differs in one point
    keep["zeta"] = zeta
    d.zeta = zeta.ctypes.data_as(C.POINTER(C.c_double))
    h = C.c_void_p()
    assert L.mam_create(C.byref(d), C.byref(h)) == 1
    assert b"same support" in L.mam_last_error(None)
    d2, keep2 = make_desc(S=(3, 2), cost_layout=1, q=[1 / 3] * 3 + [0.5, 0.5])
    assert L.mam_create(C.byref(d2), C.byref(h)) == 1
    cost = np.ones((5, 4))
    d3, keep3 = make_desc(S=(3, 2), q=[1 / 3] * 3 + [0.5, 0.5], cost_layout=1)
    d3.cost = cost.ctypes.data_as(C.POINTER(C.c_double))
    assert L.mam_create(C.byref(d3), C.byref(h)) == 1
    assert b"cost = NULL" in L.mam_last_error(None)
    d4, keep4 = make_desc(cost_layout=3)
    assert L.mam_create(C.byref(d4), C.byref(h)) == 1
    assert b"cost_layout" in L.mam_last_error(None)


def test_generated_and_shared_layouts_need_positive_alpha(L):
    d, keep = make_desc(cost_layout=2)
    keep["alpha"][:] = [1.0, 0.0]
    h = C.c_void_p()
    assert L.mam_create(C.byref(d), C.byref(h)) == 1
    assert b"alpha_m > 0" in L.mam_last_error(None)


@pytest.mark.parametrize("case", [
    dict(plan_layout=2),
    dict(plan_layout=1, sparse_slots=3),      # odd
    dict(plan_layout=1, sparse_slots=-2),
    dict(plan_layout=1, sparse_slots=10),     # above round_up(R, 8) = 8
    dict(sparse_slots=8),                     # slots without the sparse layout
    dict(plan_layout=1, cost_layout=2),       # generated costs
])
def test_invalid_plan_layout_fields(L, case):
    d, keep = make_desc(**case)
    h = C.c_void_p()
    assert L.mam_create(C.byref(d), C.byref(h)) == 1
    assert not h.value
    assert len(L.mam_last_error(None)) > 0


def test_sparse_layout_needs_one_cta_per_column(L):
    """The sparse plan layout runs on the one-CTA-per-column kernel: R up to
    12288 (round_up(R, 8) <= 12288)."""
    d, keep = make_desc(R=12289, plan_layout=1)
    h = C.c_void_p()
    assert L.mam_create(C.byref(d), C.byref(h)) == 1
    assert b"12288" in L.mam_last_error(None)
    d, keep = make_desc(R=12288, plan_layout=1)
    h = C.c_void_p()
    st = L.mam_create(C.byref(d), C.byref(h))  # valid: fails later without a GPU
    assert st != 1, L.mam_last_error(None)
    if h.value:
        L.mam_destroy(h)
