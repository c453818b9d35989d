"""CPU checks of the library's host-side factorization (Sec. 4.5): nested
dissection ordering, supernodal Cholesky and the inverse factor S with
A^-1 = S^T S (eq. Ainv_STS, two_spmv), against scipy's sparse solve."""
import ctypes
import os
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import fem, solver
from paper_2605_14526_b300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    out = tmp_path_factory.mktemp("fc") / "libfactorcheck.so"
    src = [os.path.join(ROOT, "tests", "cpp", "factor_check.cpp"),
           os.path.join(ROOT, "paper_2605_14526_b300", "csrc", "factor.cpp"),
           os.path.join(ROOT, "paper_2605_14526_b300", "csrc", "tsolve.cpp")]
    subprocess.run(["g++", "-O2", "-std=c++17", "-fopenmp", "-shared", "-fPIC", "-o", str(out), *src], check=True)
    L = ctypes.CDLL(str(out))
    L.factor_check.restype = ctypes.c_int
    L.tsolve_check.restype = ctypes.c_int
    return L


def _run(lib, A: sp.csr_matrix, xyz, b):
    A = A.tocsr()
    A.sort_indices()
    n = A.shape[0]
    ptr = np.ascontiguousarray(A.indptr, dtype=np.int64)
    idx = np.ascontiguousarray(A.indices, dtype=np.int32)
    val = np.ascontiguousarray(A.data, dtype=np.float64)
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x1 = np.zeros(n)
    x2 = np.zeros(n)
    st = np.zeros(3, dtype=np.int64)
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    rc = lib.factor_check(ctypes.c_int(n), P(ptr), P(idx), P(val), P(xyz), P(b), P(x1), P(x2), P(st))
    return rc, x1, x2, st


@pytest.mark.parametrize("shape", [(6, 3, 3), (12, 4, 4), (5, 5, 5)])
def test_factor_matches_scipy_on_pd_operator(lib, shape):
    sc = inputs.hetero_bar(nx=shape[0], ny=shape[1], nz=shape[2], block=2)
    pb = solver.build_problem(sc)
    A = pb.LA_ff.tocsr()
    xyz = sc.X[pb.free]
    rng = np.random.default_rng(0)
    b = rng.standard_normal(A.shape[0])
    rc, x1, x2, st = _run(lib, A, xyz, b)
    assert rc == 0
    ref = spla.spsolve(A.tocsc(), b)
    assert np.allclose(x1, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())
    assert np.allclose(x2, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())
    # nested dissection keeps the factor sparse: far below dense fill
    n = A.shape[0]
    assert st[0] < 0.5 * n * (n + 1) / 2 or n < 200


def test_factor_handles_disconnected_components(lib):
    # two decoupled blocks: the elimination tree is a forest
    rng = np.random.default_rng(1)
    B = sp.random(20, 20, density=0.2, random_state=1)
    B = B @ B.T + 20 * sp.identity(20)
    A = sp.block_diag([B, B * 2.0]).tocsr()
    xyz = rng.random((40, 3))
    b = rng.standard_normal(40)
    rc, x1, x2, _ = _run(lib, A, xyz, b)
    assert rc == 0
    ref = spla.spsolve(A.tocsc(), b)
    assert np.allclose(x1, ref) and np.allclose(x2, ref)


def test_factor_rejects_indefinite(lib):
    A = sp.csr_matrix(np.array([[1.0, 2.0], [2.0, 1.0]]))
    rc, _, _, _ = _run(lib, A, np.zeros((2, 3)), np.ones(2))
    assert rc == -3


def _tsolve(lib, A, xyz, B, leaf=32):
    A = A.tocsr()
    A.sort_indices()
    n = A.shape[0]
    ptr = np.ascontiguousarray(A.indptr, dtype=np.int64)
    idx = np.ascontiguousarray(A.indices, dtype=np.int32)
    val = np.ascontiguousarray(A.data, dtype=np.float64)
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    X = np.zeros_like(B)
    st = np.zeros(5, dtype=np.int64)
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    rc = lib.tsolve_check(ctypes.c_int(n), P(ptr), P(idx), P(val), P(xyz), ctypes.c_int(leaf), P(B), P(X), P(st))
    return rc, X, st


@pytest.mark.parametrize("shape,leaf", [((6, 3, 3), 8), ((12, 4, 4), 32), ((10, 10, 10), 32), ((32, 8, 8), 32)])
def test_partitioned_inverse_sweeps_match_scipy(lib, shape, leaf):
    """Mode T (level-scheduled partitioned-inverse triangular solves, Sec. 4.5
    eq. Ainv_STS with the factor instead of S) against scipy's sparse solve,
    3 right-hand sides; the node structure is checked by the harness."""
    sc = inputs.hetero_bar(nx=shape[0], ny=shape[1], nz=shape[2], block=2)
    pb = solver.build_problem(sc)
    A = pb.LA_ff.tocsr()
    rng = np.random.default_rng(2)
    B = rng.standard_normal((A.shape[0], 3))
    rc, X, st = _tsolve(lib, A, sc.X[pb.free], B, leaf)
    assert rc == 0, rc
    ref = np.stack([spla.spsolve(A.tocsc(), B[:, i]) for i in range(3)], axis=1)
    assert np.linalg.norm(X - ref) <= 1e-12 * np.linalg.norm(ref), np.linalg.norm(X - ref) / np.linalg.norm(ref)
    # the partitioned inverse stores about as many entries as L itself
    assert st[2] <= 1.6 * st[3], (st[2], st[3])
    assert st[1] >= 2 and st[0] >= st[1]


def test_partitioned_inverse_on_forest_and_tiny(lib):
    # a disconnected operator (two roots) and a 1 x 1 system
    rng = np.random.default_rng(3)
    Bm = sp.random(30, 30, density=0.15, random_state=3)
    Bm = Bm @ Bm.T + 30 * sp.identity(30)
    A = sp.block_diag([Bm, Bm * 3.0]).tocsr()
    B = rng.standard_normal((60, 3))
    rc, X, st = _tsolve(lib, A, rng.random((60, 3)), B, leaf=4)
    assert rc == 0, rc
    ref = np.linalg.solve(A.toarray(), B)
    assert np.allclose(X, ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())
    one = sp.csr_matrix(np.array([[4.0]]))
    rc, X, st = _tsolve(lib, one, np.zeros((1, 3)), np.ones((1, 3)))
    assert rc == 0 and np.allclose(X, 0.25)
