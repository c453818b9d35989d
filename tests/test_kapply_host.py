"""CPU parity of the adjoint's matrix-free K p (csrc/pd_bwd_elem.cuh: the
per-element differential record at q* and its product, Sec. 4.3 eq. tr_blend,
tr_ift and the spectral differential of p = U diag(sigma*) V^T; K = db/dq,
eq. db_dq) compiled as host C++ (tests/cpp/kapply_host.cpp), against the
oracle's explicitly assembled K for every trust-region blend, with large
rotations and inverted elements. At a converged prox minimiser the Hessian
k I + H_psi is positive semidefinite, so the blend leaves these K unchanged;
its indefinite branch is covered by the filtered-Jacobian test of
tests/test_math_host.py."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from oracle import adjoint, solver
from paper_2605_14526_b300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    out = tmp_path_factory.mktemp("kh") / "libkapplyhost.so"
    src = os.path.join(ROOT, "tests", "cpp", "kapply_host.cpp")
    shim = os.path.join(ROOT, "tests", "cpp", "host_shim")
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I", shim, "-o", str(out), src], check=True)
    return ctypes.CDLL(str(out))


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def host_kp(lib, pb, q, tau, p, fp64):
    n_e = pb.tets.shape[0]
    tets = np.ascontiguousarray(pb.tets, dtype=np.int32)
    Bm = np.ascontiguousarray(pb.rest.gradN[:, 1:4, :].reshape(n_e, 9))
    coef = np.ascontiguousarray(pb.mat.w * pb.rest.vol)
    out = np.zeros((n_e, 12))
    model = {"corotated": 0, "neohookean": 1, "corotated_volume": 2, "corotated_logvol": 3}[pb.model]
    lib.kapply_host(ctypes.c_int(1 if fp64 else 0), ctypes.c_int(model), ctypes.c_int(n_e), _p(tets), _p(Bm),
                    _p(coef), ctypes.c_double(pb.mat.mu_bar), ctypes.c_double(pb.mat.lam_bar),
                    ctypes.c_double(pb.mat.k_bar), ctypes.c_double(float(solver.rotation_share(pb)[0])),
                    ctypes.c_double(float(solver.logvol_ratio(pb)[0])), _p(np.ascontiguousarray(q)),
                    ctypes.c_double(tau), _p(np.ascontiguousarray(p)), _p(out))
    kp = np.zeros_like(q)
    np.add.at(kp, tets.ravel(), out.reshape(-1, 3))
    return kp


CASES = [("neohookean", 1.0, 0.05), ("neohookean", 1.0, 0.3), ("corotated", 1.0, 0.3), ("bar", 1.0, 0.3),
         ("neohookean", 1.6, 0.05), ("corotated_volume", 1.0, 0.05), ("corotated_volume", 1.0, 0.3),
         ("corotated_volume", 1.6, 0.05), ("corotated_logvol", 1.0, 0.05), ("corotated_logvol", 1.0, 0.3),
         ("corotated_logvol", 1.6, 0.05)]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_kapply_matches_oracle(lib, case):
    model, stretch, amp = CASES[case]
    if model == "bar":
        sc = inputs.hetero_bar(nx=8, ny=4, nz=4, block=4, steps=1)
    else:
        sc = inputs.tiny_block(model=model, steps=1, cell=0.1, n=3)
    pb = solver.build_problem(sc)
    rng = np.random.default_rng(case)
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1.0]])
    q = stretch * sc.X @ R.T + amp * 0.1 * rng.standard_normal(sc.X.shape)
    p = rng.standard_normal(sc.X.shape)
    for tau in (0.0, 0.5, 1.0):
        ref = (adjoint.assemble_K(pb, q, tau) @ p.ravel()).reshape(-1, 3)
        scale = np.linalg.norm(ref)
        assert np.linalg.norm(host_kp(lib, pb, q, tau, p, True) - ref) <= 1e-12 * scale
        assert np.linalg.norm(host_kp(lib, pb, q, tau, p, False) - ref) <= 1e-6 * scale
