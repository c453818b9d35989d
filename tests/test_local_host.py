"""CPU parity of the library's local step (csrc/pd_local.cuh, Alg. 1 and
Sec. 4.1: deformation gradient, rotation-variant SVD, corotated or
Neo-Hookean projection, the composite's or the barrier's, and the element's share of the right-hand side
w_e V_e G_e^T vec(p_e), eq. A_basic) compiled as host C++
(tests/cpp/local_host.cpp) and run over whole meshes, against the oracle's
local step and scatter on the same deformed positions."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from oracle import fem, solver
from paper_2605_14526_b300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    out = tmp_path_factory.mktemp("lh") / "liblocalhost.so"
    src = os.path.join(ROOT, "tests", "cpp", "local_host.cpp")
    shim = os.path.join(ROOT, "tests", "cpp", "host_shim")
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I", shim, "-o", str(out), src], check=True)
    return ctypes.CDLL(str(out))


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


MODEL_IDS = {"corotated": 0, "neohookean": 1, "corotated_volume": 2, "corotated_logvol": 3}


def host_rhs(lib, pb, q, fp64):
    """Elastic right-hand side sum_e w_e V_e G_e^T vec(p_e) from the host
    build's per-element corner forces, gathered per vertex in FP64."""
    n_e = pb.tets.shape[0]
    tets = np.ascontiguousarray(pb.tets, dtype=np.int32)
    Bm = np.ascontiguousarray(pb.rest.gradN[:, 1:4, :].reshape(n_e, 9))   # rows: grad N_1..3 = rows of Dm^-1
    coef = np.ascontiguousarray(pb.mat.w * pb.rest.vol)
    x = np.ascontiguousarray(q, dtype=np.float64)
    out = np.zeros((n_e, 12))
    model = MODEL_IDS[pb.model]
    lib.local_step_host(ctypes.c_int(1 if fp64 else 0), ctypes.c_int(model), ctypes.c_int(n_e), _p(tets), _p(Bm),
                        _p(coef), ctypes.c_double(pb.mat.mu_bar), ctypes.c_double(pb.mat.lam_bar),
                        ctypes.c_double(pb.mat.k_bar), ctypes.c_double(float(solver.rotation_share(pb)[0])),
                        ctypes.c_double(float(solver.logvol_ratio(pb)[0])), _p(x), _p(out))
    b = np.zeros_like(x)
    np.add.at(b, tets.ravel(), out.reshape(-1, 3))
    return b


def _scenes():
    return [inputs.tiny_block(model="neohookean", steps=1, cell=0.1, n=3),
            inputs.tiny_block(model="corotated", steps=1, cell=0.1, n=3),
            inputs.hetero_bar(nx=8, ny=4, nz=4, block=4, steps=1),
            inputs.tiny_block(model="corotated_volume", steps=1, cell=0.1, n=3),
            inputs.tiny_block(model="corotated_logvol", steps=1, cell=0.1, n=3)]


@pytest.mark.parametrize("k", range(5))
@pytest.mark.parametrize("amp", [0.05, 0.3])
def test_local_step_matches_oracle(lib, k, amp):
    """A large rotation plus per-vertex noise of amp x the 0.1 m cell; at
    amp = 0.3 some elements are inverted (det F < 0: the SVD's last value is
    negative and the prox returns positive stretches)."""
    sc = _scenes()[k]
    pb = solver.build_problem(sc)
    rng = np.random.default_rng(k)
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1.0]])
    q = sc.X @ R.T + amp * 0.1 * rng.standard_normal(sc.X.shape)
    P, _ = solver.local_step(pb, q)
    ref = fem.scatter_GT(pb.rest, pb.tets, P, pb.mat.w * pb.rest.vol, pb.n_v)
    n_inv = int(np.sum(np.linalg.det(fem.deformation_gradient(pb.rest, pb.tets, q)) <= 0))
    assert (n_inv > 0) == (amp > 0.1)
    scale = np.linalg.norm(ref)
    b64 = host_rhs(lib, pb, q, True)
    assert np.linalg.norm(b64 - ref) <= 1e-12 * scale
    b32 = host_rhs(lib, pb, q, False)
    assert np.linalg.norm(b32 - ref) <= 1e-6 * scale
