"""CPU checks of the Anderson small solve (csrc/pd_aa_solve.cuh, Sec. 4.2,
eq. aa_gamma) compiled as host C++ (tests/cpp/aa_host.cpp): the regularised
normal equations (G + reg I) gamma = rhs, reg = max(1e-6 tr(G) / n, 1e-12),
solved by an FP32 Cholesky factor and three passes of refinement with FP64
residuals. Iterative refinement with a factor of unit roundoff u contracts
the error by about cond x u per pass, so after three passes the relative
error is within (cond x 2^-24)^3 of numpy's FP64 solve; the regularisation
caps cond near 1e6 x n, where the solve is only a few digits accurate (the
mixing coefficients then carry a 1e-2 relative error, which changes the
accelerated step but not the fixed point the gate accepts)."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    out = tmp_path_factory.mktemp("aa") / "libaahost.so"
    src = os.path.join(ROOT, "tests", "cpp", "aa_host.cpp")
    shim = os.path.join(ROOT, "tests", "cpp", "host_shim")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-I", shim, "-o", str(out),
                    src], check=True)
    return ctypes.CDLL(str(out))


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def solve(lib, G, rhs, any_form):
    km = lib.aa_max_window()
    nc = G.shape[0]
    Gp = np.zeros((km, km))
    Gp[:nc, :nc] = G
    r = np.zeros(km)
    r[:nc] = rhs
    gam, gn = np.zeros(km), np.zeros(1)
    ok = lib.aa_solve_host(ctypes.c_int(nc), ctypes.c_int(any_form), _p(Gp), _p(r), _p(gam), _p(gn))
    return ok, gam[:nc], gn[0]


@pytest.mark.parametrize("dep", [1.0, 1e-2, 1e-4, 1e-6])
def test_solve_against_numpy(lib, dep):
    rng = np.random.default_rng(int(-np.log10(dep)))
    for nc in range(1, lib.aa_max_window() + 1):
        # difference columns around a common direction: small dep makes them
        # nearly dependent, as late Anderson windows are
        D = rng.standard_normal((3000, 1)) + dep * rng.standard_normal((3000, nc))
        g = rng.standard_normal(3000)
        G, rhs = D.T @ D, D.T @ g
        reg = max(1e-6 * np.trace(G) / nc, 1e-12)
        M = G + reg * np.eye(nc)
        ref = np.linalg.solve(M, rhs)
        bound = max(1e-13, (np.linalg.cond(M) * 2.0 ** -24) ** 3)
        res = [solve(lib, G, rhs, f) for f in ((0, 1) if nc <= 5 else (1,))]
        for ok, gam, gn in res:
            assert ok == 1
            assert np.abs(gam - ref).max() <= bound * np.abs(ref).max(), (nc, dep)
            assert gn == pytest.approx(float(gam @ gam), rel=1e-14)
        if len(res) == 2:   # the unrolled and the run-time forms agree
            assert np.allclose(res[0][1], res[1][1], rtol=1e-12, atol=0)


def test_refused_without_positive_pivot(lib):
    for f in (0, 1):
        ok, _, _ = solve(lib, np.diag([1.0, -0.5]), np.ones(2), f)
        assert ok == 0
        ok, _, _ = solve(lib, np.array([[np.nan]]), np.ones(1), f)
        assert ok == 0
