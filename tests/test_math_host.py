"""CPU checks of the library's per-element device math (csrc/pd_math.cuh),
compiled as host C++ (tests/cpp/math_host.cpp): the rotation-variant 3x3 SVD
of the local step (Sec. 4.1: U, V in SO(3), only the last singular value may
be negative) against numpy's SVD, and the Neo-Hookean stretch prox
(Sec. 4.1, eq. nh_prox: sigma* minimises k/2 |sigma - sigma_F|^2 + psi(sigma)
with the compressible Neo-Hookean psi) against scipy's bounded minimiser of
that objective, with the special cases the method fixes: no change at rest,
rotation invariance, an inverted element projected to positive stretches.
The prox's filtered stretch Jacobian of the backward pass (Sec. 4.3,
eq. tr_blend, tr_ift) is compared with the oracle's."""
import ctypes
import os
import subprocess

import numpy as np
import pytest
import scipy.optimize as so

from oracle import prox as oprox

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    out = tmp_path_factory.mktemp("mh") / "libmathhost.so"
    src = os.path.join(ROOT, "tests", "cpp", "math_host.cpp")
    shim = os.path.join(ROOT, "tests", "cpp", "host_shim")
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I", shim, "-o", str(out), src], check=True)
    return ctypes.CDLL(str(out))


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def svd(lib, F, dtype):
    F = np.ascontiguousarray(F, dtype=dtype)
    n = F.shape[0]
    U, V = np.zeros((n, 3, 3), dtype), np.zeros((n, 3, 3), dtype)
    s = np.zeros((n, 3), dtype)
    fn = lib.svd3_f32 if dtype == np.float32 else lib.svd3_f64
    fn(ctypes.c_int(n), _p(F), _p(U), _p(s), _p(V))
    return U.astype(np.float64), s.astype(np.float64), V.astype(np.float64)


def prox(lib, sF, mu, lam, k, dtype):
    sF = np.ascontiguousarray(sF, dtype=dtype)
    n = sF.shape[0]
    s = np.zeros((n, 3), dtype)
    it = np.zeros(n, np.int32)
    if dtype == np.float32:
        lib.nh_prox_f32(ctypes.c_int(n), _p(sF), ctypes.c_float(mu), ctypes.c_float(lam), ctypes.c_float(k), _p(s), _p(it))
    else:
        lib.nh_prox_f64(ctypes.c_int(n), _p(sF), ctypes.c_double(mu), ctypes.c_double(lam), ctypes.c_double(k), _p(s), _p(it))
    return s.astype(np.float64), it


def _rotations(rng, n):
    Q, R = np.linalg.qr(rng.standard_normal((n, 3, 3)))
    Q = Q * np.sign(np.diagonal(R, axis1=1, axis2=2))[:, None, :]
    Q[np.linalg.det(Q) < 0, :, 0] *= -1.0
    return Q


def _deformations(rng):
    n = 600
    F = np.eye(3) + 0.4 * rng.standard_normal((n, 3, 3))
    R = _rotations(rng, 200)
    stretch = np.exp(0.3 * rng.standard_normal((200, 3)))
    G = R @ (stretch[:, :, None] * _rotations(rng, 200))          # well separated
    D = R @ (np.array([1.0, 1.0 + 1e-4, 1.0 - 1e-4])[None, :, None] * _rotations(rng, 200))   # near-degenerate
    inv = G.copy()
    inv[:, :, 2] *= -1.0                                            # inverted: det < 0
    return np.concatenate([F, G, D, inv, R, np.eye(3)[None]])


@pytest.mark.parametrize("dtype,tol", [(np.float64, 1e-13), (np.float32, 3e-6)])
def test_svd_against_numpy(lib, dtype, tol):
    F = _deformations(np.random.default_rng(0))
    if dtype == np.float32:
        F = F.astype(np.float32).astype(np.float64)
    U, s, V = svd(lib, F, dtype)
    scale = np.linalg.norm(F, axis=(1, 2))
    rec = U @ (s[:, :, None] * np.transpose(V, (0, 2, 1)))
    assert (np.linalg.norm(rec - F, axis=(1, 2)) / scale).max() <= tol
    I = np.eye(3)
    for Q in (U, V):
        assert np.abs(np.transpose(Q, (0, 2, 1)) @ Q - I).max() <= tol
        assert np.abs(np.linalg.det(Q) - 1.0).max() <= 3 * tol
    ref = np.linalg.svd(F, compute_uv=False)
    assert (np.abs(np.abs(s) - ref).max(axis=1) / scale).max() <= tol
    # ordering: s0 >= s1 >= |s2|; the sign of s2 is the sign of det F
    assert np.all(s[:, 0] >= s[:, 1] - tol * scale) and np.all(s[:, 1] >= np.abs(s[:, 2]) - tol * scale)
    det = np.linalg.det(F)
    clear = np.abs(det) > 1e-3 * scale ** 3
    assert np.array_equal(np.sign(s[clear, 2]), np.sign(det[clear]))


def test_svd_rotation_equivariance(lib):
    """F -> R F leaves sigma unchanged and maps U to R U (away from repeated
    singular values, where U is unique up to the pairwise sign convention)."""
    rng = np.random.default_rng(1)
    R = _rotations(rng, 300)
    F = _rotations(rng, 300) @ (np.exp(0.3 * rng.standard_normal((300, 3)))[:, :, None] * _rotations(rng, 300))
    U, s, V = svd(lib, F, np.float64)
    U2, s2, V2 = svd(lib, R @ F, np.float64)
    assert np.abs(s2 - s).max() <= 1e-13 * np.abs(s).max()
    P1 = U @ np.transpose(V, (0, 2, 1))          # the corotated projection UV^T
    P2 = U2 @ np.transpose(V2, (0, 2, 1))
    assert np.abs(P2 - R @ P1).max() <= 1e-12


def _psi_obj(s, sF, mu, lam, k):
    lnJ = np.log(np.prod(s))
    return 0.5 * k * np.sum((s - sF) ** 2) + 0.5 * mu * (np.sum(s * s) - 3.0) - mu * lnJ + 0.5 * lam * lnJ ** 2


def _psi_grad(s, sF, mu, lam, k):
    lnJ = np.log(np.prod(s))
    return k * (s - sF) + mu * (s - 1.0 / s) + lam * lnJ / s


# Lame parameters of E = 1e5 Pa, nu = 0.45 (the bar's soft/stiff mean is of
# this order) and the Neo-Hookean projective weight k = 2 mu + lam
E, NU = 1e5, 0.45
MU, LAM = E / (2 * (1 + NU)), E * NU / ((1 + NU) * (1 - 2 * NU))
K = 2 * MU + LAM


@pytest.mark.parametrize("dtype,tol", [(np.float64, 2e-8), (np.float32, 2e-6)])
def test_nh_prox_against_scipy_minimiser(lib, dtype, tol):
    """The same minimum as scipy's L-BFGS-B (which stops near 1e-9 relative:
    the FP64 prox is pinned tighter by its first-order condition below). A
    cold-started FP32 prox can end at its iteration cap when its gradient sits
    at the FP32 rounding floor (about 1 call in 200 here; 1 in 200,000 when
    started from the previous local step's sigma*, as the rollouts do); its
    result is then still the minimiser to FP32 accuracy."""
    rng = np.random.default_rng(2)
    sF = np.exp(0.25 * rng.standard_normal((200, 3)))
    sF[:20, 2] *= -0.5                        # inverted elements: sigma_F,3 < 0
    s, it = prox(lib, sF, MU, LAM, K, dtype)
    assert np.all(s > 0)
    if dtype == np.float64:
        assert np.all(it < 40)
    for i in range(sF.shape[0]):
        res = so.minimize(_psi_obj, np.maximum(sF[i], 0.1), args=(sF[i], MU, LAM, K), jac=_psi_grad,
                          method="L-BFGS-B", bounds=[(1e-6, None)] * 3,
                          options={"ftol": 1e-15, "gtol": 1e-12 * K, "maxiter": 10000})
        assert np.abs(s[i] - res.x).max() <= tol * np.abs(res.x).max(), (i, s[i], res.x)
        assert _psi_obj(s[i], sF[i], MU, LAM, K) <= res.fun + 1e-9 * abs(res.fun) + 1e-12 * K
    if dtype == np.float64:
        g = np.array([_psi_grad(s[i], sF[i], MU, LAM, K) for i in range(sF.shape[0])])
        assert np.abs(g).max() <= 1e-11 * K


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_nh_prox_fixed_at_rest(lib, dtype):
    """sigma_F = 1: psi has zero gradient at the rest shape, so the prox
    returns exactly 1 without a Newton step (zero force at rest)."""
    s, it = prox(lib, np.ones((4, 3)), MU, LAM, K, dtype)
    assert np.array_equal(s, np.ones((4, 3))) and np.all(it == 0)


def test_spd_inverse(lib):
    rng = np.random.default_rng(3)
    for _ in range(50):
        A = rng.standard_normal((3, 3))
        H = np.ascontiguousarray(A @ A.T + 0.1 * np.eye(3))
        Hi = np.zeros((3, 3))
        assert lib.spd_inv3_f64(_p(H), _p(Hi)) == 1
        assert np.abs(Hi @ H - np.eye(3)).max() <= 1e-10 * np.linalg.cond(H)
    Hn = np.ascontiguousarray(np.diag([1.0, -1.0, 2.0]))
    assert lib.spd_inv3_f64(_p(Hn), _p(np.zeros((3, 3)))) == 0


def _fjac(lib, ss, mu, lam, k, tau, dtype):
    ss = np.ascontiguousarray(ss, dtype=dtype)
    n = ss.shape[0]
    J = np.zeros((n, 3, 3), dtype)
    if dtype == np.float32:
        lib.filtered_jacobian_f32(ctypes.c_int(n), _p(ss), ctypes.c_float(mu), ctypes.c_float(lam), ctypes.c_float(k),
                                  ctypes.c_float(tau), _p(J))
    else:
        lib.filtered_jacobian_f64(ctypes.c_int(n), _p(ss), ctypes.c_double(mu), ctypes.c_double(lam),
                                  ctypes.c_double(k), ctypes.c_double(tau), _p(J))
    return J.astype(np.float64)


@pytest.mark.parametrize("tau", [0.0, 0.5, 1.0])
@pytest.mark.parametrize("kscale", [1.0, 0.05])
def test_filtered_jacobian_against_oracle(lib, tau, kscale):
    """Definite and indefinite prox Hessians (wide stretches; a small weight
    k makes most of them indefinite), every trust-region blend: the FP64
    build matches the oracle's eigen-decomposition form, clamped directions
    included; the FP32 build matches where the blended Hessian is not close
    to singular."""
    rng = np.random.default_rng(int(10 * tau + 100 * kscale))
    k = K * kscale
    ss = np.exp(0.6 * rng.standard_normal((2000, 3)))
    Jo, _, n_indef = oprox.filtered_sigma_jacobian(ss, MU, LAM, k, tau)
    assert n_indef > 50                      # the filtered branch is exercised
    scale = np.abs(Jo).max(axis=(1, 2))
    J64 = _fjac(lib, ss, MU, LAM, k, tau, np.float64)
    assert (np.abs(J64 - Jo).max(axis=(1, 2)) / scale).max() <= 1e-10
    J32 = _fjac(lib, ss.astype(np.float32).astype(np.float64), MU, LAM, k, tau, np.float32)
    lam_h = np.linalg.eigvalsh(k * np.eye(3) + oprox.nh_hess_sigma(ss, MU, LAM))
    blended = (1.0 - tau) * lam_h + tau * np.abs(lam_h)
    far = np.abs(blended).min(axis=1) > 0.1 * k
    assert (np.abs(J32 - Jo).max(axis=(1, 2))[far] / scale[far]).max() <= 1e-4


@pytest.mark.parametrize("dtype,tol", [(np.float64, 1e-12), (np.float32, 3e-6)])
def test_barrier_prox_against_oracle(lib, dtype, tol):
    """The log-volume barrier's prox (eq. pd_log_volume divided by its weight
    lambda_e: NHMean with mu = r, lam = k = 1 and no deviatoric term) against
    the oracle's, on random, inverted, strongly compressed and strongly
    stretched stretch triples, and its filtered Jacobian at tau = 1/2 and 1."""
    rng = np.random.default_rng(12)
    sF = np.exp(0.3 * rng.standard_normal((300, 3)))
    sF[:30, 2] *= -0.4                           # inverted
    sF[30:45] *= 0.2                             # strongly compressed
    sF[45:60] *= 3.0                             # strongly stretched
    sF = -np.sort(-np.abs(sF), axis=1) * np.where(np.arange(300)[:, None] < 30, [1.0, 1.0, -1.0], 1.0)
    r = (1 - 2 * NU) / (2 * NU)
    ref, _ = oprox.logvol_prox_sigma(sF, r)
    s = np.ascontiguousarray(sF, dtype=dtype)
    out = np.zeros_like(s)
    it = np.zeros(300, np.int32)
    if dtype == np.float32:
        lib.barrier_prox_f32(ctypes.c_int(300), _p(s), ctypes.c_float(r), _p(out), _p(it))
    else:
        lib.barrier_prox_f64(ctypes.c_int(300), _p(s), ctypes.c_double(r), _p(out), _p(it))
    assert np.all(out > 0)
    assert np.abs(out - ref).max() <= tol * np.abs(ref).max()
    for tau in (0.5, 1.0):
        J = np.zeros((300, 9))
        lib.barrier_jacobian_f64(ctypes.c_int(300), _p(np.ascontiguousarray(ref)), ctypes.c_double(r),
                                 ctypes.c_double(tau), _p(J))
        Jo, _, _ = oprox.logvol_sigma_jacobian(ref, r, tau)
        assert np.abs(J.reshape(-1, 3, 3) - Jo).max() <= 1e-9 * np.abs(Jo).max()
