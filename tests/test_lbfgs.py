"""The inverse-problem optimiser (no GPU needed: it is host code of the
library). The oracle's L-BFGS (oracle/lbfgs.py, Nocedal and Wright 2006:
Alg. 7.4 two-loop recursion, Alg. 3.5 / 3.6 strong-Wolfe line search) is
pinned by known minimisers, the strong Wolfe conditions at every accepted
step and an independent implementation (scipy's L-BFGS-B); the library's
pd_lbfgs_* (csrc/lbfgs.cpp, reverse communication) must then evaluate the
same sequence of points as the oracle."""
import math

import numpy as np
import pytest
import scipy.optimize

from oracle import lbfgs as olb
from paper_2605_14526_b300 import binding
from paper_2605_14526_b300.build import build
from paper_2605_14526_b300.inverse import lbfgs


def rosenbrock(x):
    f = 100.0 * (x[1] - x[0] ** 2) ** 2 + (1.0 - x[0]) ** 2
    g = np.array([-400.0 * x[0] * (x[1] - x[0] ** 2) - 2.0 * (1.0 - x[0]), 200.0 * (x[1] - x[0] ** 2)])
    return f, g


def rosenbrock_nd(x):
    f = np.sum(100.0 * (x[1:] - x[:-1] ** 2) ** 2 + (1.0 - x[:-1]) ** 2)
    g = np.zeros_like(x)
    g[:-1] += -400.0 * x[:-1] * (x[1:] - x[:-1] ** 2) - 2.0 * (1.0 - x[:-1])
    g[1:] += 200.0 * (x[1:] - x[:-1] ** 2)
    return f, g


def _quadratic(n=20, seed=0):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, n))
    Q = B @ B.T + n * np.eye(n) * 0.1
    b = rng.standard_normal(n)
    return (lambda x: (0.5 * x @ Q @ x - b @ x, Q @ x - b)), np.linalg.solve(Q, b)


def barrier(x):
    """Smooth inside the unit ball around (2, 0, ...), +inf outside: trial
    steps that leave the domain must be shortened."""
    r2 = np.sum((x - 2.0 * np.eye(x.size)[0]) ** 2)
    if r2 >= 1.0:
        return math.inf, np.full_like(x, math.nan)
    f = np.sum(x ** 2) - np.log(1.0 - r2)
    g = 2.0 * x + 2.0 * (x - 2.0 * np.eye(x.size)[0]) / (1.0 - r2)
    return f, g


# function, start, gtol: each gtol lies above the case's rounding floor, where
# f differences still decide the line search (below it any implementation
# ends in a failed line search, at a point set by rounding)
CASES = {
    "rosenbrock": (rosenbrock, np.array([-1.2, 1.0]), 1e-9),
    "rosenbrock10": (rosenbrock_nd, np.linspace(-1.0, 0.5, 10), 1e-9),
    "quadratic": (_quadratic()[0], np.zeros(20), 1e-6),
    "barrier": (barrier, np.array([2.5, 0.3, -0.2]), 1e-6),
}


def test_oracle_reaches_known_minimisers():
    r = olb.minimize(rosenbrock, [-1.2, 1.0], gtol=1e-10, ftol=0.0, max_iters=500, max_evals=1000)
    assert r["status"] == "converged" and np.allclose(r["x"], 1.0, atol=1e-8)
    fun, xs = _quadratic()
    r = olb.minimize(fun, np.zeros(20), gtol=1e-7, ftol=0.0)
    assert r["status"] == "converged" and np.allclose(r["x"], xs, atol=1e-8)
    r = olb.minimize(rosenbrock_nd, np.linspace(-1.0, 0.5, 10), gtol=1e-10, ftol=0.0, max_iters=1000,
                     max_evals=3000)
    assert np.allclose(r["x"], 1.0, atol=1e-7)


@pytest.mark.parametrize("case", sorted(CASES))
def test_oracle_steps_satisfy_the_strong_wolfe_conditions(case):
    fun, x0, gtol = CASES[case]
    r = olb.minimize(fun, x0, gtol=gtol, ftol=0.0, max_iters=200, max_evals=600)
    assert r["status"] == "converged"
    its = r["iterates"]
    assert len(its) > 3
    for a, b in zip(its[:-1], its[1:]):
        fa, ga = fun(a)
        fb, gb = fun(b)
        s = b - a
        assert fb <= fa + 1e-4 * (ga @ s) + 1e-14 * abs(fa)     # sufficient decrease (eq. 3.7a)
        assert abs(gb @ s) <= 0.9 * abs(ga @ s) * (1 + 1e-12)   # curvature (eq. 3.7b)
        assert ga @ s < 0.0                                      # a descent direction


@pytest.mark.parametrize("case", ["rosenbrock", "rosenbrock10", "quadratic", "barrier"])
def test_oracle_agrees_with_an_independent_lbfgs(case):
    fun, x0, gtol = CASES[case]
    r = olb.minimize(fun, x0, gtol=gtol, ftol=0.0, max_iters=1000, max_evals=3000)
    s = scipy.optimize.minimize(fun, x0, jac=True, method="L-BFGS-B",
                                options={"gtol": gtol, "ftol": 0.0, "maxiter": 5000, "maxfun": 10000})
    assert np.allclose(r["x"], s.x, atol=1e-6)


@pytest.fixture(scope="module")
def built():
    build()


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("m", [3, 10])
def test_library_lbfgs_evaluates_the_oracles_points(built, case, m):
    fun, x0, gtol = CASES[case]
    opts = binding.pd_lbfgs_default_options()
    opts.m, opts.gtol, opts.ftol, opts.max_iters, opts.max_evals = m, gtol, 0.0, 200, 600
    got = lbfgs(fun, x0, opts)
    want = olb.minimize(fun, x0, m=m, gtol=gtol, ftol=0.0, max_iters=200, max_evals=600)
    assert got["status"] == want["status"] == "converged"
    # the same decisions step by step: the first 40 evaluated points agree to
    # rounding (the two-loop dots are summed in another order; on the 10-d
    # Rosenbrock valley that difference grows by about 10x per 5 evaluations
    # and reaches 1e-8 after some 60, so the runs may end a few evaluations
    # apart, at the same minimiser)
    n = min(40, len(got["points"]), len(want["points"]))
    assert n == 40 or len(got["points"]) == len(want["points"])
    for k in range(n):
        assert np.allclose(got["points"][k], want["points"][k], rtol=1e-8, atol=1e-10), k
    assert abs(got["evals"] - want["evals"]) <= 0.05 * want["evals"]
    assert np.allclose(got["x"], want["x"], rtol=1e-6, atol=1e-8)


def test_library_lbfgs_stop_rules_and_errors(built):
    opts = binding.pd_lbfgs_default_options()
    assert opts.m == 10 and opts.max_ls == 20 and abs(opts.c2 - 0.9) < 1e-15
    opts.max_evals = 7
    r = lbfgs(rosenbrock, [-1.2, 1.0], opts)
    assert r["status"] == "stop" and r["evals"] == 7
    w = olb.minimize(rosenbrock, [-1.2, 1.0], max_evals=7)
    assert w["status"] == "stop" and np.allclose(r["x"], w["x"], rtol=1e-12)
    # converged at the start
    r = lbfgs(lambda x: (float(x @ x), 2 * x), np.zeros(3))
    assert r["status"] == "converged" and r["evals"] == 1 and r["iters"] == 0
    bad = binding.pd_lbfgs_default_options()
    bad.c2 = 0.5e-4   # c2 must exceed c1
    with pytest.raises(binding.PDError):
        binding.pd_lbfgs_create(3, bad)
    with pytest.raises(binding.PDError):
        binding.pd_lbfgs_create(0, None)
    o = binding.pd_lbfgs_create(2, None)
    try:
        with pytest.raises(binding.PDError):   # non-finite value at the start
            binding.pd_lbfgs_next(o, np.zeros(2), math.nan, np.zeros(2))
    finally:
        binding.pd_lbfgs_destroy(o)
