"""L-BFGS with a strong-Wolfe line search, FP64, plain Python (test
infrastructure: the reference the library's optimiser is checked against;
nothing in the package imports it).

The paper runs its inverse problems (Sec. 5.4, 5.5: system identification
and initial-state tasks) with an L-BFGS optimiser on the adjoint gradients
and does not restate the method. This follows Nocedal and Wright,
Numerical Optimization, 2nd ed. (2006):

* search direction d = -H g by the two-loop recursion (Alg. 7.4), initial
  matrix H0 = gamma I with gamma = s^T y / y^T y of the newest pair
  (eq. 7.20); a pair is stored only if s^T y > 1e-12 y^T y; memory m;
* line search for the strong Wolfe conditions (eq. 3.7) with c1 = 1e-4,
  c2 = 0.9: bracketing (Alg. 3.5) from a = 1 (from step0 / ||g|| along
  steepest descent), doubling the step while the slope stays negative;
  zoom (Alg. 3.6) with the minimiser of the interpolating cubic (eq. 3.59)
  kept 10% inside the bracket, bisection when it has none or a bracket end
  is not finite;
* an empty memory or a non-descent direction gives steepest descent; a line
  search that fails (20 evaluations, or a collapsed bracket) with curvature
  pairs stored clears them and starts again along steepest descent, and
  fails for good along steepest descent;
* stop at max |g| <= gtol, or a relative decrease of f of at most ftol,
  or max_iters iterations, or max_evals evaluations.
"""
from __future__ import annotations

import math

import numpy as np


def _cubic_min(a, fa, da, b, fb, db):
    """Minimiser of the cubic matching f and f' at a and b (eq. 3.59), within
    [lo + 0.1 w, hi - 0.1 w]; the midpoint where there is none."""
    lo, hi = min(a, b), max(a, b)
    w = hi - lo
    t = 0.5 * (a + b)
    if math.isfinite(fa) and math.isfinite(fb) and a != b:
        d1 = da + db - 3.0 * (fa - fb) / (a - b)
        disc = d1 * d1 - da * db
        if disc >= 0.0:
            d2 = math.copysign(1.0, b - a) * math.sqrt(disc)
            den = db - da + 2.0 * d2
            if den != 0.0:
                c = b - (b - a) * (db + d2 - d1) / den
                if math.isfinite(c):
                    t = c
    return min(max(t, lo + 0.1 * w), hi - 0.1 * w)


def minimize(fun, x0, m=10, max_iters=100, max_evals=200, max_ls=20, gtol=1e-8, ftol=1e-12, c1=1e-4,
             c2=0.9, step0=1.0):
    """fun(x) -> (f, g). Returns a dict: x, f, g, status ('converged',
    'stop', 'failed'), iters, evals, and the lists of every evaluated point
    (`points`) and of the accepted iterates (`iterates`)."""
    x = np.array(x0, dtype=np.float64)
    f, g = fun(x)
    g = np.asarray(g, dtype=np.float64)
    points = [x.copy()]
    iterates = [x.copy()]
    evals, iters = 1, 0
    S, Y = [], []                      # oldest first
    if np.abs(g).max() <= gtol:
        return dict(x=x, f=f, g=g, status="converged", iters=0, evals=1, points=points, iterates=iterates)

    while True:
        # direction (Alg. 7.4)
        steepest = not S
        if not steepest:
            q = g.copy()
            alphas = []
            for s, y in zip(reversed(S), reversed(Y)):
                al = (s @ q) / (s @ y)
                alphas.append(al)
                q = q - al * y
            q = q * ((S[-1] @ Y[-1]) / (Y[-1] @ Y[-1]))
            for (s, y), al in zip(zip(S, Y), reversed(alphas)):
                be = (y @ q) / (s @ y)
                q = q + s * (al - be)
            d = -q
            if not (g @ d < 0.0):
                S, Y = [], []
                steepest = True
        if steepest:
            d = -g
        dphi0 = g @ d
        a = step0 / math.sqrt(-dphi0) if steepest else 1.0

        # line search (Alg. 3.5 / 3.6)
        a_prev, f_prev, d_prev = 0.0, f, dphi0
        zoom = False
        lo = hi = None
        ls = 0
        result = None                  # 'accept' or 'fail'
        while True:
            if evals >= max_evals:
                return dict(x=x, f=f, g=g, status="stop", iters=iters, evals=evals, points=points,
                            iterates=iterates)
            xt = x + a * d
            ft, gt = fun(xt)
            gt = np.asarray(gt, dtype=np.float64)
            points.append(xt.copy())
            evals += 1
            ls += 1
            ok = math.isfinite(ft) and bool(np.all(np.isfinite(gt)))
            dphi = float(gt @ d) if ok else 0.0
            fv = ft if ok else math.inf
            armijo = f + c1 * a * dphi0
            if not zoom:
                if (not ok) or fv > armijo or (ls > 1 and fv >= f_prev):
                    zoom, lo, hi = True, (a_prev, f_prev, d_prev), (a, fv, dphi)
                elif abs(dphi) <= -c2 * dphi0:
                    result = "accept"
                elif dphi >= 0.0:
                    zoom, lo, hi = True, (a, fv, dphi), (a_prev, f_prev, d_prev)
                else:
                    a_prev, f_prev, d_prev = a, fv, dphi
                    a = 2.0 * a
            else:
                if (not ok) or fv > armijo or fv >= lo[1]:
                    hi = (a, fv, dphi)
                elif abs(dphi) <= -c2 * dphi0:
                    result = "accept"
                else:
                    if dphi * (hi[0] - lo[0]) >= 0.0:
                        hi = lo
                    lo = (a, fv, dphi)
            if result == "accept":
                break
            if evals >= max_evals:
                return dict(x=x, f=f, g=g, status="stop", iters=iters, evals=evals, points=points,
                            iterates=iterates)
            collapsed = zoom and abs(hi[0] - lo[0]) <= 1e-14 * max(lo[0], hi[0])
            if ls >= max_ls or collapsed:
                result = "fail"
                break
            if zoom:
                if math.isfinite(lo[1]) and math.isfinite(hi[1]):
                    a = _cubic_min(lo[0], lo[1], lo[2], hi[0], hi[1], hi[2])
                else:
                    a = 0.5 * (lo[0] + hi[0])
        if result == "fail":
            if steepest:
                return dict(x=x, f=f, g=g, status="failed", iters=iters, evals=evals, points=points,
                            iterates=iterates)
            S, Y = [], []
            continue

        s = a * d
        y = gt - g
        if s @ y > 1e-12 * (y @ y):
            S.append(s)
            Y.append(y)
            if len(S) > m:
                S.pop(0)
                Y.pop(0)
        f_old = f
        x, f, g = x + a * d, ft, gt
        iters += 1
        iterates.append(x.copy())
        if np.abs(g).max() <= gtol or f_old - f <= ftol * max(abs(f_old), abs(f), 1.0):
            status = "converged"
        elif iters >= max_iters or evals >= max_evals:
            status = "stop"
        else:
            continue
        return dict(x=x, f=f, g=g, status=status, iters=iters, evals=evals, points=points, iterates=iterates)
