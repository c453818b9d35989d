// L-BFGS for the inverse-problem driver, by reverse communication (host,
// FP64). Nocedal and Wright, Numerical Optimization (2nd ed., 2006): the
// two-loop recursion (Alg. 7.4) with the scaled initial matrix
// H0 = (s^T y / y^T y) I (Sec. 7.2), and a line search for the strong Wolfe
// conditions (Alg. 3.5: bracketing, with the trial step doubled while the
// slope stays negative; Alg. 3.6: zoom, trial steps by the cubic
// interpolation of eq. 3.59 kept 10% inside the bracket, bisection when the
// cubic has no real minimiser or a bracket end has a non-finite value).
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "../../include/pd_b300.h"

namespace {

enum State { kStart = 0, kSearch = 1, kAfterIterate = 2, kDone = 3 };

double dot(const std::vector<double>& a, const std::vector<double>& b) {
  double s = 0.0;
  for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];
  return s;
}

double amax(const std::vector<double>& a) {
  double m = 0.0;
  for (double v : a) m = std::max(m, std::fabs(v));
  return m;
}

bool finite_all(const double* a, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

// minimiser of the cubic through (a, fa, da) and (b, fb, db) (eq. 3.59),
// kept inside [lo + 0.1 w, hi - 0.1 w]; the midpoint when there is none
double cubic_step(double a, double fa, double da, double b, double fb, double db) {
  const double lo = std::min(a, b), hi = std::max(a, b), w = hi - lo;
  double t = 0.5 * (a + b);
  if (std::isfinite(fa) && std::isfinite(fb) && a != b) {
    const double d1 = da + db - 3.0 * (fa - fb) / (a - b);
    const double disc = d1 * d1 - da * db;
    if (disc >= 0.0) {
      const double d2 = (b > a ? 1.0 : -1.0) * std::sqrt(disc);
      const double den = db - da + 2.0 * d2;
      if (den != 0.0) {
        const double c = b - (b - a) * (db + d2 - d1) / den;
        if (std::isfinite(c)) t = c;
      }
    }
  }
  return std::min(std::max(t, lo + 0.1 * w), hi - 0.1 * w);
}

}  // namespace

struct pd_lbfgs {
  int n = 0;
  pd_lbfgs_options o{};
  std::vector<double> x, g, d;          // iterate, its gradient, search direction
  double f = 0.0;
  std::vector<std::vector<double>> S, Y;  // curvature pairs, ring of o.m
  std::vector<double> rho;
  int npairs = 0, head = 0;             // stored pairs, slot of the next pair
  int iters = 0, evals = 0, state = kStart;
  // line search along d from x: phi(a) = f(x + a d)
  double dphi0 = 0.0, a = 0.0;          // slope at 0, current trial step
  bool zoom = false, first = true, steepest = false;
  int ls_evals = 0;
  double a_prev = 0.0, f_prev = 0.0;    // bracketing: the previous trial
  double a_lo = 0.0, f_lo = 0.0, d_lo = 0.0, a_hi = 0.0, f_hi = 0.0, d_hi = 0.0;
};

namespace {

void clear_memory(pd_lbfgs* o) {
  o->npairs = 0;
  o->head = 0;
}

void write_trial(pd_lbfgs* o, double* x) {
  for (int i = 0; i < o->n; ++i) x[i] = o->x[i] + o->a * o->d[i];
}

void write_iterate(const pd_lbfgs* o, double* x) {
  for (int i = 0; i < o->n; ++i) x[i] = o->x[i];
}

// d = -H g by the two-loop recursion (Alg. 7.4); steepest descent with an
// empty memory or when the result is not a descent direction
void direction(pd_lbfgs* o) {
  const int n = o->n, m = o->o.m;
  o->steepest = o->npairs == 0;
  if (!o->steepest) {
    std::vector<double> q = o->g, alpha(o->npairs);
    for (int k = 0; k < o->npairs; ++k) {   // newest to oldest
      const int j = (o->head - 1 - k + m) % m;
      alpha[k] = o->rho[j] * dot(o->S[j], q);
      for (int i = 0; i < n; ++i) q[i] -= alpha[k] * o->Y[j][i];
    }
    const int jn = (o->head - 1 + m) % m;
    const double gamma = dot(o->S[jn], o->Y[jn]) / dot(o->Y[jn], o->Y[jn]);
    for (int i = 0; i < n; ++i) q[i] *= gamma;
    for (int k = o->npairs - 1; k >= 0; --k) {   // oldest to newest
      const int j = (o->head - 1 - k + m) % m;
      const double beta = o->rho[j] * dot(o->Y[j], q);
      for (int i = 0; i < n; ++i) q[i] += o->S[j][i] * (alpha[k] - beta);
    }
    for (int i = 0; i < n; ++i) o->d[i] = -q[i];
    o->dphi0 = dot(o->g, o->d);
    if (!(o->dphi0 < 0.0)) {
      clear_memory(o);
      o->steepest = true;
    }
  }
  if (o->steepest) {
    for (int i = 0; i < n; ++i) o->d[i] = -o->g[i];
    o->dphi0 = dot(o->g, o->d);
  }
}

// a new line search from the current iterate: the first trial step is 1
// (a quasi-Newton step), or step0 / ||g|| along steepest descent
void begin_search(pd_lbfgs* o, double* x) {
  direction(o);
  o->a = o->steepest ? o->o.step0 / std::sqrt(-o->dphi0) : 1.0;
  o->zoom = false;
  o->first = true;
  o->ls_evals = 0;
  o->a_prev = 0.0;
  o->f_prev = o->f;
  o->state = kSearch;
  write_trial(o, x);
}

void enter_zoom(pd_lbfgs* o, double alo, double flo, double dlo, double ahi, double fhi, double dhi) {
  o->zoom = true;
  o->a_lo = alo;
  o->f_lo = flo;
  o->d_lo = dlo;
  o->a_hi = ahi;
  o->f_hi = fhi;
  o->d_hi = dhi;
}

}  // namespace

extern "C" {

void pd_lbfgs_default_options(pd_lbfgs_options* opts) {
  if (!opts) return;
  opts->m = 10;
  opts->max_iters = 100;
  opts->max_evals = 200;
  opts->max_ls = 20;
  opts->gtol = 1e-8;
  opts->ftol = 1e-12;
  opts->c1 = 1e-4;
  opts->c2 = 0.9;
  opts->step0 = 1.0;
}

int pd_lbfgs_create(int32_t n, const pd_lbfgs_options* opts, pd_lbfgs** out) {
  if (!out) return PD_ERR_ARG;
  *out = nullptr;
  pd_lbfgs_options o;
  pd_lbfgs_default_options(&o);
  if (opts) o = *opts;
  if (n < 1 || o.m < 1 || o.max_iters < 1 || o.max_evals < 2 || o.max_ls < 1 || !(o.c1 > 0.0) ||
      !(o.c2 > o.c1) || !(o.c2 < 1.0) || !(o.step0 > 0.0) || !(o.gtol >= 0.0) || !(o.ftol >= 0.0))
    return PD_ERR_ARG;
  pd_lbfgs* p = new (std::nothrow) pd_lbfgs;
  if (!p) return PD_ERR_OOM;
  p->n = n;
  p->o = o;
  p->x.assign(n, 0.0);
  p->g.assign(n, 0.0);
  p->d.assign(n, 0.0);
  p->S.assign(o.m, std::vector<double>(n, 0.0));
  p->Y.assign(o.m, std::vector<double>(n, 0.0));
  p->rho.assign(o.m, 0.0);
  *out = p;
  return PD_OK;
}

int pd_lbfgs_next(pd_lbfgs* o, double* x, double f, const double* g, int32_t* task) {
  if (!o || !x || !task) return PD_ERR_ARG;
  const int n = o->n;
  if (o->state == kDone) return PD_ERR_ARG;
  if (o->state == kStart) {
    if (!g) return PD_ERR_ARG;
    if (!std::isfinite(f) || !finite_all(g, n)) return PD_ERR_NUMERIC;
    o->evals = 1;
    for (int i = 0; i < n; ++i) {
      o->x[i] = x[i];
      o->g[i] = g[i];
    }
    o->f = f;
    if (amax(o->g) <= o->o.gtol) {
      o->state = kDone;
      *task = PD_LBFGS_CONVERGED;
      return PD_OK;
    }
    begin_search(o, x);
    *task = PD_LBFGS_EVAL;
    return PD_OK;
  }
  if (o->state == kAfterIterate) {
    if (o->evals >= o->o.max_evals) {
      o->state = kDone;
      write_iterate(o, x);
      *task = PD_LBFGS_STOP;
      return PD_OK;
    }
    begin_search(o, x);
    *task = PD_LBFGS_EVAL;
    return PD_OK;
  }
  // kSearch: f, g at the trial step a
  if (!g) return PD_ERR_ARG;
  o->evals += 1;
  o->ls_evals += 1;
  const double a = o->a;
  const bool ok = std::isfinite(f) && finite_all(g, n);
  double dphi = 0.0;
  if (ok)
    for (int i = 0; i < n; ++i) dphi += g[i] * o->d[i];
  const double ft = ok ? f : INFINITY;
  const double armijo = o->f + o->o.c1 * a * o->dphi0;
  bool accept = false;
  if (!o->zoom) {
    if (!ok || ft > armijo || (!o->first && ft >= o->f_prev)) {
      enter_zoom(o, o->a_prev, o->f_prev, o->first ? o->dphi0 : o->d_lo, a, ft, dphi);
    } else if (std::fabs(dphi) <= -o->o.c2 * o->dphi0) {
      accept = true;
    } else if (dphi >= 0.0) {
      enter_zoom(o, a, ft, dphi, o->a_prev, o->f_prev, o->first ? o->dphi0 : o->d_lo);
    } else {
      o->a_prev = a;
      o->f_prev = ft;
      o->d_lo = dphi;   // slope at a_prev, kept for a later zoom
      o->first = false;
      o->a = 2.0 * a;
    }
  } else {
    if (!ok || ft > armijo || ft >= o->f_lo) {
      o->a_hi = a;
      o->f_hi = ft;
      o->d_hi = dphi;
    } else if (std::fabs(dphi) <= -o->o.c2 * o->dphi0) {
      accept = true;
    } else {
      if (dphi * (o->a_hi - o->a_lo) >= 0.0) {
        o->a_hi = o->a_lo;
        o->f_hi = o->f_lo;
        o->d_hi = o->d_lo;
      }
      o->a_lo = a;
      o->f_lo = ft;
      o->d_lo = dphi;
    }
  }
  if (accept) {
    const int m = o->o.m, j = o->head;
    double sy = 0.0, yy = 0.0;
    for (int i = 0; i < n; ++i) {
      o->S[j][i] = a * o->d[i];
      o->Y[j][i] = g[i] - o->g[i];
      sy += o->S[j][i] * o->Y[j][i];
      yy += o->Y[j][i] * o->Y[j][i];
    }
    if (sy > 1e-12 * yy) {
      o->rho[j] = 1.0 / sy;
      o->head = (j + 1) % m;
      o->npairs = std::min(o->npairs + 1, m);
    }
    const double f_old = o->f;
    for (int i = 0; i < n; ++i) {
      o->x[i] += a * o->d[i];
      o->g[i] = g[i];
    }
    o->f = f;
    o->iters += 1;
    write_iterate(o, x);
    const bool conv = amax(o->g) <= o->o.gtol ||
                      f_old - f <= o->o.ftol * std::max(std::max(std::fabs(f_old), std::fabs(f)), 1.0);
    if (conv) {
      o->state = kDone;
      *task = PD_LBFGS_CONVERGED;
    } else if (o->iters >= o->o.max_iters || o->evals >= o->o.max_evals) {
      o->state = kDone;
      *task = PD_LBFGS_STOP;
    } else {
      o->state = kAfterIterate;
      *task = PD_LBFGS_ITERATE;
    }
    return PD_OK;
  }
  if (o->evals >= o->o.max_evals) {
    o->state = kDone;
    write_iterate(o, x);
    *task = PD_LBFGS_STOP;
    return PD_OK;
  }
  const bool collapsed = o->zoom && std::fabs(o->a_hi - o->a_lo) <= 1e-14 * std::max(o->a_lo, o->a_hi);
  if (o->ls_evals >= o->o.max_ls || collapsed) {
    // line search failure: restart from steepest descent once, else give up
    if (!o->steepest) {
      clear_memory(o);
      begin_search(o, x);
      *task = PD_LBFGS_EVAL;
      return PD_OK;
    }
    o->state = kDone;
    write_iterate(o, x);
    *task = PD_LBFGS_FAILED;
    return PD_OK;
  }
  if (o->zoom) {
    o->a = (std::isfinite(o->f_lo) && std::isfinite(o->f_hi))
               ? cubic_step(o->a_lo, o->f_lo, o->d_lo, o->a_hi, o->f_hi, o->d_hi)
               : 0.5 * (o->a_lo + o->a_hi);
  }
  write_trial(o, x);
  *task = PD_LBFGS_EVAL;
  return PD_OK;
}

int pd_lbfgs_info(const pd_lbfgs* o, int32_t* iters, int32_t* evals, double* f, double* gmax) {
  if (!o) return PD_ERR_ARG;
  if (iters) *iters = o->iters;
  if (evals) *evals = o->evals;
  if (f) *f = o->f;
  if (gmax) *gmax = amax(o->g);
  return PD_OK;
}

void pd_lbfgs_destroy(pd_lbfgs* o) { delete o; }

}  // extern "C"
