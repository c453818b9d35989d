"""Oracle of the frictional contact step (TEST INFRASTRUCTURE ONLY).

Sec. 4.6 (Signorini-Coulomb complementarity, eq. fb_n, eq. contact_system,
eq. q_update) with the reading the paper leaves open: the factor of A is kept
fixed; contacts are vertex-ground (z >= z_g, normal +z) and vertex-box-bottom
(z <= z_box(t), normal -z) at the position level; friction is Tresca with
disk radius mu * lambda_n from the normal solve of the same iteration
("staggered"), acting on the tangential displacement since q_t.

Because A = L_A (x) I_3 and the normals are +-z, the normal and the
tangential problems of one local-global iteration decouple by axis and share
the scalar Delassus matrix W = (L_A^-1)_CC of the candidate vertices C:

  q_u      = A^-1 b(q)                                    (the plain global step)
  g_c      = n_c (q_u,z[v_c] - z_c)                       (gaps; z_c the obstacle height)
  normal   0 <= lam_n  _|_  D W D lam_n + g >= 0          (D = diag(n_c))
  friction lam_f = argmin 1/2 sum_axes lam^T W lam + lam^T s,  |lam_f,c| <= mu lam_n,c
           s_c = q_u,xy[v_c] - q_t,xy[v_c]
  q        = q_u + A^-1 J^T lam,  J^T lam = (lam_f,c, n_c lam_n,c) at v_c

Bilateral attachments (vertex v held at a prescribed target p(t), Sec. 4.6)
are three equality rows at v with free multipliers: their z row joins the
normal problem (a mixed LCP: no sign constraint, zero residual), their x and
y rows join the friction problem (no disk), with p(t) in place of the
obstacle height and of q_t,xy.

Both subproblems are strictly convex QPs in W (SPD), so their solutions are
unique. The normal LCP is solved exactly by Murty's least-index principal
pivoting method (finite for positive definite matrices); the friction QP by
block projected Gauss-Seidel on the disks; both solutions are checked against
their KKT conditions. A step is the fixed point of the contact-corrected
local-global map (Anderson-mixed Picard iterations, to 1e-13 by default).
"""
from __future__ import annotations

import numpy as np

from . import solver


def delassus(pb: solver.Problem, verts: np.ndarray) -> np.ndarray:
    """W = (L_A^-1)_CC for candidate vertices (all free), one solve per column."""
    pos = np.searchsorted(pb.free, verts)
    assert np.array_equal(pb.free[pos], verts), "contact candidates must be free vertices"
    K = verts.size
    W = np.zeros((K, K))
    for j in range(K):
        e = np.zeros(pb.free.size)
        e[pos[j]] = 1.0
        W[:, j] = pb.lu.solve(e)[pos]
    return 0.5 * (W + W.T)


def lcp_murty(M: np.ndarray, q: np.ndarray, max_iter: int = 100000):
    """w = M z + q >= 0, z >= 0, z^T w = 0 for positive definite M, by Murty's
    least-index principal pivoting: complementary basis given by the set of
    indices with z basic; at each step the least index whose basic variable
    is negative switches side."""
    K = q.size
    basic_z = np.zeros(K, dtype=bool)
    for _ in range(max_iter):
        z = np.zeros(K)
        a = np.nonzero(basic_z)[0]
        if a.size:
            z[a] = np.linalg.solve(M[np.ix_(a, a)], -q[a])
        w = M @ z + q
        w[a] = 0.0
        bad = np.nonzero((basic_z & (z < 0)) | (~basic_z & (w < 0)))[0]
        if bad.size == 0:
            return z
        basic_z[bad[0]] = not basic_z[bad[0]]
    raise RuntimeError("principal pivoting did not terminate")


def mixed_lcp(M: np.ndarray, q: np.ndarray, free: np.ndarray):
    """z with w = M z + q: w_F = 0 on the free rows, and z_N >= 0, w_N >= 0,
    z_N^T w_N = 0 on the others, for positive definite M. The free rows are
    eliminated exactly (their Schur complement is positive definite) and
    the remaining LCP is solved by principal pivoting."""
    F = np.asarray(free, dtype=bool)
    N = ~F
    z = np.zeros(q.size)
    if not F.any():
        return lcp_murty(M, q)
    MFF = M[np.ix_(F, F)]
    if N.any():
        MFN = M[np.ix_(F, N)]
        X = np.linalg.solve(MFF, MFN)
        xq = np.linalg.solve(MFF, q[F])
        z[N] = lcp_murty(M[np.ix_(N, N)] - MFN.T @ X, q[N] - MFN.T @ xq)
        z[F] = -(xq + X @ z[N])
    else:
        z[F] = np.linalg.solve(MFF, -q[F])
    return z


def mixed_lcp_kkt(M, q, z, free) -> float:
    """Largest violation of the mixed LCP's conditions (scaled)."""
    F = np.asarray(free, dtype=bool)
    w = M @ z + q
    s = max(np.abs(q).max(initial=0.0), 1e-300)
    viol = np.abs(w[F]).max(initial=0.0) / s
    if (~F).any():
        viol = max(viol, lcp_kkt(M[np.ix_(~F, ~F)], w[~F] - M[np.ix_(~F, ~F)] @ z[~F], z[~F]))
    return float(viol)


def lcp_kkt(M, q, z) -> float:
    """Largest violation of z >= 0, w >= 0, z_i w_i = 0 (scaled)."""
    w = M @ z + q
    s = max(np.abs(q).max(), 1e-300)
    return float(max(-z.min(initial=0.0) * np.abs(M).max() / s, -w.min(initial=0.0) / s,
                     np.abs(z * w).max(initial=0.0) * np.abs(M).max() / s ** 2))


def tresca_kkt(W, s, rho, lam) -> float:
    """KKT violation of min 1/2 lam^T (W (x) I2) lam + s^T lam over disks
    |lam_c| <= rho_c (rho_c = inf: a free row): with slip u = s + W lam, a
    contact inside its disk has u_c = 0, a contact on its boundary has
    u_c = -t lam_c, t >= 0."""
    u = s + W @ lam
    sc = max(np.abs(s).max(), 1e-300)
    fin = np.isfinite(rho)
    rmax = max(rho[fin].max(initial=0.0), 1e-300)
    viol = 0.0
    for c in range(lam.shape[0]):
        r = np.linalg.norm(lam[c])
        if not fin[c]:            # a free row (attachment): zero residual
            viol = max(viol, np.linalg.norm(u[c]) / sc)
            continue
        viol = max(viol, (r - rho[c]) / rmax)
        if r < rho[c] * (1 - 1e-10) or rho[c] == 0.0:
            if rho[c] > 0:
                viol = max(viol, np.linalg.norm(u[c]) / sc)
        else:
            # u_c must be a non-positive multiple of lam_c
            cross = u[c, 0] * lam[c, 1] - u[c, 1] * lam[c, 0]
            viol = max(viol, abs(cross) / (sc * max(r, 1e-300)), max(0.0, u[c] @ lam[c]) / (sc * max(r, 1e-300)))
    return float(viol)


def tresca(W: np.ndarray, s: np.ndarray, rho: np.ndarray, lam0=None, tol: float = 1e-12):
    """lam [K,2] minimising 1/2 sum_axes lam^T W lam + s^T lam over the disks
    |lam_c| <= rho_c: block projected Gauss-Seidel (from lam0), checked
    against the KKT conditions."""
    lam0 = np.zeros_like(s) if lam0 is None else np.asarray(lam0, dtype=np.float64)
    lam = tresca_pgs(W, s, rho, lam0, tol)
    assert tresca_kkt(W, s, rho, lam) <= 1e-9, "friction QP not solved"
    return lam


def tresca_pgs(W, s, rho, lam0, tol=1e-12, max_sweeps=200000):
    """Block projected Gauss-Seidel on the disks (exact block minimiser, then
    projection onto the disk), from lam0."""
    lam = lam0.copy()
    K = s.shape[0]
    for _ in range(max_sweeps):
        dmax = 0.0
        for c in range(K):
            if rho[c] <= 0:
                lam[c] = 0.0
                continue
            r = s[c] + W[c] @ lam
            new = lam[c] - r / W[c, c]
            nn = np.linalg.norm(new)
            if nn > rho[c]:           # never for a free row (rho = inf)
                new *= rho[c] / nn
            dmax = max(dmax, np.abs(new - lam[c]).max())
            lam[c] = new
        scale = max(rho[np.isfinite(rho)].max(initial=0.0), np.abs(lam).max(), 1e-300)
        if dmax <= 1e-15 * scale and tresca_kkt(W, s, rho, lam) <= tol:
            break
    return lam


class ContactProblem:
    """Candidate set, its Delassus matrix and the obstacle heights of a scene."""

    def __init__(self, pb: solver.Problem, spec):
        self.spec = spec
        att = np.asarray(spec.attach, dtype=np.int64)
        self.verts = np.concatenate([spec.ground, spec.box, att]).astype(np.int64)
        self.normal = np.concatenate([np.ones(spec.ground.size), -np.ones(spec.box.size), np.ones(att.size)])
        # attachment rows: index into the spec's attachment arrays, else -1
        self.att_index = np.concatenate([-np.ones(spec.ground.size + spec.box.size, dtype=np.int64),
                                         np.arange(att.size)])
        order = np.argsort(self.verts, kind="stable")
        self.verts, self.normal, self.att_index = self.verts[order], self.normal[order], self.att_index[order]
        self.is_att = self.att_index >= 0
        self.pos = np.searchsorted(pb.free, self.verts)
        self.W = delassus(pb, self.verts)
        # slip below which a contact counts as sticking: 1e-7 of the rest
        # mesh's bounding-box diagonal
        X = pb.X
        self.slip_tol = 1e-7 * float(np.linalg.norm(X.max(axis=0) - X.min(axis=0)))

    def heights(self, t: int) -> np.ndarray:
        """Per candidate: the obstacle height, or an attachment's target z."""
        h = np.where(self.normal > 0, self.spec.ground_z, self.spec.box_z(t) if self.spec.box.size else 0.0)
        if self.is_att.any():
            h = np.where(self.is_att, self.targets(t)[:, 2], h)
        return h

    def targets(self, t: int) -> np.ndarray:
        """[K,3] attachment targets at the end of step t (zeros on obstacle rows)."""
        out = np.zeros((self.verts.size, 3))
        if self.is_att.any():
            out[self.is_att] = self.spec.attach_target(t)[self.att_index[self.is_att]]
        return out


def correct(pb: solver.Problem, cp: ContactProblem, q_u_free, q_t, t: int, lam_f0=None):
    """Contact-corrected global step: (q_free, lam_n, lam_f) from the plain
    global step q_u (free DoFs); lam_f0 warm-starts the friction solve."""
    D = cp.normal
    g = D * (q_u_free[cp.pos, 2] - cp.heights(t))
    M = (D[:, None] * cp.W) * D[None, :]
    lam_n = mixed_lcp(M, g, cp.is_att)
    assert mixed_lcp_kkt(M, g, lam_n, cp.is_att) <= 1e-9, "normal LCP not solved"
    # tangential reference: q_t,xy for contacts, the target for attachments
    ref = np.where(cp.is_att[:, None], cp.targets(t)[:, :2], q_t[cp.verts, :2])
    slip = q_u_free[cp.pos, :2] - ref
    rho = np.where(cp.is_att, np.inf, cp.spec.mu * lam_n)
    lam_f = tresca(cp.W, slip, rho, lam_f0)
    r = np.zeros((pb.free.size, 3))
    r[cp.pos, 0] = lam_f[:, 0]
    r[cp.pos, 1] = lam_f[:, 1]
    r[cp.pos, 2] = D * lam_n
    return q_u_free + solver.solve_A(pb, r), lam_n, lam_f


def contact_picard(pb, cp, b0, q, q_t, t, lam_f0=None):
    """One contact-corrected local-global iteration q <- T(q)."""
    q_u = solver.solve_A(pb, solver.free_rhs(pb, solver.rhs(pb, b0, q)))
    qf, lam_n, lam_f = correct(pb, cp, q_u, q_t, t, lam_f0)
    return solver.full(pb, qf), lam_n, lam_f


def step(pb, cp, q_t, v_t, f_ext, t, tol=1e-13, max_iter=5000, m=5):
    """One contact step: the fixed point q* = T(q*) of the contact-corrected
    local-global map from q_t, reached by type-II Anderson mixing of T
    (solver.aa_mix; it changes the path, not the fixed point) until
    ||T(q) - q|| <= tol ||q||. Returns (q_{t+1}, lam_n, lam_f, iterations)."""
    b0 = solver.rhs_const(pb, q_t, v_t, f_ext)
    q = q_t.copy()
    hq, hg = [], []
    lam_f = None
    for k in range(1, max_iter + 1):
        qh, lam_n, lam_f = contact_picard(pb, cp, b0, q, q_t, t, lam_f)
        g = qh - q
        if np.linalg.norm(g) <= tol * np.linalg.norm(qh):
            return qh, lam_n, lam_f, k
        hq.append(q)
        hg.append(g)
        if len(hq) > m + 1:
            hq.pop(0)
            hg.pop(0)
        q, reset = solver.aa_mix(hq, hg, qh, g)
        if reset:
            hq, hg = [], []
    raise RuntimeError("contact step did not converge")


def rollout(pb, scene, cp=None):
    cp = cp or ContactProblem(pb, scene.contact)
    q, v = scene.x0.copy(), scene.v0.copy()
    recs = []
    for t in range(scene.steps):
        f = scene.f_ext[t if scene.f_ext.shape[0] > 1 else 0]
        qn, lam_n, lam_f, k = step(pb, cp, q, v, f, t)
        recs.append({"q_t": q, "v_t": v, "q_next": qn, "lam_n": lam_n, "lam_f": lam_f, "iters": k})
        v = (qn - q) / pb.h
        q = qn
    return q, v, recs, cp


# ---------------------------------------------------------------- adjoint

def active_sets(cp: ContactProblem, lam_n, q_next, q_t):
    """Normal-active contacts (lam_n above 1e-9 of the step's total normal
    impulse) and sticking ones among them: those whose tangential slip
    q_xy - q_t,xy over the step is at most cp.slip_tol. At an exact solution
    a contact with friction strictly inside its disk does not slip and a
    sliding one has its friction on the disk boundary, so this is the same
    split as the one by the multipliers; it reads the positions, which an
    iterative inner solver determines far better than the multipliers in
    the ill-conditioned directions of W. Attachments are always in both sets
    and stay out of the impulse total."""
    con = ~cp.is_att
    act = con & (lam_n > 1e-9 * lam_n[con].sum())
    slip = np.linalg.norm(q_next[cp.verts, :2] - q_t[cp.verts, :2], axis=1)
    stick = act & (slip <= cp.slip_tol) & (cp.spec.mu > 0.0)   # no friction: never held
    # attachments: all three rows are equalities at every step
    return act | cp.is_att, stick | cp.is_att


def constraint_rows(pb, cp: ContactProblem, act, stick):
    """G on the free DoFs (rows: z of normal-active candidates with sign n_c,
    then x and y of sticking ones) and the (candidate, axis) of each row."""
    import scipy.sparse as sp
    rows, cols, vals, tags = [], [], [], []
    for c in np.nonzero(act)[0]:
        rows.append(len(tags)); cols.append(3 * cp.pos[c] + 2); vals.append(cp.normal[c]); tags.append((c, 2))
    for c in np.nonzero(stick)[0]:
        for ax in (0, 1):
            rows.append(len(tags)); cols.append(3 * cp.pos[c] + ax); vals.append(1.0); tags.append((c, ax))
    G = sp.csr_matrix((vals, (rows, cols)), shape=(len(tags), 3 * pb.free.size))
    return G, tags


def backward_step(pb, cp: ContactProblem, rec, tau: float, qbar_next, vbar_next):
    """Adjoint of one contact step with the active sets of the converged step
    held fixed (reading): active normal contacts and sticking friction are
    equality constraints G q = h (h: obstacle heights; q_t,xy for sticking
    contacts), a sliding contact's friction force is held at its converged
    value. With R = A q - b(q) - G^T lam_eq - f_slide = 0 and G q = h:
      (A - K) a + G^T nu = q_bar,  G a = 0,
      dL/dtheta = a^T db/dtheta + nu^T dh/dtheta,
    so the routing of the plain step applies with a, and dL/dq_t gains
    J_S^T nu_S from the sticking rows. Direct sparse LU of the KKT matrix."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    from . import adjoint
    h = pb.h
    qbar = qbar_next + vbar_next / h
    q_star, q_t = rec["q_next"], rec["q_t"]
    act, stick = active_sets(cp, rec["lam_n"], rec["q_next"], rec["q_t"])
    G, tags = constraint_rows(pb, cp, act, stick)
    K = adjoint.assemble_K(pb, q_star, tau)
    f3 = (3 * pb.free[:, None] + np.arange(3)[None, :]).ravel()
    M = sp.kron(pb.LA_ff, sp.identity(3), format="csr") - K[f3][:, f3]
    nc = G.shape[0]
    KKT = sp.bmat([[M.T, G.T], [G, None]], format="csc")
    rhs = np.concatenate([qbar[pb.free].ravel(), np.zeros(nc)])
    sol = spla.spsolve(KKT, rhs)
    a = np.zeros_like(q_star)
    a[pb.free] = sol[:3 * pb.free.size].reshape(-1, 3)
    nu = sol[3 * pb.free.size:]
    g = adjoint.route_step(pb, q_t, q_star, tau, a, vbar_next)
    for (c, ax), val in zip(tags, nu):
        if ax < 2 and not cp.is_att[c]:     # an attachment's h is its target, not q_t
            g.dq_t[cp.verts[c], ax] += val
    return g


def rollout_backward(pb, cp: ContactProblem, records, dqT, dvT, taus=None):
    """Walk the contact steps backwards (taus: the trust-region choice per
    step; an exact fixed point gives tau = 1/2, R8)."""
    from . import adjoint
    qbar, vbar = dqT.copy(), dvT.copy()
    n_e = pb.tets.shape[0]
    dw_tot, dw1_tot, db_tot = np.zeros(n_e), np.zeros(n_e), np.zeros(n_e)
    dmu = dlam = dk = dr = 0.0
    dfs = []
    for t in reversed(range(len(records))):
        tau = 0.5 if taus is None else taus[t]
        g = backward_step(pb, cp, records[t], tau, qbar, vbar)
        qbar, vbar = g.dq_t, g.dv_t
        dw_tot += g.dw
        if g.dw1 is not None:
            dw1_tot += g.dw1
        db_tot += g.dbeta
        dmu += g.dmu_bar
        dlam += g.dlam_bar
        dk += g.dk_bar
        dr += g.dr
        dfs.append(g.df_ext)
    dE, dnu = adjoint.chain_material(pb, dw_tot, db_tot, dmu, dlam, dk, dw1=dw1_tot, dr=dr)
    return adjoint.RolloutGrad(qbar, vbar, dE, dnu, np.stack(dfs[::-1]), dw_tot)
