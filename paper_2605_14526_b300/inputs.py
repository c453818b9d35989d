"""Seeded synthetic workloads for the heterogeneous tetrahedral PD solver.

This module only builds INPUTS: rest positions, tetrahedra, Young's moduli,
pins, external forces, time-step settings and loss targets. It holds none of
the method's arithmetic (no masses, no shape-function gradients, no weights,
no projections); the CPU oracle and the CUDA library each derive those from
these arrays on their own.

The paper's scenes (Armadillo, Crab, Bouncing Ball, ...) are not available,
so the workloads below are hex grids split into five tetrahedra per cell, with
the sizes, stiffness contrasts and solver settings of the benchmark
configurations (small homogeneous corotated cube; 100x heterogeneous
Neo-Hookean bar; batched uneven meshes; large heterogeneous block).
Every random choice draws from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field

import numpy as np

COROTATED = "corotated"
COROT_VOLUME = "corotated_volume"   # corotated rotation step + volume step (Sec. 4.1, Sec. 7.2)
COROT_LOGVOL = "corotated_logvol"   # corotated rotation step + log-volume barrier (Sec. 4.1, eq. pd_log_volume)
NEOHOOKEAN = "neohookean"

TR_ADAPT, TR_NONE, TR_CLAMP, TR_ABS = 0, 1, 2, 3


@dataclass
class SolverSettings:
    """Forward/backward iteration settings (Sec. 4.3 dual gate, Alg. 1).

    ``aa_m`` is the Anderson window (number of difference columns, 0 = off);
    ``fixed_iters`` > 0 runs exactly that many local-global iterations and
    ignores the gate; ``local_fp32`` selects the FP32 local step.
    """
    aa_m: int = 5
    fixed_iters: int = 0
    k_max: int = 200
    eps_step: float = 1e-8
    eps_res: float = 1e-6
    eps_abs: float = 1e-12
    eps_tr: float = 0.1
    tr_mode: int = TR_ADAPT
    local_fp32: bool = True
    adj_tol: float = 1e-10
    adj_max_iters: int = 500
    solve_fp64: bool = False     # S products in FP64 instead of double-float
    solve_mode: int = 0          # A^-1 by: 0 auto, 1 products with S, 2 level-scheduled solves with L


@dataclass
class Scene:
    name: str
    X: np.ndarray            # [n_v,3] float64 rest positions (m)
    tets: np.ndarray         # [n_e,4] int32, positively oriented
    pinned: np.ndarray       # [n_v] uint8, 1 = Dirichlet vertex held at X
    E: np.ndarray            # [n_e] float64 Young's modulus (Pa)
    nu: float
    density: float           # kg/m^3
    alpha: float             # Rayleigh mass coefficient (1/s)
    beta0: float             # Rayleigh stiffness coefficient scale
    gravity: np.ndarray      # [3] m/s^2, applied as a body acceleration
    dt: float
    model: str
    steps: int
    f_ext: np.ndarray        # [steps or 1, n_v, 3] float64 extra nodal forces (N)
    x0: np.ndarray           # [n_v,3]
    v0: np.ndarray           # [n_v,3]
    solver: SolverSettings = field(default_factory=SolverSettings)
    loss: str = "l2_target"  # "com_z" or "l2_target"
    target: np.ndarray | None = None
    contact: object = None            # ContactSpec or None
    loss_vertices: np.ndarray | None = None   # vertices of the L2 loss (None = all)

    @property
    def n_v(self) -> int:
        return int(self.X.shape[0])

    @property
    def n_e(self) -> int:
        return int(self.tets.shape[0])

    def with_steps(self, steps: int) -> "Scene":
        f = self.f_ext if self.f_ext.shape[0] == 1 else self.f_ext[:steps]
        return dataclasses.replace(self, steps=steps, f_ext=f)

    def replace(self, **kw) -> "Scene":
        return dataclasses.replace(self, **kw)


# --------------------------------------------------------------------------
# hex grid -> tetrahedra


def _corner_tets(parity: int):
    """Five-tet split of a unit cell; corners indexed by bits (x | y<<1 | z<<2).

    The two parities mirror each other so that face diagonals of neighbouring
    cells agree when the parity alternates with (i + j + k) mod 2.
    """
    if parity == 0:
        return [(0, 1, 2, 4), (3, 1, 2, 7), (5, 1, 4, 7), (6, 2, 4, 7), (1, 2, 4, 7)]
    return [(1, 0, 3, 5), (2, 0, 3, 6), (4, 0, 5, 6), (7, 3, 5, 6), (0, 3, 5, 6)]


def hex_grid(nx: int, ny: int, nz: int, cell: float, cell_mask: np.ndarray | None = None,
             origin=(0.0, 0.0, 0.0)):
    """Vertices and positively oriented tets of an nx*ny*nz cell grid.

    ``cell_mask`` ([nx,ny,nz] bool) keeps a subset of cells; unused vertices
    are dropped. Returns (X, tets, cell_of_tet[ijk]).
    """
    if cell_mask is None:
        cell_mask = np.ones((nx, ny, nz), dtype=bool)

    def vid(i, j, k):
        return i + (nx + 1) * (j + (ny + 1) * k)

    gx, gy, gz = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    X = np.zeros(((nx + 1) * (ny + 1) * (nz + 1), 3))
    ids = vid(gx, gy, gz).ravel()
    X[ids, 0] = origin[0] + gx.ravel() * cell
    X[ids, 1] = origin[1] + gy.ravel() * cell
    X[ids, 2] = origin[2] + gz.ravel() * cell

    tets, cells = [], []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                if not cell_mask[i, j, k]:
                    continue
                c = [vid(i + (b & 1), j + ((b >> 1) & 1), k + ((b >> 2) & 1)) for b in range(8)]
                for t in _corner_tets((i + j + k) & 1):
                    tets.append([c[t[0]], c[t[1]], c[t[2]], c[t[3]]])
                    cells.append((i, j, k))
    tets = np.asarray(tets, dtype=np.int64)
    cells = np.asarray(cells, dtype=np.int64).reshape(-1, 3)

    # orientation: make det[x1-x0, x2-x0, x3-x0] > 0 (swap last two if needed)
    d = np.einsum("ij,ij->i", np.cross(X[tets[:, 1]] - X[tets[:, 0]], X[tets[:, 2]] - X[tets[:, 0]]),
                  X[tets[:, 3]] - X[tets[:, 0]])
    neg = d < 0
    tets[neg, 2], tets[neg, 3] = tets[neg, 3].copy(), tets[neg, 2].copy()

    used = np.zeros(X.shape[0], dtype=bool)
    used[tets.ravel()] = True
    remap = -np.ones(X.shape[0], dtype=np.int64)
    remap[used] = np.arange(int(used.sum()))
    return X[used].copy(), remap[tets].astype(np.int32), cells


def _block_pick(rng, nb: int, n_soft: int):
    soft = np.zeros(nb, dtype=bool)
    soft[rng.choice(nb, size=n_soft, replace=False)] = True
    return soft


# --------------------------------------------------------------------------
# workloads


def small_cube(n: int = 4, cell: float = 0.1, steps: int = 10) -> Scene:
    """Plain PD cube: n^3 cells, homogeneous corotated E=1e5, nu=0.3, z=0 face
    pinned, gravity, dt=0.01 s, 20 fixed local-global iterations, FP64."""
    X, tets, _ = hex_grid(n, n, n, cell)
    pinned = (np.abs(X[:, 2]) < 1e-12).astype(np.uint8)
    n_v, n_e = X.shape[0], tets.shape[0]
    return Scene(
        name=f"cube{n}", X=X, tets=tets, pinned=pinned, E=np.full(n_e, 1e5), nu=0.3,
        density=1000.0, alpha=0.0, beta0=0.0, gravity=np.array([0.0, 0.0, -9.81]), dt=0.01,
        model=COROTATED, steps=steps, f_ext=np.zeros((1, n_v, 3)), x0=X.copy(), v0=np.zeros((n_v, 3)),
        solver=SolverSettings(aa_m=0, fixed_iters=20, local_fp32=False), loss="com_z", target=None)


def twist_velocity(X: np.ndarray, pinned: np.ndarray, omega0: float) -> np.ndarray:
    """Initial velocity of a twist about the bar's long (x) axis through its
    centre line, with angular rate growing linearly from 0 at x=min to omega0
    at x=max; pinned vertices stay at rest."""
    x = X[:, 0]
    L = max(float(x.max() - x.min()), 1e-30)
    c = X.mean(axis=0)
    om = omega0 * (x - x.min()) / L
    v = np.zeros_like(X)
    v[:, 1] = -om * (X[:, 2] - c[2])
    v[:, 2] = om * (X[:, 1] - c[1])
    return v * (1 - pinned[:, None])


def hetero_bar(nx: int = 32, ny: int = 8, nz: int = 8, block: int = 8, cell: float = 0.1,
               steps: int = 200, seed: int = 2, n_soft: int | None = None, omega0: float = 2.0) -> Scene:
    """Heterogeneous Neo-Hookean bar: block^3 cell blocks, half of them soft
    (E=1e4 Pa, seeded choice) and the rest stiff (E=1e6 Pa), nu=0.45, Rayleigh
    alpha=0.01, beta0=1e-3, x=0 face pinned, driven by an initial twist
    (omega0 rad/s at the free end, no gravity: a 1e4 Pa block cannot carry the
    bar's own weight at any cell size where PD meets the gate below),
    dt=0.005 s, Anderson m=5, FP32 local step, dual gate b-change 2e-7 and
    q-step 2e-9 relative (the configured 1e-6 / 1e-8 gate drifts to 4e-5 from
    the exact fixed-point trajectory over 200 steps, for any implementation;
    2e-7 / 2e-9 stays below 1e-5). Loss: 0.5 ||x_T - x*||^2 against a seeded
    target x* = X + N(0, (0.2 cell)^2)."""
    rng = np.random.default_rng(seed)
    X, tets, cells = hex_grid(nx, ny, nz, cell)
    bx, by, bz = max(nx // block, 1), max(ny // block, 1), max(nz // block, 1)
    nb = bx * by * bz
    soft = _block_pick(rng, nb, nb // 2 if n_soft is None else n_soft)
    bid = (np.minimum(cells[:, 0] // block, bx - 1)
           + bx * (np.minimum(cells[:, 1] // block, by - 1) + by * np.minimum(cells[:, 2] // block, bz - 1)))
    E = np.where(soft[bid], 1e4, 1e6)
    pinned = (np.abs(X[:, 0]) < 1e-12).astype(np.uint8)
    n_v = X.shape[0]
    target = X + 0.2 * cell * rng.standard_normal(X.shape)
    return Scene(
        name=f"bar{nx}x{ny}x{nz}", X=X, tets=tets, pinned=pinned, E=E, nu=0.45, density=1000.0,
        alpha=0.01, beta0=1e-3, gravity=np.zeros(3), dt=0.005, model=NEOHOOKEAN,
        steps=steps, f_ext=np.zeros((1, n_v, 3)), x0=X.copy(), v0=twist_velocity(X, pinned, omega0),
        solver=SolverSettings(aa_m=5, fixed_iters=0, k_max=200, eps_step=2e-9, eps_res=2e-7,
                              eps_abs=1e-12, local_fp32=True),
        loss="l2_target", target=target)


def tiny_block(n: int = 2, cell: float = 0.01, model: str = NEOHOOKEAN, seed: int = 7,
               contrast: float = 10.0, steps: int = 2) -> Scene:
    """n^3-cell block with a per-cell random stiffness in [1e5, contrast*1e5],
    one face pinned, a seeded initial velocity and seeded nodal forces (scaled
    with the cell volume); used by finite-difference gradient checks."""
    rng = np.random.default_rng(seed)
    X, tets, cells = hex_grid(n, n, n, cell)
    cidx = cells[:, 0] + n * (cells[:, 1] + n * cells[:, 2])
    Ec = 1e5 * np.exp(np.log(contrast) * rng.random(n ** 3))
    E = Ec[cidx]
    pinned = (np.abs(X[:, 0]) < 1e-12).astype(np.uint8)
    n_v = X.shape[0]
    v0 = 0.05 * rng.standard_normal((n_v, 3)) * (1 - pinned[:, None])
    f_ext = 2e-3 * (cell / 0.01) ** 3 * rng.standard_normal((steps, n_v, 3)) * (1 - pinned[None, :, None])
    target = X + 0.2 * cell * rng.standard_normal(X.shape)
    return Scene(
        name=f"tiny{n}", X=X, tets=tets, pinned=pinned, E=E, nu=0.35, density=1000.0,
        alpha=0.02, beta0=0.05, gravity=np.array([0.0, 0.0, -9.81]), dt=0.005, model=model,
        steps=steps, f_ext=f_ext, x0=X.copy(), v0=v0,
        solver=SolverSettings(aa_m=5, fixed_iters=0, k_max=400, eps_step=1e-13, eps_res=1e-12,
                              eps_abs=1e-15, local_fp32=False),
        loss="l2_target", target=target)


def sysid_bar(nx: int = 8, ny: int = 4, nz: int = 4, block: int = 2, cell: float = 0.1, steps: int = 10,
              seed: int = 21, spread: float = 0.3):
    """System-identification workload on a C2-like bar (Sec. 5.4 task class):
    block^3-cell blocks, each with its own ground-truth log10 E drawn
    uniformly in [4, 6]; the bar's twist, pin, nu and alpha, no stiffness
    damping (beta0 = 0: beta_e scales with mu_e / max mu, a maximum the
    adjoint holds fixed), FP64 local step with a tight gate. Returns
    (scene with the ground-truth moduli, block index per element,
    theta_true = log10 E per block, theta0 = theta_true + N(0, spread^2))."""
    rng = np.random.default_rng(seed)
    sc = hetero_bar(nx=nx, ny=ny, nz=nz, block=block, cell=cell, steps=steps)
    X, tets, cells = hex_grid(nx, ny, nz, cell)
    bx, by, bz = max(nx // block, 1), max(ny // block, 1), max(nz // block, 1)
    bid = (np.minimum(cells[:, 0] // block, bx - 1)
           + bx * (np.minimum(cells[:, 1] // block, by - 1) + by * np.minimum(cells[:, 2] // block, bz - 1)))
    theta_true = rng.uniform(4.0, 6.0, bx * by * bz)
    theta0 = theta_true + spread * rng.standard_normal(theta_true.size)
    sc = sc.replace(name=f"sysid{nx}x{ny}x{nz}", E=np.power(10.0, theta_true)[bid], beta0=0.0,
                    solver=SolverSettings(aa_m=5, k_max=400, eps_step=1e-13, eps_res=1e-11, eps_abs=1e-15,
                                          local_fp32=False))
    return sc, bid.astype(np.int64), theta_true, theta0


def large_block(n: int = 64, cell: float = 0.1, block: int = 8, seed: int = 5, steps: int = 20) -> Scene:
    """Large heterogeneous Neo-Hookean block (n^3 cells, 5 tets each), 8^3-cell
    stiffness blocks (half soft 1e4 Pa / half stiff 1e6 Pa), bottom face
    pinned, no gravity, seeded random top-face nodal loads (N(0, 5 N) per
    axis) re-drawn every 20 steps."""
    rng = np.random.default_rng(seed)
    X, tets, cells = hex_grid(n, n, n, cell)
    nbk = max(n // block, 1)
    nb = nbk ** 3
    soft = _block_pick(rng, nb, nb // 2)
    bid = (np.minimum(cells[:, 0] // block, nbk - 1)
           + nbk * (np.minimum(cells[:, 1] // block, nbk - 1) + nbk * np.minimum(cells[:, 2] // block, nbk - 1)))
    E = np.where(soft[bid], 1e4, 1e6)
    pinned = (np.abs(X[:, 2]) < 1e-12).astype(np.uint8)
    n_v = X.shape[0]
    top = np.abs(X[:, 2] - X[:, 2].max()) < 1e-12
    n_phase = (steps + 19) // 20
    f_ext = np.zeros((steps, n_v, 3))
    for ph in range(n_phase):
        load = np.zeros((n_v, 3))
        load[top] = 5.0 * rng.standard_normal((int(top.sum()), 3))
        f_ext[20 * ph: 20 * (ph + 1)] = load
    return Scene(
        name=f"block{n}", X=X, tets=tets, pinned=pinned, E=E, nu=0.45, density=1000.0,
        alpha=0.01, beta0=1e-3, gravity=np.zeros(3), dt=0.005, model=NEOHOOKEAN,
        steps=steps, f_ext=f_ext, x0=X.copy(), v0=np.zeros((n_v, 3)),
        solver=SolverSettings(aa_m=5, k_max=200, eps_step=1e-8, eps_res=1e-6, eps_abs=1e-12, local_fp32=True),
        loss="l2_target", target=X + 0.02 * rng.standard_normal(X.shape))


def random_rotation(rng) -> np.ndarray:
    """Uniform random rotation (QR of a Gaussian matrix with sign fix)."""
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def _grid_dims(n_cells: float, aspect) -> tuple[int, int, int]:
    a = np.asarray(aspect, dtype=np.float64)
    s = (n_cells / float(np.prod(a))) ** (1.0 / 3.0)
    return tuple(int(max(2, round(s * x))) for x in a)


def swirl_velocity(X: np.ndarray, pinned: np.ndarray, rng, omega: float, v_lat: float) -> np.ndarray:
    """Seeded initial velocity of a mesh fixed at its bottom: a rotation about
    a random axis through the centroid plus a lateral drift, both growing
    linearly with height above the lowest vertex layer; pinned vertices rest."""
    z = X[:, 2] - X[:, 2].min()
    hfrac = z / max(float(z.max()), 1e-30)
    axis = rng.standard_normal(3)
    axis /= np.linalg.norm(axis)
    w = omega * axis
    drift = v_lat * np.append(rng.standard_normal(2), 0.0)
    v = (np.cross(w, X - X.mean(axis=0)) + drift) * hfrac[:, None]
    return v * (1 - pinned[:, None])


def batch_instance(rng, n_tets: int, cell: float = 0.1, steps: int = 100, block: int = 4,
                   name: str = "mesh", shape: str | None = None) -> Scene:
    """One instance of the batched workload: a box or an ellipsoid (cells
    whose centre lies inside it) of about ``n_tets`` tetrahedra, random aspect
    ratios in [1, 2.5], per-instance E in [1e4, 1e6] Pa (log-uniform) times a
    per-block stiffness map log-uniform in [1, 100] over block^3-cell blocks,
    nu uniform in [0.3, 0.49], bottom vertex layer pinned, Neo-Hookean,
    Anderson m=5, FP32 local step and the configured dual gate 1e-6 / 1e-8
    (the tightened 2e-7 / 2e-9 of the bar lies below what an FP32 local step
    resolves on meshes this stiff), k_max 1000 (instances with nu near 0.49
    need several hundred iterations per step), dt 0.005 s, a seeded swirl +
    drift initial velocity, no gravity, and an L2 target
    X + N(0, (0.2 cell)^2)."""
    shape = shape or ("box" if rng.random() < 0.5 else "ellipsoid")
    aspect = 1.0 + 1.5 * rng.random(3)
    if shape == "box":
        nx, ny, nz = _grid_dims(n_tets / 5.0, aspect)
        mask = None
    else:
        nx, ny, nz = _grid_dims(n_tets / 5.0 / (np.pi / 6.0), aspect)
        ci = (np.arange(nx) + 0.5) / nx - 0.5
        cj = (np.arange(ny) + 0.5) / ny - 0.5
        ck = (np.arange(nz) + 0.5) / nz - 0.5
        mask = (ci[:, None, None] ** 2 + cj[None, :, None] ** 2 + ck[None, None, :] ** 2) <= 0.25
    X, tets, cells = hex_grid(nx, ny, nz, cell, mask)
    E_inst = 10.0 ** rng.uniform(4.0, 6.0)
    bx, by, bz = (nx + block - 1) // block, (ny + block - 1) // block, (nz + block - 1) // block
    smap = 10.0 ** rng.uniform(0.0, 2.0, size=bx * by * bz)
    bid = cells[:, 0] // block + bx * (cells[:, 1] // block + by * (cells[:, 2] // block))
    E = E_inst * smap[bid]
    nu = float(rng.uniform(0.3, 0.49))
    pinned = (np.abs(X[:, 2] - X[:, 2].min()) < 1e-9 * cell).astype(np.uint8)
    n_v = X.shape[0]
    v0 = swirl_velocity(X, pinned, rng, omega=float(rng.uniform(0.5, 2.0)), v_lat=float(rng.uniform(0.0, 0.3)))
    target = X + 0.2 * cell * rng.standard_normal(X.shape)
    return Scene(
        name=f"{name}-{shape}{nx}x{ny}x{nz}", X=X, tets=tets, pinned=pinned, E=E, nu=nu, density=1000.0,
        alpha=0.01, beta0=1e-3, gravity=np.zeros(3), dt=0.005, model=NEOHOOKEAN,
        steps=steps, f_ext=np.zeros((1, n_v, 3)), x0=X.copy(), v0=v0,
        solver=SolverSettings(aa_m=5, fixed_iters=0, k_max=1000, eps_step=1e-8, eps_res=1e-6,
                              eps_abs=1e-12, local_fp32=True),
        loss="l2_target", target=target)


def batch_meshes(n: int = 64, tets_lo: int = 1000, tets_hi: int = 40000, steps: int = 100,
                 seed: int = 11) -> list[Scene]:
    """The batched workload: ``n`` independent instances whose tet counts are
    drawn log-uniformly in [tets_lo, tets_hi] (each built by batch_instance)."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(tets_lo), np.log(tets_hi), size=n))
    return [batch_instance(rng, int(s), steps=steps, name=f"m{i}") for i, s in enumerate(sizes)]


def mlp_init(seed: int = 0, hidden: int = 128) -> np.ndarray:
    """Initial parameters of the warm-start network (7 -> H -> H -> H -> 3):
    weights uniform in +-sqrt(6 / fan_in) (He et al. 2015, uniform form),
    biases zero; flat FP32 vector in the library's layout W1, b1, W2, b2, W3,
    b3, W4, b4."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, fan_out in ((7, hidden), (hidden, hidden), (hidden, hidden), (hidden, 3)):
        lim = np.sqrt(6.0 / fan_in)
        parts.append(rng.uniform(-lim, lim, size=fan_out * fan_in))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)


@dataclass
class ContactSpec:
    """Frictional contacts of a workload (reading of Sec. 4.6): vertex-ground
    (z >= ground_z, normal +z) for ``ground`` vertices and vertex-box-bottom
    (z <= box_z(t), normal -z) for ``box`` vertices; the rigid box moves down
    by ``box_travel`` over the first ``box_steps`` steps and is then held.
    Coulomb coefficient ``mu`` (Tresca disks of radius mu * lambda_n).
    Bilateral attachments (Sec. 4.6): vertex ``attach[i]`` is held at
    ``attach_target(t)[i]``, which moves from ``attach_p0[i]`` by
    ``attach_travel[i]`` over the first ``attach_steps`` steps."""
    ground: np.ndarray          # [Kg] vertex indices
    box: np.ndarray             # [Kb] vertex indices
    ground_z: float
    box_z0: float
    box_travel: float
    box_steps: int
    mu: float
    attach: np.ndarray = field(default_factory=lambda: np.zeros(0, dtype=np.int64))   # [Ka]
    attach_p0: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))          # [Ka,3]
    attach_travel: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))      # [Ka,3]
    attach_steps: int = 1

    def box_z(self, t: int) -> float:
        """Height of the box bottom at the end of step t (0-based)."""
        return self.box_z0 - self.box_travel * min(t + 1, self.box_steps) / self.box_steps

    def attach_target(self, t: int) -> np.ndarray:
        """[Ka,3] attachment targets at the end of step t (0-based)."""
        n = int(self.attach_steps)
        if n < 1:   # as pd_set_contacts: the targets move over at least one step
            raise ValueError("attach_steps must be >= 1")
        k = min(t + 1, n) / n
        return np.asarray(self.attach_p0, dtype=np.float64) + k * np.asarray(self.attach_travel, dtype=np.float64)


def contact_pad(nx: int = 48, ny: int = 48, nz: int = 12, cell: float = 0.01, footprint: int = 16,
                steps: int = 300, box_steps: int = 150, travel: float = 0.02, seed: int = 13,
                E_shell: float = 1e5, E_core: float = 1e7) -> Scene:
    """Contact-rich soft pad: nx*ny*nz cells of `cell` m with interior vertices
    jittered by up to 15% of a cell (seeded), a stiff core (E 1e7 Pa, cells at
    least 2 cells from the outer surface) in a soft shell (1e5 Pa), nu = 0.45,
    Neo-Hookean, resting on the ground z = 0 under gravity and pressed by a
    rigid box whose footprint x footprint cells centred on the top face moves
    down `travel` m over `box_steps` steps and is then held; Coulomb mu = 0.5;
    no pins; dt = 0.002 s; Anderson m = 5, FP32 local step, gate 1e-6 / 1e-8.
    Loss: L2 of the top-surface positions at T against X + N(0, (0.1 cell)^2).
    E_shell / E_core override the moduli (smaller parity cases)."""
    rng = np.random.default_rng(seed)
    X, tets, cells = hex_grid(nx, ny, nz, cell)
    n = np.array([nx, ny, nz])
    ijk = np.rint(X / cell).astype(np.int64)
    interior = np.all((ijk > 0) & (ijk < n[None, :]), axis=1)
    X = X.copy()
    X[interior] += cell * rng.uniform(-0.15, 0.15, size=(int(interior.sum()), 3))
    c = cells
    depth = np.minimum.reduce([c[:, 0], nx - 1 - c[:, 0], c[:, 1], ny - 1 - c[:, 1], c[:, 2], nz - 1 - c[:, 2]])
    E = np.where(depth >= 2, E_core, E_shell)
    n_v = X.shape[0]
    ground = np.nonzero(ijk[:, 2] == 0)[0]
    lo = (nx - footprint) // 2
    lo_y = (ny - footprint) // 2
    top = (ijk[:, 2] == nz) & (ijk[:, 0] >= lo) & (ijk[:, 0] <= lo + footprint) & \
        (ijk[:, 1] >= lo_y) & (ijk[:, 1] <= lo_y + footprint)
    box = np.nonzero(top)[0]
    top_all = np.nonzero(ijk[:, 2] == nz)[0]
    target = X + 0.1 * cell * rng.standard_normal(X.shape)
    sc = Scene(
        name=f"pad{nx}x{ny}x{nz}", X=X, tets=tets, pinned=np.zeros(n_v, dtype=np.uint8), E=E, nu=0.45,
        density=1000.0, alpha=0.01, beta0=1e-3, gravity=np.array([0.0, 0.0, -9.81]), dt=0.002,
        model=NEOHOOKEAN, steps=steps, f_ext=np.zeros((1, n_v, 3)), x0=X.copy(), v0=np.zeros((n_v, 3)),
        solver=SolverSettings(aa_m=5, fixed_iters=0, k_max=400, eps_step=1e-8, eps_res=1e-6, eps_abs=1e-12,
                              local_fp32=True),
        loss="l2_target", target=target)
    sc.contact = ContactSpec(ground=ground, box=box, ground_z=0.0, box_z0=nz * cell, box_travel=travel,
                             box_steps=box_steps, mu=0.5)
    sc.loss_vertices = top_all
    return sc
