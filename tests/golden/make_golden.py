"""Write oracle-only expected values for the benchmark workload.

Runs the FP64 oracle (exact fixed point per step, direct adjoint) on the
heterogeneous Neo-Hookean bar (32x8x8 cells, 200 steps, seed 2) and stores
the final state, sampled intermediate states (positions and velocities)
and the gradients of the loss
0.5 ||x_T - x*||^2. Calls nothing but ``oracle/`` and the seeded inputs.

  python tests/golden/make_golden.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import adjoint, solver  # noqa: E402
from paper_2605_14526_b300 import inputs  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "bar32x8x8_T200.npz")
SAMPLES = (1, 10, 50, 100, 150)


def main():
    sc = inputs.hetero_bar()
    t0 = time.time()
    pb = solver.build_problem(sc)
    qT, vT, recs = solver.rollout(pb, sc, mode="exact")
    t1 = time.time()
    _, dq, dv = adjoint.loss_and_grad(sc, pb, qT, vT)
    g = adjoint.rollout_backward(pb, recs, dq, dv)
    t2 = time.time()
    np.savez_compressed(OUT, qT=qT, vT=vT, dq0=g.dx0, dv0=g.dv0, dE=g.dE, dnu=np.array([g.dnu]),
                        sample_steps=np.array(SAMPLES), samples=np.stack([recs[s].q_t for s in SAMPLES]),
                        samples_v=np.stack([recs[s].v_t for s in SAMPLES]),
                        seconds=np.array([t1 - t0, t2 - t1]))
    print(f"wrote {OUT}: forward {t1 - t0:.0f} s, backward {t2 - t1:.0f} s")


if __name__ == "__main__":
    main()
