"""Write oracle-only expected values for the batched workload.

Runs the FP64 oracle (exact fixed point per step, direct adjoint) on the
smallest, the median and the largest instance of the benchmark batch (64
seeded meshes of 1k-40k tets, seed 11, 100 steps, each instance's configured
settings) and stores, per instance, the final state and the gradients of its
loss 0.5 ||x_T - x*||^2 with respect to x0, v0 and E. Calls nothing but
``oracle/`` and the seeded inputs.

  python tests/golden/make_golden_batch.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import adjoint, solver  # noqa: E402
from paper_2605_14526_b300 import inputs  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "batch64_seed11_T100.npz")


def main():
    scenes = inputs.batch_meshes(seed=11)
    order = np.argsort([s.n_e for s in scenes], kind="stable")
    picks = {"smallest": int(order[0]), "median": int(order[len(order) // 2]), "largest": int(order[-1])}
    out = {}
    for name, i in picks.items():
        sc = scenes[i]
        t0 = time.time()
        pb = solver.build_problem(sc)
        qT, vT, recs = solver.rollout(pb, sc, mode="exact")
        _, dq, dv = adjoint.loss_and_grad(sc, pb, qT, vT)
        g = adjoint.rollout_backward(pb, recs, dq, dv)
        out[f"{name}_index"] = np.array([i])
        out[f"{name}_qT"] = qT
        out[f"{name}_dq0"] = g.dx0
        out[f"{name}_dv0"] = g.dv0
        out[f"{name}_dE"] = g.dE
        out[f"{name}_seconds"] = np.array([time.time() - t0])
        print(f"{name}: instance {i}, {sc.n_e} tets, {time.time() - t0:.0f} s", flush=True)
    np.savez_compressed(OUT, **out)
    print(f"wrote {OUT}")


if __name__ == "__main__":
    main()
