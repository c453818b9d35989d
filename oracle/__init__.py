"""Plain FP64 CPU oracle for the heterogeneous differentiable PD hot path.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call or
execute this package; only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it. It shares no code with the CUDA
library: the two meet only through the seeded inputs in
``paper_2605_14526_b300.inputs``.

Every function restates the paper (arXiv 2605.14526, "DiffPhD") section or
equation it follows, written slowly and in FP64 with numpy/scipy primitives
(``numpy.linalg.svd``/``eigh``, ``scipy.sparse.linalg.splu``). Where the paper
is silent or inconsistent, the reading taken is stated beside the code.

Modules:
  fem      - rest shape, lumped mass, Lame/weights, the global operator A, G and G^T
  prox     - rotation-variant SVD, corotated, Neo-Hookean, corotated + volume and
             corotated + log-volume barrier local steps, their differentials
             and the trust-region filter (Sec. 4.1, 4.3)
  solver   - right-hand side b(q), fixed point of q = A^-1 b(q), Anderson +
             dual gate reference, rollouts (Alg. 1)
  adjoint  - explicit per-element K_e, the adjoint solve and gradient routing
             (Sec. 4.7, Alg. 2)

Parity unpinned: whole-trajectory values at benchmark scale have no external
reference; they are pinned only through the component pins in tests/.
"""
