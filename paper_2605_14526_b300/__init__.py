"""B300-native differentiable heterogeneous Projective Dynamics hot path.

The compute path lives in the C-ABI library built from ``csrc/``; the Python
modules here only marshal arguments (``binding``) and wrap the rollout as a
``torch.autograd.Function`` (``autograd``). ``inputs`` builds seeded
synthetic workloads.
"""
