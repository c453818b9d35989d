import os
import sys

# The oracle's dense linear algebra runs many small BLAS calls; a threaded
# BLAS pool spins on them and, next to any other busy process, slows them by
# an order of magnitude (the contact oracle's 2-step pad: 38 s with one BLAS
# thread, 866 s with eight). The variables must be set before numpy loads;
# the library's own OpenMP threads (the host factorisation) are not limited.
for _v in ("OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import pytest  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device and the built C-ABI library")
    config.addinivalue_line("markers", "slow: long CPU test")
    try:   # numpy may already be loaded by a plugin: limit its pool directly where possible
        from threadpoolctl import threadpool_limits
        threadpool_limits(limits=1, user_api="blas")
    except ImportError:
        pass
