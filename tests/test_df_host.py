"""CPU checks of the library's double-float arithmetic (csrc/pd_df.cuh)
compiled as host C++ (tests/cpp/df_host.cpp) and driven in the order of the
inverse-factor products (Sec. 4.5, eq. two_spmv): a segment dot product
spread over 32 lanes x 4 accumulator pairs and a butterfly across the lanes,
against the exact rational sum of the FP64 inputs. The design claims an error
below 2^-44 of the sum of magnitudes and the same result in every lane."""
import ctypes
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    out = tmp_path_factory.mktemp("df") / "libdfhost.so"
    src = os.path.join(ROOT, "tests", "cpp", "df_host.cpp")
    shim = os.path.join(ROOT, "tests", "cpp", "host_shim")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-I", shim, "-o", str(out),
                    src], check=True)
    return ctypes.CDLL(str(out))


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def seg_dot(lib, s, x):
    s = np.ascontiguousarray(s, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros((32, 2), np.float32)
    lib.df_segment_dot(ctypes.c_int(s.size), _p(s), _p(x), _p(out))
    return out


def _values(rng, n, spread):
    return rng.choice([-1.0, 1.0], n) * np.exp(spread * rng.standard_normal(n))


@pytest.mark.parametrize("n", [1, 31, 32, 97, 128, 129, 200, 511, 512, 2000])
@pytest.mark.parametrize("spread", [0.5, 4.0])
def test_segment_dot_within_bound_and_lane_invariant(lib, n, spread):
    rng = np.random.default_rng(n * 7 + int(spread))
    s, x = _values(rng, n, spread), _values(rng, n, spread)
    out = seg_dot(lib, s, x)
    assert np.array_equal(out, np.broadcast_to(out[0], out.shape))   # every lane holds the sum
    hi, lo = float(out[0, 0]), float(out[0, 1])
    exact = sum(Fraction(a) * Fraction(b) for a, b in zip(s, x))
    mag = sum(abs(Fraction(a) * Fraction(b)) for a, b in zip(s, x))
    err = abs(Fraction(hi) + Fraction(lo) - exact)
    assert err <= Fraction(1, 2 ** 44) * mag, float(err / mag)
    assert abs(lo) <= 2.0 ** -24 * abs(hi)                            # renormalised


def test_low_part_is_needed(lib):
    """The bound above is not met by the high part alone (a dropped low part
    or cross term would fail it): plain FP32 accuracy is about 2^-24."""
    rng = np.random.default_rng(5)
    worst = 0.0
    for _ in range(5):
        s, x = _values(rng, 300, 1.0), _values(rng, 300, 1.0)
        out = seg_dot(lib, s, x)
        exact = sum(Fraction(a) * Fraction(b) for a, b in zip(s, x))
        mag = sum(abs(Fraction(a) * Fraction(b)) for a, b in zip(s, x))
        worst = max(worst, float(abs(Fraction(float(out[0, 0])) - exact) / mag))
    assert worst > 2.0 ** -44


def test_cancelling_sum(lib):
    """Terms that cancel to a small total: the error stays below 2^-44 of the
    magnitudes (not of the small result)."""
    rng = np.random.default_rng(6)
    s = _values(rng, 256, 1.0)
    x = np.concatenate([rng.standard_normal(128), np.zeros(128)])
    x[128:] = -x[:128] * s[:128] / s[128:]    # second half cancels the first
    x[0] += 1e-9
    out = seg_dot(lib, s, x)
    exact = sum(Fraction(a) * Fraction(b) for a, b in zip(s, x))
    mag = sum(abs(Fraction(a) * Fraction(b)) for a, b in zip(s, x))
    assert abs(Fraction(float(out[0, 0])) + Fraction(float(out[0, 1])) - exact) <= Fraction(1, 2 ** 44) * mag


def test_split_join_round_trip(lib):
    rng = np.random.default_rng(7)
    x = _values(rng, 4000, 20.0)
    x = x[np.abs(x) < 1e37]
    hl = np.zeros((x.size, 2), np.float32)
    back = np.zeros(x.size)
    lib.df_split_join(ctypes.c_int(x.size), _p(np.ascontiguousarray(x)), _p(hl), _p(back))
    assert np.all(np.abs(back - x) <= 2.0 ** -47 * np.abs(x))
    assert np.all(np.abs(hl[:, 1].astype(np.float64)) <= 2.0 ** -24 * np.abs(hl[:, 0].astype(np.float64)))
