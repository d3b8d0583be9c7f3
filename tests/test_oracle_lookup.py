"""Pins of the oracle's per-point operator lookup (Sec. III, nearest entry)."""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def _cases():
    out = []
    with open(os.path.join(HERE, "golden", "lookup_cases.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            q, s, nk, e = line.split()
            out.append((float.fromhex(q), float.fromhex(s), int(nk), int(e)))
    return out


def test_golden_lookup_cases(oracle_mod):
    for q, s, nk, e in _cases():
        assert np.float32(q) == q and np.float32(s) == s
        assert int(oracle_mod.lookup_index(q, s, nk)) == e, (q, s, nk, e)


def test_lookup_matches_numpy_fp32(oracle_mod):
    # numpy's float32 multiply and rint (half to even) as an independent implementation
    rng = np.random.default_rng(5)
    q = rng.uniform(0, 2000, 4000).astype(np.float32)
    s = (1.0 / rng.uniform(700, 2300, 4000)).astype(np.float32)
    ref = np.clip(np.rint(q * s), 0, 1023).astype(np.int64)
    assert np.array_equal(oracle_mod.lookup_index(q, s, 1024), ref)


def test_lookup_nan_is_zero(oracle_mod):
    assert int(oracle_mod.lookup_index(5.0, float("nan"), 1024)) == 0


def test_slowness_is_correctly_rounded(oracle_mod):
    v = np.array([750.0, 1000.0, 1234.5, 2250.0, 3.0], dtype=np.float32)
    ref = (1.0 / v.astype(np.float64)).astype(np.float32)   # one rounding from the exact quotient
    assert np.array_equal(oracle_mod.slowness(v), ref)
