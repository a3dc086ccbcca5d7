"""CPU checks of the tensor-core path's exactness plan (host logic, no GPU).

The external product runs on fp16 tensor cores with fp32 accumulators
(§2.1's RGSW product recast as a dense contraction): it is bit-exact only if
no fp32 partial sum leaves the integers that fp32 holds exactly (|x| <= 2^24,
a 24-bit significand).  fhe_tc_plan_query reports the plan the kernel uses;
these tests check it for every parameter set the library accepts.
"""
import itertools

import numpy as np
import pytest

from paper_2309_09025_gb300 import synth


@pytest.fixture(scope="module")
def fhe():
    from paper_2309_09025_gb300 import build, fhe as F
    build.build()
    return F


def _grid():
    for N, log2_bg, l in itertools.product((256, 512, 1024, 2048), range(1, 16), range(1, 5)):
        if log2_bg * l <= 32:
            yield dict(synth.P630, N=N, log2_bg=log2_bg, l=l)


def test_presets(fhe):
    plans = {n: fhe.tc_plan(synth.PRESETS[n]) for n in ("P64", "T0", "P630", "P750")}
    assert plans["P64"]["available"] == 0  # N = 256
    for n in ("T0", "P630", "P750"):
        assert plans[n]["available"] == 1
    # P630: 7-bit digits, two rows per drain; P750: 10-bit digits split 5 + 5
    assert (plans["P630"]["sub_shift"], plans["P630"]["chunk_rows"]) == (0, 2)
    assert (plans["P750"]["sub_shift"], plans["P750"]["digit_rows"]) == (5, 8)


def test_every_available_plan_is_exact_and_maximal(fhe):
    """For every accepted (N, Bg, l): an available plan keeps every partial
    sum within 2^24, drains after a whole number of chunks that never mixes
    low and high sub-digit rows, and uses the largest such chunk."""
    seen = 0
    for P in _grid():
        plan = fhe.tc_plan(P)
        if not plan["available"]:
            continue
        seen += 1
        R, N = plan["key_rows"], P["N"]
        assert R == (P["k"] + 1) * P["l"]
        assert plan["digit_rows"] == (2 * R if plan["sub_shift"] else R)
        assert plan["max_partial"] == plan["max_digit"] * 128 * plan["chunk_rows"] * N
        assert plan["max_partial"] <= 2 ** 24
        assert plan["chunk_rows"] >= 1 and R % plan["chunk_rows"] == 0
        assert plan["max_digit"] < 512
        bigger = [c for c in range(plan["chunk_rows"] + 1, R + 1) if R % c == 0]
        assert all(plan["max_digit"] * 128 * c * N > 2 ** 24 for c in bigger)
    assert seen >= 20


def test_sub_digit_split_bound():
    """The digit phase's split of a balanced 10-bit digit d in [-512, 512)
    (P750) into a balanced 5-bit low part lo = ((d + 16) & 31) - 16 and
    hi = (d - lo) >> 5, d = lo + 32 hi, keeps both within the plan's
    max_digit = 16 (every d checked)."""
    d = np.arange(-512, 512)
    lo = ((d + 16) & 31) - 16
    hi = (d - lo) >> 5
    assert np.array_equal(lo + 32 * hi, d)
    assert np.abs(lo).max() <= 16 and np.abs(hi).max() <= 16


def test_fp32_accumulation_exact_within_bound_only():
    """Why 2^24: an fp32 running sum of integer products is exact while every
    partial sum stays within 2^24 (P630's worst case, 2048 products of
    64 * 128, lands exactly on 2^24), and loses the integer once a partial
    sum passes it with an odd value."""
    worst = np.full(2048, 64 * 128, np.float32)
    assert float(np.cumsum(worst, dtype=np.float32)[-1]) == 2.0 ** 24
    g = np.random.default_rng(3)
    terms = (g.integers(-64, 65, 2048) * g.integers(-128, 129, 2048)).astype(np.int64)
    acc = np.float32(0)
    for t in terms:
        acc = np.float32(acc + np.float32(t))
    assert int(acc) == int(terms.sum())
    over = np.float32(np.float32(2.0 ** 24) + np.float32(1.0))
    assert float(over) != 2.0 ** 24 + 1


def test_plan_query_rejects_bad_input(fhe):
    import ctypes
    out = fhe.TcPlan()
    assert fhe.lib().fhe_tc_plan_query(None, ctypes.byref(out)) == fhe.FHE_EINVAL
    p = fhe.Params.from_dict(dict(synth.P630, k=2))
    assert fhe.lib().fhe_tc_plan_query(ctypes.byref(p), ctypes.byref(out)) == fhe.FHE_EINVAL
