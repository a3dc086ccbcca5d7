"""Pins of the oracle's primitives (CPU only).

Each test checks the oracle against something other than itself: published
SplitMix64 vectors, numpy polynomial products, exhaustive recomposition of the
gadget digits, exact rational rounding, closed-form noise moments.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2309_09025_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
MASK32 = (1 << 32) - 1


def _parse_int(tok):
    return int(tok, 16) if tok.startswith("0x") else int(tok)


def test_splitmix64_published_vectors():
    """Counter-based generator = SplitMix64's published outputs."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 2
    for row in rows:
        state = _parse_int(row[0])
        expected = [_parse_int(t) for t in row[1:]]
        got = [O.splitmix_out(state, i) for i in range(3)]
        assert got == expected


def test_draw_is_stream_of_streams():
    # draw(seed, domain, i) is output i of the generator seeded by output
    # `domain` of the generator seeded by `seed`; distinct domains differ.
    s = O.splitmix_out(77, 3)
    assert O.draw(77, 3, 5) == O.splitmix_out(s, 5)
    assert O.draw(77, 2, 5) != O.draw(77, 3, 5)


@pytest.mark.parametrize("noise_log2", [20, 25, 30])
def test_noise_moments(noise_log2):
    """Irwin-Hall(12) sampler: mean ~0, variance ~ 2^(64-2x) + 1/12 (closed form
    of a sum of 12 uniform 32-bit signed integers scaled by 2^-x and rounded)."""
    vals = np.array([O.noise(11, 3, i, noise_log2) for i in range(20000)], np.uint32)
    e = vals.astype(np.int64)
    e = np.where(e >= 2 ** 31, e - 2 ** 32, e).astype(np.float64)
    var_expected = 2.0 ** (64 - 2 * noise_log2) + 1.0 / 12.0
    std = np.sqrt(var_expected)
    assert abs(e.mean()) < 5 * std / np.sqrt(len(e)) + 0.5
    ratio = e.var() / var_expected
    assert 0.95 < ratio < 1.05
    # Irwin-Hall(12) support: |e| <= 6 * 2^(32 - x) (+1 for rounding)
    assert np.abs(e).max() <= 6 * 2.0 ** (32 - noise_log2) + 1


def test_noise_disabled():
    assert all(O.noise(5, 1, i, 64) == 0 for i in range(100))


def _numpy_negacyclic(a, b):
    """Reference: full product with numpy.convolve, then fold X^N = -1."""
    N = len(a)
    full = np.convolve(np.asarray(a, dtype=object), np.asarray(b, dtype=object))
    full = np.concatenate([full, np.zeros(2 * N - len(full), dtype=object)])
    res = full[:N] - full[N:]
    return np.array([int(x) & MASK32 for x in res], np.uint32)


@pytest.mark.parametrize("N", [4, 16, 256])
def test_negacyclic_mul_vs_numpy(N):
    g = np.random.default_rng(N)
    for _ in range(3):
        a = g.integers(0, 2 ** 32, N, dtype=np.uint64).astype(np.uint32)
        b = g.integers(0, 2 ** 32, N, dtype=np.uint64).astype(np.uint32)
        assert np.array_equal(O.negacyclic_mul(a, b), _numpy_negacyclic(a, b))


def test_negacyclic_hand_example():
    # (1 + 2X)(3 + X^3) = 3 + 6X + X^3 + 2X^4 = 1 + 6X + X^3  mod X^4 + 1
    out = O.negacyclic_mul(np.array([1, 2, 0, 0]), np.array([3, 0, 0, 1]))
    assert out.tolist() == [1, 6, 0, 1]


def test_monomials_and_rotation():
    N = 16
    g = np.random.default_rng(1)
    P = g.integers(0, 2 ** 32, N, dtype=np.uint64).astype(np.uint32)
    for e in [0, 1, 5, N - 1, N, N + 3, 2 * N - 1]:
        mono = np.zeros(N, np.uint32)
        if e < N:
            mono[e] = 1
        else:
            mono[e - N] = MASK32  # X^e = -X^(e-N)
        assert np.array_equal(O.poly_rotate(P, e), _numpy_negacyclic(mono, P))
    # X^N = -1 and X^a X^b = X^(a+b)
    assert np.array_equal(O.poly_rotate(P, N), (-P.astype(np.int64)) & MASK32)
    assert np.array_equal(O.poly_rotate(O.poly_rotate(P, 7), 12), O.poly_rotate(P, 19))


def _round_top(x, bits):
    """x rounded (half up) to a multiple of 2^(32-bits), mod 2^32."""
    if bits >= 32:
        return x
    unit = 1 << (32 - bits)
    return ((x + unit // 2) // unit * unit) & MASK32


@pytest.mark.parametrize("log2_base,levels", [(4, 4), (8, 2), (2, 7)])
def test_decompose_exhaustive_top_bits(log2_base, levels):
    """Every value of the kept top bits (random low bits): digits in
    [-B/2, B/2) and sum_lam d_lam 2^(32 - lam*log2 B) = round(x) mod 2^32."""
    bits = log2_base * levels
    g = np.random.default_rng(bits)
    B = 1 << log2_base
    for top in range(1 << bits):
        low = int(g.integers(0, 1 << (32 - bits))) if bits < 32 else 0
        x = ((top << (32 - bits)) | low) & MASK32
        d = O.decompose(x, log2_base, levels)
        assert d.min() >= -B // 2 and d.max() < B // 2
        rec = sum(int(d[lam]) << (32 - log2_base * (lam + 1)) for lam in range(levels)) & MASK32
        assert rec == _round_top(x, bits)


@pytest.mark.parametrize("P", [synth.P630, synth.P750])
def test_decompose_random_params(P):
    g = np.random.default_rng(3)
    for bits_, lv in [(P["log2_bg"], P["l"]), (P["log2_bks"], P["l_ks"])]:
        for x in g.integers(0, 2 ** 32, 3000, dtype=np.uint64):
            d = O.decompose(int(x), bits_, lv)
            rec = sum(int(d[i]) << (32 - bits_ * (i + 1)) for i in range(lv)) & MASK32
            assert rec == _round_top(int(x), bits_ * lv)
            assert d.min() >= -(1 << bits_) // 2 and d.max() < (1 << bits_) // 2


@pytest.mark.parametrize("N", [256, 1024, 2048])
def test_mod_switch_is_rounded_rational(N):
    # round(a * 2N / q) mod 2N with ties up, by exact integer rational rounding
    g = np.random.default_rng(N)
    vals = list(g.integers(0, 2 ** 32, 5000, dtype=np.uint64)) + [0, 1, 2 ** 32 - 1]
    unit = 2 ** 32 // (2 * N)
    vals += [unit // 2 - 1, unit // 2, unit // 2 + 1, 2 ** 32 - unit // 2, 2 ** 32 - unit // 2 - 1]
    for a in vals:
        a = int(a)
        expected = ((2 * a * 2 * N + 2 ** 32) // (2 * 2 ** 32)) % (2 * N)
        assert O.mod_switch(a, N) == expected


def test_lwe_encrypt_decrypt_roundtrip(oracle_keys):
    for name in ["P64", "P630", "T0"]:
        P, K = oracle_keys(name, 5)
        p = 1 << P["log2_p"]
        m = np.arange(-p, p, dtype=np.int32)
        for seed in (1, 2, 3):
            ct = O.encrypt(P, K, m, seed)
            assert np.array_equal(O.decrypt(P, K, ct), m)
            # phase = Delta*m + e with |e| bounded by the sampler's support
            ph = O.phase(P, K, ct).astype(np.int64)
            err = ((ph - m.astype(np.int64) * O.delta(P) + 2 ** 31) % 2 ** 32) - 2 ** 31
            assert np.abs(err).max() <= 6 * 2 ** (32 - P["lwe_noise_log2"]) + 1


def test_lwe_linearity(oracle_keys):
    """Eq. (noise grows), 4.1: sum w LWE(x) = LWE(sum w x).  The phase is
    linear exactly (mod q), checked with numpy's integer matmul."""
    P, K = oracle_keys("P64", 5)
    p = 1 << P["log2_p"]
    g = np.random.default_rng(9)
    x = g.integers(-2, 3, 40).astype(np.int32)
    W = g.integers(-4, 5, (12, 40)).astype(np.int32)
    bias = g.integers(-3, 4, 12).astype(np.int32)
    ct = O.encrypt(P, K, x, 13)
    out = O.lwe_linear(P, W, ct, bias)
    ph_in = O.phase(P, K, ct).astype(np.int64)
    ph_out = O.phase(P, K, out).astype(np.int64)
    exp_phase = (W.astype(np.int64) @ ph_in + bias.astype(np.int64) * O.delta(P)) % 2 ** 32
    assert np.array_equal(ph_out, exp_phase)
    exp_msg = ((W.astype(np.int64) @ x + bias + p) % (2 * p)) - p
    assert np.array_equal(O.decrypt(P, K, out), exp_msg)


def test_lwe_conv2d_vs_scipy(oracle_keys):
    from scipy.signal import correlate2d
    P, K = oracle_keys("P64", 5)
    p = 1 << P["log2_p"]
    g = np.random.default_rng(4)
    cin, h, w, cout, kh, stride, pad = 2, 9, 8, 3, 3, 2, 1
    img = g.integers(0, 3, (cin, h, w)).astype(np.int32)
    W = g.integers(-2, 3, (cout, cin, kh, kh)).astype(np.int32)
    ct = O.encrypt(P, K, img.reshape(-1), 21)
    out = O.lwe_conv2d(P, W, ct, cin, h, w, stride, pad)
    ho, wo = O.conv_out_hw(h, w, kh, kh, stride, pad)
    ref = np.zeros((cout, ho, wo), np.int64)
    padded = np.pad(img, ((0, 0), (pad, pad), (pad, pad)))
    for co in range(cout):
        full = sum(correlate2d(padded[ci], W[co, ci], mode="valid") for ci in range(cin))
        ref[co] = full[::stride, ::stride][:ho, :wo]
    exp = ((ref.reshape(-1) + p) % (2 * p)) - p
    assert np.array_equal(O.decrypt(P, K, out), exp)
    # phases are the same linear combination of input phases (exact)
    ph_in = O.phase(P, K, ct).astype(np.int64).reshape(cin, h, w)
    ph_pad = np.pad(ph_in, ((0, 0), (pad, pad), (pad, pad)))
    ref_ph = np.zeros((cout, ho, wo), np.int64)
    for co in range(cout):
        full = sum(correlate2d(ph_pad[ci], W[co, ci], mode="valid") for ci in range(cin))
        ref_ph[co] = full[::stride, ::stride][:ho, :wo]
    assert np.array_equal(O.phase(P, K, out).astype(np.int64), ref_ph.reshape(-1) % 2 ** 32)
