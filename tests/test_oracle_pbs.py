"""Pins of the oracle's bootstrapping (CPU only).

External product and blind rotation are checked against the homomorphic
identities of paper 2.1 (RGSW product, ACC[-b + sum a_i s_i]) and against the
closed-form noise of the construction; PBS is brute-forced over every message
(Thm 2.1: bootstrap(LWE(m)) = LWE(g(m))).
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2309_09025_gb300 import synth

MASK32 = (1 << 32) - 1


def _signed(x):
    x = np.asarray(x, np.int64) & MASK32
    return np.where(x >= 2 ** 31, x - 2 ** 32, x)


def _exact_phase_tilde(P, K, ct):
    """phi~ = b~ - sum a~_i s_i mod 2N with the secret key (modulus-switched)."""
    N = P["N"]
    n = P["n"]
    bb = O.mod_switch(int(ct[n]), N)
    s = 0
    for i in range(n):
        s += O.mod_switch(int(ct[i]), N) * int(K["lwe_key"][i])
    return (bb - s) % (2 * N)


def _rot_expected(tv, e):
    """Noiseless X^(-e) TV (negacyclic), built from numpy indexing."""
    N = len(tv)
    out = np.zeros(N, np.int64)
    for c in range(N):
        idx = c + e
        sign = 1
        idx %= 2 * N
        if idx >= N:
            idx -= N
            sign = -1
        out[c] = sign * int(tv[idx])
    return out & MASK32


def test_external_product_noiseless(oracle_keys):
    """RLWE(m) <> RGSW(X^0 or X^0*s_i) = s_i * RLWE(m), error only from the
    gadget rounding: |err| <= (1 + kN) * 2^(31 - l*log2 Bg) per coefficient."""
    P, K = oracle_keys("P64", 7, lwe_noise_log2=64, glwe_noise_log2=64)
    N, k, l = P["N"], P["k"], P["l"]
    g = np.random.default_rng(2)
    rows = (k + 1) * l
    ggsw_sz = rows * (k + 1) * N
    bound = (1 + k * N) * 2 ** (31 - l * P["log2_bg"])
    seen = set()
    for i in range(8):
        si = int(K["lwe_key"][i])
        seen.add(si)
        ggsw = K["bsk"][i * ggsw_sz:(i + 1) * ggsw_sz]
        glwe = g.integers(0, 2 ** 32, (k + 1) * N, dtype=np.uint64).astype(np.uint32)
        out = O.external_product(P, ggsw, glwe)
        ph_in = O.glwe_phase(P, K, glwe).astype(np.int64)
        ph_out = O.glwe_phase(P, K, out).astype(np.int64)
        err = _signed(ph_out - si * ph_in)
        assert np.abs(err).max() <= bound
    assert seen == {0, 1}


def test_sample_extract_exact(oracle_keys):
    """Extraction keeps coefficient 0 of the GLWE phase exactly (2.1)."""
    P, K = oracle_keys("P64", 7)
    g = np.random.default_rng(5)
    glwe = g.integers(0, 2 ** 32, (P["k"] + 1) * P["N"], dtype=np.uint64).astype(np.uint32)
    big = O.sample_extract(P, glwe)
    z = K["glwe_key"].astype(np.int64)
    ph = (int(big[-1]) - int(big[:-1].astype(np.int64) @ z)) & MASK32
    assert ph == int(O.glwe_phase(P, K, glwe)[0])


@pytest.mark.parametrize("name,samples", [("P64", 1500), ("P630", 1000)])
def test_key_switch_noise_closed_form(oracle_keys, name, samples):
    """KS: phase_s(out) = phase_z(in) + e with
    Var e = kN/2 * (2^(32 - lks*log2 Bks))^2/12 + kN*lks*(Bks^2+2)/12 * sigma^2.
    At P630 (Bks = 2^2, lks = 7: 14 bits kept) the rounding term dominates,
    sigma ~ 2^20.7: the per-output noise that a WeightSum then multiplies."""
    P, K = oracle_keys(name, 7)
    n, kN = P["n"], P["k"] * P["N"]
    g = np.random.default_rng(6)
    z = K["glwe_key"].astype(np.int64)
    s = K["lwe_key"].astype(np.int64)
    errs = []
    for _ in range(samples):
        big = g.integers(0, 2 ** 32, kN + 1, dtype=np.uint64).astype(np.uint32)
        ph_z = (int(big[-1]) - int(big[:-1].astype(np.int64) @ z)) & MASK32
        out = O.key_switch(P, K, big)
        ph_s = (int(out[-1]) - int(out[:-1].astype(np.int64) @ s)) & MASK32
        errs.append(int(_signed(ph_s - ph_z)))
    errs = np.array(errs, np.float64)
    Bks = 2 ** P["log2_bks"]
    sig = 2.0 ** (32 - P["lwe_noise_log2"])
    var = kN / 2 * (2.0 ** (32 - P["l_ks"] * P["log2_bks"])) ** 2 / 12 \
        + kN * P["l_ks"] * (Bks ** 2 + 2) / 12 * sig ** 2
    assert 0.85 < errs.var() / var < 1.15


def test_blind_rotation_lands_on_test_poly(oracle_keys):
    """ACC ends at X^(-phi~) TV (2.1 Blind Rotation: ACC[-b + sum a_i s_i]),
    with phi~ computed from the secret key; error within 6 sigma of the
    closed-form blind-rotation noise."""
    P, K = oracle_keys("T0", 3)
    p = 1 << P["log2_p"]
    f = synth.uniform_messages(8, p, 2 * p) - p
    tv = O.test_poly(P, f)
    g = np.random.default_rng(1)
    for m in g.integers(0, 2 * p, 3):
        ct = O.encrypt(P, K, [int(m)], 100 + int(m))[0]
        acc = O.blind_rotate(P, K, ct, tv)
        ph = O.glwe_phase(P, K, acc).astype(np.int64)
        exp = _rot_expected(tv, _exact_phase_tilde(P, K, ct))
        err = _signed(ph - exp)
        assert np.abs(err).max() < 2 ** 24  # T0 noise std ~2^17


def _br_noise_var(P):
    """Closed-form blind-rotation output variance (u32 units^2):
    n (k+1) l N (Bg^2+2)/12 sigma_g^2   [digits x key noise]
    + n/2 (1 + kN/2) (2^(32 - l log2 Bg))^2 / 12   [gadget rounding x key]."""
    n, k, N, l = P["n"], P["k"], P["N"], P["l"]
    Bg = 2 ** P["log2_bg"]
    sg = 2.0 ** (32 - P["glwe_noise_log2"])
    return n * (k + 1) * l * N * (Bg ** 2 + 2) / 12 * sg ** 2 \
        + n / 2 * (1 + k * N / 2) * (2.0 ** (32 - l * P["log2_bg"])) ** 2 / 12


def test_blind_rotation_noise_variance(oracle_keys):
    """Sample variance of the blind-rotation error over all coefficients of
    many accumulators within [0.7, 1.3] of the closed form."""
    P, K = oracle_keys("P64", 11)
    p = 1 << P["log2_p"]
    tv = O.test_poly(P, synth.identity_plus_threshold_lut(p))
    errs = []
    g = np.random.default_rng(7)
    for j in range(20):
        ct = O.encrypt(P, K, [int(g.integers(0, p))], 500 + j)[0]
        acc = O.blind_rotate(P, K, ct, tv)
        ph = O.glwe_phase(P, K, acc).astype(np.int64)
        exp = _rot_expected(tv, _exact_phase_tilde(P, K, ct))
        errs.append(_signed(ph - exp))
    errs = np.concatenate(errs).astype(np.float64)
    ratio = errs.var() / _br_noise_var(P)
    assert 0.7 < ratio < 1.3, ratio


def _brute_force_luts(P):
    p = 1 << P["log2_p"]
    g = np.random.default_rng(12)
    return [synth.identity_plus_threshold_lut(p),
            (g.integers(-p, p, p)).astype(np.int32)]


def test_pbs_brute_force_every_message(oracle_keys):
    """Thm 2.1: bootstrap(LWE(m)) decrypts to f(m) for m in [0, p) and to
    -f(m - p) for m in [p, 2p) (negacyclic half), for every message."""
    P, K = oracle_keys("T0", 21)
    p = 1 << P["log2_p"]
    m = np.arange(2 * p, dtype=np.int32)
    ct = O.encrypt(P, K, m, 99)
    for f in _brute_force_luts(P):
        out = O.pbs(P, K, ct, f[None])[0]
        got = O.decrypt(P, K, out)
        fe = np.concatenate([f, -f]).astype(np.int64)
        exp = ((fe + p) % (2 * p)) - p
        assert np.array_equal(got, exp)


def test_pbs_multi_value_brute_force(oracle_keys):
    """Two LUTs from one blind rotation decrypt to (f_0(m), f_1(m))."""
    P, K = oracle_keys("T0", 21)
    p = 1 << P["log2_p"]
    m = np.arange(p, dtype=np.int32)
    ct = O.encrypt(P, K, m, 98)
    luts = O.lif_luts(P, v_th=4, leak_shift=1, spike_scale=1)
    out = O.pbs(P, K, ct, luts)
    for j in range(2):
        assert np.array_equal(O.decrypt(P, K, out[j]), luts[j])


def test_multi_value_identity():
    """(1 - X) * sum_i X^i = 2 mod X^N + 1, so r_j * TV0 = Delta * coeffs_j."""
    P = dict(synth.P64)
    p = 1 << P["log2_p"]
    d = O.delta(P)
    for f in O.lif_luts(P, 8, 1, 1):
        co = O.lut_coeffs(P, f).astype(np.int64)
        r = np.empty_like(co)
        r[0] = co[0] + co[-1]
        r[1:] = co[1:] - co[:-1]
        tv0 = np.full(P["N"], d // 2, np.int64)
        prod = O.negacyclic_mul(r & MASK32, tv0 & MASK32)
        assert np.array_equal(prod.astype(np.int64), (co * d) & MASK32)
        assert np.count_nonzero(r) <= 5  # sparse: jumps of the LUT only


def test_test_poly_box_lookup():
    """Coefficient 0 of X^(-phi) TV is Delta*f(round(phi p / N)) in the first
    half turn and -Delta*f(round(phi p/N) - p) in the second (Thm 2.1)."""
    P = dict(synth.P64)
    N, p = P["N"], 1 << P["log2_p"]
    f = synth.uniform_messages(3, p, p)
    tv = O.test_poly(P, f).astype(np.int64)
    d = O.delta(P)
    for phi in range(2 * N):
        box = ((2 * phi * p + N) // (2 * N)) % (2 * p)  # round(phi p / N) mod 2p
        val = int(f[box]) * d if box < p else -int(f[box - p]) * d
        assert int(_rot_expected(tv, phi)[0]) == val & MASK32


def test_multi_value_output_noise(oracle_keys):
    """Multi-value PBS output error (4.2, read as one blind rotation of TV0, then r_j * ACC,
    extraction, key switch).  r_j * X^(-phi~) TV0 = X^(-phi~) Delta coeffs_j, so
    the noiseless phase is coefficient 0 of X^(-phi~) TV_j; the error is
    (r_j * E_BR)[0] + e_KS with variance ||r_j||^2 Var_BR + Var_KS.  The sample
    variance of the error, each sample scaled by its predicted standard
    deviation, lies within [0.7, 1.3] of 1."""
    P, K = oracle_keys("P64", 13)
    p = 1 << P["log2_p"]
    n, kN = P["n"], P["k"] * P["N"]
    luts = O.lif_luts(P, v_th=8, leak_shift=1, spike_scale=1)
    g = np.random.default_rng(17)
    m = g.integers(0, p, 600).astype(np.int32)
    ct = O.encrypt(P, K, m, 4242)
    out = O.pbs(P, K, ct, luts)
    Bks = 2 ** P["log2_bks"]
    sig = 2.0 ** (32 - P["lwe_noise_log2"])
    var_ks = kN / 2 * (2.0 ** (32 - P["l_ks"] * P["log2_bks"])) ** 2 / 12 \
        + kN * P["l_ks"] * (Bks ** 2 + 2) / 12 * sig ** 2
    scaled = []
    for j in range(2):
        co = O.lut_coeffs(P, luts[j]).astype(np.int64)
        r = np.empty_like(co)
        r[0] = co[0] + co[-1]
        r[1:] = co[1:] - co[:-1]
        var = float((r * r).sum()) * _br_noise_var(P) + var_ks
        tv = O.test_poly(P, luts[j])
        ph = O.phase(P, K, out[j]).astype(np.int64)
        for i in range(len(m)):
            exp = int(_rot_expected(tv, _exact_phase_tilde(P, K, ct[i]))[0])
            scaled.append(float(_signed(int(ph[i]) - exp)) / np.sqrt(var))
    ratio = float(np.var(scaled))
    assert 0.7 < ratio < 1.3, ratio


def test_p630_lif_golden_file_starts_with_the_oracles_bootstraps():
    """The stored P630 LIF hashes (tests/golden/p630_lif_pbs_1000.txt) are
    the oracle's: its first four entries are recomputed here from the same
    seeds (keys 2, messages and encryption 6, the LIF pair of 4.2), and the
    outputs decrypt to the table values of the bootstrap (Thm 2.1)."""
    import hashlib
    from paper_2309_09025_gb300 import synth
    path = os.path.join(os.path.dirname(__file__), "golden", "p630_lif_pbs_1000.txt")
    golden = [l.split()[1:] for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(golden) == 1000
    P = dict(synth.P630)
    p = 1 << P["log2_p"]
    keys = O.keygen(P, 2)
    m = synth.uniform_messages(6, 1000, 2 * p)[:4]
    ct = O.encrypt(P, keys, m, 6)[:4]
    lif = synth.LIF_DEFAULT
    luts = O.lif_luts(P, lif["v_th"], lif["leak_shift"], lif["spike_scale"])
    out = O.pbs(P, keys, ct, luts, nthreads=os.cpu_count())
    for i in range(4):
        for j in range(2):
            h = hashlib.sha256(np.ascontiguousarray(out[j, i], dtype="<u4").tobytes()).hexdigest()[:16]
            assert h == golden[i][j], (i, j)
    # decryptions equal f(u) (u < p) or -f(u - p) (negacyclic half) up to a
    # neighbouring box (the set's modulus-switch failures)
    for j in range(2):
        dec = O.decrypt(P, keys, out[j]).astype(np.int64)
        exp = O.plain_bootstrap(luts[j], m.astype(np.int64), p, centre=False)
        near = [O.plain_bootstrap(luts[j], m.astype(np.int64) + d, p, centre=False) for d in (-1, 1)]
        assert np.all((dec == exp) | (dec == near[0]) | (dec == near[1]))
