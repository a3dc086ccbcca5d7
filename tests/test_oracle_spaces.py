"""Pins of the oracle's per-layer message spaces (CPU only).

The dynamic message space of DiNN, which the paper carries over (5.2, Parameters Selection): a
bootstrap reads its input with the boxes of one space Z_{2 p_in} and writes
each table in the encoding Delta_out = q / (2 p_out) of the space that reads
it.  Pinned by brute force over every message (Thm 2.1 read across two
spaces), the plaintext multi-value identity with scaled r_j, the closed-form
output noise, a hand-worked network whose spike depends on the layer's
wrap-around, and the encrypted network against the plaintext one.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2309_09025_gb300 import synth

from test_oracle_pbs import MASK32, _br_noise_var, _exact_phase_tilde, _rot_expected, _signed


def _expected(f, m, p_in, p_out):
    """Thm 2.1 across spaces: f(m) for m in [0, p_in), -f(m - p_in) on the
    negacyclic half, read mod 2 p_out."""
    f = np.asarray(f, np.int64)
    m = np.asarray(m, np.int64)
    v = np.where(m < p_in, f[np.minimum(m, p_in - 1)], -f[np.maximum(m - p_in, 0)])
    return ((v + p_out) % (2 * p_out)) - p_out


@pytest.mark.parametrize("lp_in,lp_out", [(4, 2), (3, 4), (2, 5), (4, 4)])
def test_pbs_between_spaces_every_message(oracle_keys, lp_in, lp_out):
    """One table: the input encrypted with Delta_in = q / 2^(lp_in + 1)
    decrypts, after the bootstrap, to f(m) with Delta_out, for every message
    of Z_{2 p_in} (low-noise set, no failures)."""
    P, K = oracle_keys("T0", 21)
    Pi, Po = dict(P, log2_p=lp_in), dict(P, log2_p=lp_out)
    p_in, p_out = 1 << lp_in, 1 << lp_out
    m = np.arange(2 * p_in, dtype=np.int32)
    ct = O.encrypt(Pi, K, m, 41)
    f = np.random.default_rng(lp_in * 8 + lp_out).integers(-p_out, p_out, p_in).astype(np.int32)
    out = O.pbs(Pi, K, ct, f[None], log2_p_out=[lp_out])[0]
    assert np.array_equal(O.decrypt(Po, K, out), _expected(f, m, p_in, p_out))


@pytest.mark.parametrize("lp_out", [(2, 4), (5, 3), (3, 3)])
def test_multi_value_mixed_spaces_every_message(oracle_keys, lp_out):
    """Two tables from one blind rotation, each written in its own space.
    The tables step by at most 6 between boxes, as LIF tables do: the
    multi-value output noise grows with ||r_j|| (the tables' jumps), and a
    table of uniform values over all of Z_{2p} would fail on the noise of the
    split alone."""
    P, K = oracle_keys("T0", 22)
    p = 1 << P["log2_p"]
    m = np.arange(2 * p, dtype=np.int32)
    ct = O.encrypt(P, K, m, 42)
    g = np.random.default_rng(3)
    luts = g.integers(-3, 4, (2, p)).astype(np.int32)
    out = O.pbs(P, K, ct, luts, log2_p_out=list(lp_out))
    for j, lo in enumerate(lp_out):
        got = O.decrypt(dict(P, log2_p=lo), K, out[j])
        assert np.array_equal(got, _expected(luts[j], m, p, 1 << lo))


def test_scaled_multi_value_identity():
    """(Delta_j / Delta_min) (1 - X) coeffs_j * (Delta_min / 2) sum X^i =
    Delta_j coeffs_j mod X^N + 1: the scaled r_j land every table in its own
    encoding from the one rotated TV0."""
    P = dict(synth.P64)
    N = P["N"]
    luts = O.lif_luts(P, 8, 1, 1)
    lp_out = [3, 5]
    lp_max = max(lp_out)
    tv0 = np.full(N, 1 << (30 - lp_max), np.int64)
    for j, lo in enumerate(lp_out):
        co = O.lut_coeffs(P, luts[j]).astype(np.int64)
        r = np.empty_like(co)
        r[0] = co[0] + co[-1]
        r[1:] = co[1:] - co[:-1]
        r *= 1 << (lp_max - lo)
        prod = O.negacyclic_mul(r & MASK32, tv0 & MASK32).astype(np.int64)
        assert np.array_equal(prod, (co << (31 - lo)) & MASK32)


def test_mixed_space_output_noise(oracle_keys):
    """A table written p_max / p_j times coarser than TV0 carries
    (p_max / p_j)^2 ||r_j||^2 Var_BR + Var_KS of output noise: the sample
    variance of each error, scaled by its predicted deviation, lies within
    [0.7, 1.3] of 1."""
    P, K = oracle_keys("P64", 13)
    p = 1 << P["log2_p"]
    kN = P["k"] * P["N"]
    luts = O.lif_luts(P, v_th=8, leak_shift=1, spike_scale=1)
    lp_out = [P["log2_p"] - 2, P["log2_p"]]
    m = np.random.default_rng(19).integers(0, p, 500).astype(np.int32)
    ct = O.encrypt(P, K, m, 4343)
    out = O.pbs(P, K, ct, luts, log2_p_out=lp_out)
    Bks = 2 ** P["log2_bks"]
    sig = 2.0 ** (32 - P["lwe_noise_log2"])
    var_ks = kN / 2 * (2.0 ** (32 - P["l_ks"] * P["log2_bks"])) ** 2 / 12 \
        + kN * P["l_ks"] * (Bks ** 2 + 2) / 12 * sig ** 2
    phi = [_exact_phase_tilde(P, K, ct[i]) for i in range(len(m))]
    for j, lo in enumerate(lp_out):
        co = O.lut_coeffs(P, luts[j]).astype(np.int64)
        r = np.empty_like(co)
        r[0] = co[0] + co[-1]
        r[1:] = co[1:] - co[:-1]
        r *= 1 << (max(lp_out) - lo)
        var = float((r * r).sum()) * _br_noise_var(P) + var_ks
        # noiseless phase: coefficient 0 of X^(-phi~) Delta_j coeffs_j
        tvj = (co << (31 - lo)) & MASK32
        ph = O.phase(P, K, out[j]).astype(np.int64)
        errs = np.array([float(_signed(int(ph[i]) - int(_rot_expected(tvj, phi[i])[0])))
                         for i in range(len(m))])
        ratio = float(np.var(errs / np.sqrt(var)))
        assert 0.7 < ratio < 1.3, (j, ratio)


def _two_layer(w0, w1, lp1):
    return {"layers": [{"type": "fc", "W": np.array([[w0]], np.int32)},
                       {"type": "fc", "W": np.array([[w1]], np.int32), "log2_p": lp1}],
            "lif": dict(v_th=1, leak_shift=1, spike_scale=1), "T": 1, "static_input": False}


def test_plain_layer_space_wraps_hand_worked():
    """Hand-worked: layer 0 (p = 32) fires on I = 5 >= V_th = 1.  Layer 1
    reads that spike with weight w.  In p_1 = 4 the centred input is
    u = H + 2 mod 8: w = 1 gives u = 3 < 4, v = 1 >= V_th, a spike; w = 2 gives
    H = 2, outside the table's range [-p_1/2, p_1/2) = [-2, 2): u = 4 lands on
    the negacyclic half, -Fire(v = -2) = 0, no spike.  In the key's space
    p = 32 the same w = 2 fires (u = 18, v = 2)."""
    P = dict(synth.P64)  # log2_p = 5
    x = np.array([[5]])
    r1 = O.snn_plain(P, _two_layer(1, 1, 2), x)
    assert r1["spikes"][0].tolist() == [[1]] and r1["spikes"][1].tolist() == [[1]]
    assert r1["h"][1].tolist() == [[1]]
    r2 = O.snn_plain(P, _two_layer(1, 2, 2), x)
    assert r2["h"][1].tolist() == [[2]] and r2["spikes"][1].tolist() == [[0]]
    r3 = O.snn_plain(P, _two_layer(1, 2, 5), x)
    assert r3["h"][1].tolist() == [[2]] and r3["spikes"][1].tolist() == [[1]]
    assert r3["scores"].tolist() == [1]


def _spaces_net(seed, lps, T=3):
    g = np.random.default_rng(seed)
    W1 = g.integers(-1, 2, (5, 6)).astype(np.int32)
    W2 = g.integers(-1, 2, (4, 5)).astype(np.int32)
    W3 = g.integers(-1, 2, (3, 4)).astype(np.int32)
    layers = [{"type": "fc", "W": W} for W in (W1, W2, W3)]
    for layer, lp in zip(layers, lps):
        layer["log2_p"] = lp
    return {"layers": layers, "lif": dict(v_th=1, leak_shift=1, spike_scale=1), "T": T,
            "static_input": False}


@pytest.mark.parametrize("lps", [(3, 3, 2), (4, 2, 3), (2, 4, 4)])
def test_encrypted_spaces_match_plain(oracle_keys, lps):
    """Encrypted network with per-layer spaces (layer 0's weights scaled by
    p / p_0 in the ciphertext domain, Fire written in the reading layer's
    space) = plaintext network with per-layer wrap, spike for spike, on the
    low-noise set; spikes decrypt in the space of the layer that reads them
    and the scores in the key's space."""
    P, K = oracle_keys("T0", 31)
    net = _spaces_net(5, lps)
    x = synth.bernoulli_spikes(6, 3, 6, 0.5)
    plain = O.snn_plain(P, net, x)
    enc = O.snn_encrypted(P, K, net, O.encrypt(P, K, x.reshape(-1), 77).reshape(3, 6, -1))
    reads = list(lps[1:]) + [P["log2_p"]]
    for li in range(3):
        got = O.decrypt(dict(P, log2_p=reads[li]), K,
                        enc["spikes"][li].reshape(-1, P["n"] + 1)).reshape(3, -1)
        assert np.array_equal(got, plain["spikes"][li])
    assert np.array_equal(O.decrypt(P, K, enc["scores"]), plain["scores"])


def test_encrypted_spaces_poisson_first_layer(oracle_keys):
    """A Poisson first layer compares pixels in the key's space and writes
    its spikes in the next layer's smaller space."""
    P, K = oracle_keys("T0", 31)
    g = np.random.default_rng(9)
    net = {"layers": [{"type": "poisson", "M": synth.poisson_thresholds(9, 3, 6, 8)},
                      {"type": "fc", "W": g.integers(-1, 2, (3, 6)).astype(np.int32),
                       "log2_p": 2}],
           "lif": dict(v_th=1, leak_shift=1, spike_scale=1), "T": 3, "static_input": True}
    px = np.random.default_rng(10).integers(0, 8, 6).astype(np.int32)
    plain = O.snn_plain(P, net, px)
    enc = O.snn_encrypted(P, K, net, O.encrypt(P, K, px, 12))
    got = O.decrypt(dict(P, log2_p=2), K, enc["spikes"][0].reshape(-1, P["n"] + 1)).reshape(3, -1)
    assert np.array_equal(got, plain["spikes"][0])
    assert np.array_equal(O.decrypt(P, K, enc["scores"]), plain["scores"])


def test_layer_spaces_rejects_what_cannot_be_encoded():
    P = dict(synth.T0)  # log2_p = 5, N = 1024
    assert O.layer_spaces(P, _spaces_net(1, (4, 2, 9))) == [4, 2, 9]
    with pytest.raises(ValueError):  # the input's Delta cannot be divided
        O.layer_spaces(P, _spaces_net(1, (6, 2, 2)))
    with pytest.raises(ValueError):  # 2 p > N
        O.layer_spaces(P, _spaces_net(1, (4, 10, 2)))
    net = _spaces_net(1, (4, 3, 3))
    net["lif_mode"] = "two_pbs"
    with pytest.raises(ValueError):
        O.layer_spaces(P, net)
