"""Pins of the oracle's spiking-network compositions (CPU only).

The plaintext DiCSNN is pinned by a hand-worked LIF trace (Thm 3.2); the
encrypted DiCSNN is pinned to the plaintext network spike for spike on the
low-noise test set (4.2 FHE-Fire / FHE-Reset, Thm 4.1 respected).
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2309_09025_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _traces():
    out = []
    for line in open(os.path.join(GOLDEN, "lif_trace.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        parts = [p.split() for p in line.split("|")]
        v_th, leak = int(parts[0][0]), int(parts[0][1])
        I, H, S, V = ([int(x) for x in p] for p in parts[1:])
        out.append((v_th, leak, I, H, S, V))
    return out


@pytest.mark.parametrize("trace", _traces())
def test_plain_lif_matches_hand_worked_trace(trace):
    v_th, leak, I, H, S, V = trace
    P = dict(synth.P64)  # p = 32: every value of the trace is in [-16, 16)
    net = {"layers": [{"type": "fc", "W": np.array([[1]], np.int32)}],
           "lif": dict(v_th=v_th, leak_shift=leak, spike_scale=1), "T": len(I),
           "static_input": False}
    res = O.snn_plain(P, net, np.array(I, np.int64).reshape(-1, 1))
    assert res["h"][0][:, 0].tolist() == H
    assert res["spikes"][0][:, 0].tolist() == S
    assert int(res["scores"][0]) == sum(S)
    # V trace: V[t] = Reset(H[t]) is what the next step adds to I[t+1]
    assert [H[t + 1] - I[t + 1] for t in range(len(I) - 1)] == V[:-1]


def test_lif_luts_follow_fhe_fire_and_reset():
    """Eq. FHE-Fire: 2*Spike = Sign(m)+1 style step at V_th; Eq. FHE-Reset:
    0 above threshold, leak in [0, V_th), 0 below 0 -- on the centred input."""
    P = dict(synth.P630)
    p = 1 << P["log2_p"]
    fire, reset = O.lif_luts(P, v_th=8, leak_shift=1, spike_scale=2)
    v = np.arange(p) - p // 2
    assert np.array_equal(fire[v >= 8], np.full((v >= 8).sum(), 2))
    assert np.all(fire[v < 8] == 0)
    assert np.all(reset[v >= 8] == 0) and np.all(reset[v < 0] == 0)
    mid = (v >= 0) & (v < 8)
    assert reset[mid].tolist() == [0, 0, 1, 1, 2, 2, 3, 3]


def _small_net(seed, T=3):
    g = np.random.default_rng(seed)
    W1 = g.integers(-1, 2, (5, 6)).astype(np.int32)
    W2 = g.integers(-1, 2, (3, 5)).astype(np.int32)
    return {"layers": [{"type": "fc", "W": W1}, {"type": "fc", "W": W2}],
            "lif": dict(v_th=2, leak_shift=1, spike_scale=1), "T": T,
            "static_input": False}


def test_thm41_invariant_plain():
    """Thm 4.1: if V_th + max|I| <= p/2 then H in [V_th - p/2, p/2)."""
    P = dict(synth.T0)
    p = 1 << P["log2_p"]
    net = _small_net(3, T=6)
    x = synth.bernoulli_spikes(4, 6, 6, 0.5)
    res = O.snn_plain(P, net, x)
    for li, layer in enumerate(net["layers"]):
        max_I = np.abs(layer["W"]).sum(axis=1).max()
        assert net["lif"]["v_th"] + max_I <= p // 2
        H = res["h"][li]
        assert H.min() >= net["lif"]["v_th"] - p // 2 and H.max() < p // 2


def test_encrypted_snn_matches_plain(oracle_keys):
    """Encrypted DiCSNN = plaintext DiCSNN spike for spike on the low-noise
    set (bootstraps never fail there), including the spike-count scores."""
    P, K = oracle_keys("T0", 31)
    net = _small_net(5, T=3)
    x = synth.bernoulli_spikes(6, 3, 6, 0.5)
    plain = O.snn_plain(P, net, x)
    ct = O.encrypt(P, K, x.reshape(-1), 77).reshape(3, 6, -1)
    enc = O.snn_encrypted(P, K, net, ct)
    for li in range(2):
        got = O.decrypt(P, K, enc["spikes"][li].reshape(-1, P["n"] + 1)).reshape(3, -1)
        assert np.array_equal(got, plain["spikes"][li])
    assert np.array_equal(O.decrypt(P, K, enc["scores"]), plain["scores"])


def test_encrypted_conv_snn_static_input(oracle_keys):
    """Conv layer on pixel ciphertexts computed once and reused each step."""
    P, K = oracle_keys("T0", 31)
    g = np.random.default_rng(8)
    net = {"layers": [{"type": "conv", "W": g.integers(-1, 2, (2, 1, 3, 3)).astype(np.int32),
                       "cin": 1, "h": 5, "w": 5, "stride": 2, "pad": 0},
                      {"type": "fc", "W": g.integers(-1, 2, (2, 8)).astype(np.int32)}],
           "lif": dict(v_th=2, leak_shift=1, spike_scale=1), "T": 2, "static_input": True}
    img = g.integers(0, 2, 25).astype(np.int32)
    plain = O.snn_plain(P, net, img)
    enc = O.snn_encrypted(P, K, net, O.encrypt(P, K, img, 5))
    got = O.decrypt(P, K, enc["spikes"][0].reshape(-1, P["n"] + 1)).reshape(2, -1)
    assert np.array_equal(got, plain["spikes"][0])
    assert np.array_equal(O.decrypt(P, K, enc["scores"]), plain["scores"])


def test_paper_csnn_pool_folded_into_fc():
    """3.3: the 2x2 average pooling's division moved into the next layer's
    weights -- the composed FC equals sum-pooling followed by the FC, checked
    on random spike maps by brute force."""
    net = synth.paper_csnn_net(seed=6)
    W1 = net["layers"][1]["W"].astype(np.int64)
    g = np.random.default_rng(0)
    Wfc = synth.rng(6)
    Wc = Wfc.integers(-3, 4, size=(10, 1, 8, 8), dtype=np.int64)  # same draw order
    Wp = Wfc.integers(-3, 4, size=(160, 10, 6, 6), dtype=np.int64)
    for _ in range(5):
        s = g.integers(0, 2, (10, 12, 12))
        pooled = s.reshape(10, 6, 2, 6, 2).sum(axis=(2, 4))
        ref = np.tensordot(Wp, pooled, axes=([1, 2, 3], [0, 1, 2]))
        assert np.array_equal(W1 @ s.reshape(-1), ref)
    assert np.array_equal(net["layers"][0]["W"], Wc)
    assert net["layers"][0]["pad"] == 1 and W1.shape == (160, 1440)


def test_poisson_rate_follows_pixel_intensity():
    """2.3, Eq. Poisson-coding: with M_t uniform over `levels` values a pixel
    x spikes in a fraction x / levels of the steps -- the comparison is
    strict (x = 0 never spikes; '>=' would give (x + 1) / levels)."""
    levels, T = 16, 4000
    M = synth.poisson_thresholds(11, T, levels, levels)  # column x: thresholds of pixel x
    assert M.min() == 0 and M.max() == levels - 1
    x = np.arange(levels)
    rates = np.stack([O.poisson_spikes(x, M[t], 1) for t in range(T)]).mean(axis=0)
    expect = x / levels
    sd = np.sqrt(expect * (1 - expect) / T)
    assert np.all(np.abs(rates - expect) <= 5 * sd + 1e-12)
    assert rates[0] == 0.0
    assert np.array_equal(O.poisson_spikes([3, 3], [2, 3], 2), [2, 0])


def test_two_pbs_luts_follow_fhe_fire_and_reset():
    """Eq. FHE-Fire (bootstrap_sign(H - V_th) + 1 = 2 Spike) and Eq. FHE-Reset
    evaluated by negacyclic bootstraps without centring (Thm 2.1), over the
    whole range Thm 4.1 allows with the paper's modulus 2p: H in
    [V_th - p, p).  Branch 3 of FHE-Reset (0 on [V_th - p, 0)) is the
    negacyclic image of branch 1."""
    P = dict(synth.P630)
    p = 1 << P["log2_p"]
    v_th = 8
    g = O.lif_luts_two_pbs(P, v_th, 1)
    H = np.arange(v_th - p, p)
    fire = O.wrap2p(O.plain_bootstrap(g[0], H - v_th, p, centre=False) + 1, p)
    assert np.array_equal(fire, np.where(H >= v_th, 2, 0))
    reset = O.plain_bootstrap(g[1], H, p, centre=False)
    assert np.array_equal(reset, np.where(H >= v_th, 0, np.where(H >= 0, H >> 1, 0)))
    # the negacyclic condition g(m + p') = -g(m) of 4.2 (p' = 2p here)
    m = np.arange(2 * p)
    assert np.array_equal(O.wrap2p(O.plain_bootstrap(g[1], m + p, p, centre=False), p),
                          O.wrap2p(-O.plain_bootstrap(g[1], m, p, centre=False), p))


def _two_pbs(net):
    net = dict(net)
    net["lif"] = dict(net["lif"], spike_scale=2)
    net["lif_mode"] = "two_pbs"
    return net


def test_two_pbs_plain_equals_multi_value_in_range():
    """When Thm 4.1 holds both evaluations of 4.2 are the same LIF network
    (spike value 2 in both)."""
    P = dict(synth.T0)
    net = _small_net(5, T=5)
    net["lif"]["spike_scale"] = 2
    x = synth.bernoulli_spikes(6, 5, 6, 0.5)
    a = O.snn_plain(P, net, x)
    b = O.snn_plain(P, _two_pbs(net), x)
    for li in range(2):
        assert np.array_equal(a["spikes"][li], b["spikes"][li])
        assert np.array_equal(a["h"][li], b["h"][li])
    assert np.array_equal(a["scores"], b["scores"])


def _small_poisson_net(seed, T=3, n_px=6, levels=8):
    g = np.random.default_rng(seed)
    return {"layers": [{"type": "poisson", "M": synth.poisson_thresholds(seed, T, n_px, levels)},
                       {"type": "fc", "W": g.integers(-1, 2, (3, n_px)).astype(np.int32)}],
            "lif": dict(v_th=2, leak_shift=1, spike_scale=1), "T": T, "static_input": True}


def test_encrypted_two_pbs_matches_plain(oracle_keys):
    """Two separate bootstraps per neuron-step (4.2 as printed) on ciphertexts
    = plaintext network spike for spike (low-noise set)."""
    P, K = oracle_keys("T0", 31)
    net = _two_pbs(_small_net(5, T=3))
    x = synth.bernoulli_spikes(6, 3, 6, 0.5)
    plain = O.snn_plain(P, net, x)
    ct = O.encrypt(P, K, x.reshape(-1), 77).reshape(3, 6, -1)
    enc = O.snn_encrypted(P, K, net, ct)
    for li in range(2):
        got = O.decrypt(P, K, enc["spikes"][li].reshape(-1, P["n"] + 1)).reshape(3, -1)
        assert np.array_equal(got, plain["spikes"][li])
    assert np.array_equal(O.decrypt(P, K, enc["scores"]), plain["scores"])


@pytest.mark.parametrize("mode", ["multi", "two_pbs"])
def test_encrypted_poisson_matches_plain(oracle_keys, mode):
    """Poisson encoder (2.3) on pixel ciphertexts: one comparison bootstrap
    per pixel and step, then a LIF layer; = plaintext spike for spike."""
    P, K = oracle_keys("T0", 31)
    net = _small_poisson_net(9)
    if mode == "two_pbs":
        net = _two_pbs(net)
    px = np.random.default_rng(10).integers(0, 8, 6).astype(np.int32)
    plain = O.snn_plain(P, net, px)
    enc = O.snn_encrypted(P, K, net, O.encrypt(P, K, px, 12))
    for li in range(2):
        got = O.decrypt(P, K, enc["spikes"][li].reshape(-1, P["n"] + 1)).reshape(3, -1)
        assert np.array_equal(got, plain["spikes"][li])
    assert np.array_equal(O.decrypt(P, K, enc["scores"]), plain["scores"])


def test_poisson_workload_within_table_range():
    """The Poisson-encoded workload keeps every bootstrap input inside the
    table's range: x - M_t + V_th - 1 in [-p/2, p/2) for the encoder, and
    V_th + max|I| <= p/2 (Thm 4.1) for the FC layers on calibration images."""
    P = dict(synth.P630)
    p = 1 << P["log2_p"]
    net = synth.poisson_fc_net(T=20)
    lv, vth = synth.POISSON_LEVELS, net["lif"]["v_th"]
    assert -(lv - 1) + vth - 1 >= -p // 2 and (lv - 1) + vth - 1 < p // 2
    img = synth.stroke_images(1000, 1, levels=lv)[0].reshape(-1)
    res = O.snn_plain(P, net, img)
    for li in (1, 2):
        H = res["h"][li].astype(np.int64)
        assert H.min() >= vth - p // 2 and H.max() < p // 2
