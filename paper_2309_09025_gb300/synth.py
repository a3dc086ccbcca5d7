"""Seeded synthetic inputs and parameter presets.

This module holds workload definitions only: parameter sets, message draws,
spike trains, integer weights and MNIST-shaped stroke images.  It contains none
of the method's arithmetic (no encryption, no bootstrapping, no LIF update), so
the CPU oracle and the CUDA path can both be fed from it.  It imports neither.

Randomness here comes from numpy's PCG64 generator keyed by an integer seed.
"""
import numpy as np

# Parameter presets.  Noise is a power of two: sigma = 2^-x torus units.
# P64: toy encrypted LIF layer (n=64, N=256, Bg=2^8 l=2, Bks=2^4 lks=4, p=32).
P64 = dict(n=64, k=1, N=256, log2_bg=8, l=2, log2_bks=4, l_ks=4, log2_p=5,
           lwe_noise_log2=20, glwe_noise_log2=25)
# P630: MNIST-shaped conv-SNN / batched PBS (n=630, N=1024, Bg=2^7 l=3,
# Bks=2^2 lks=7, p=64).  No noise levels are given with this set; the
# readings 2^-20 (LWE) and 2^-30 (GLWE) keep the key-switch and blind-rotation
# output noise below 1/40 of a message box (with 2^-15 / 2^-25 the key-switch
# noise alone reaches ~0.8 of the half box and outputs misdecode).
P630 = dict(n=630, k=1, N=1024, log2_bg=7, l=3, log2_bks=2, l_ks=7, log2_p=6,
            lwe_noise_log2=20, glwe_noise_log2=30)
# P750: large set (n=750, N=2048, Bg=2^10 l=2); key-switch parameters and
# noise levels are readings (Bks=2^2 lks=7, 2^-20 / 2^-31).
P750 = dict(n=750, k=1, N=2048, log2_bg=10, l=2, log2_bks=2, l_ks=7, log2_p=6,
            lwe_noise_log2=20, glwe_noise_log2=31)
# T0: test-only low-noise set whose bootstraps essentially never fail.
T0 = dict(n=32, k=1, N=1024, log2_bg=8, l=3, log2_bks=4, l_ks=5, log2_p=5,
          lwe_noise_log2=25, glwe_noise_log2=30)

PRESETS = {"P64": P64, "P630": P630, "P750": P750, "T0": T0}

# LIF settings of the workloads: threshold 8, leak = right shift by 1
# (tau = 2), reset to 0, spike encoded as 1.
LIF_DEFAULT = dict(v_th=8, leak_shift=1, spike_scale=1)

# Per-layer weight divisors of the MNIST-shaped conv-SNN (conv, FC1, FC2):
# raw weights uniform in [-15, 15] are divided by d_l and rounded half away
# from zero.  The values were chosen by oracle/calibrate_divisors.py so that
# |I| <= p/2 - V_th on 64 calibration images (Thm 4.1's condition).
CSNN_DIVISORS = (13, 15, 7)

# Poisson-encoded comparison network (2.3, 5.1 Table Poisson): pixel
# intensities quantised to POISSON_LEVELS levels, per-step thresholds M_t
# uniform over the same levels (the paper draws M_t in [0, 255] against
# normalised pixels; 16 levels keep x - M_t + V_th - 1 inside [-p/2, p/2) for
# p = 64).  FC weight divisors chosen by oracle/calibrate_divisors.py.
POISSON_LEVELS = 16
POISSON_DIVISORS = (23, 7)


def rng(seed):
    return np.random.Generator(np.random.PCG64(int(seed)))


def uniform_messages(seed, count, p):
    """Messages uniform in Z_p = {0..p-1}."""
    return rng(seed).integers(0, p, size=int(count), dtype=np.int64).astype(np.int32)


def identity_plus_threshold_lut(p):
    """f(u) = (u + [u >= p/2]) mod p on u in [0, p): the throughput sweep LUT."""
    u = np.arange(p, dtype=np.int64)
    return ((u + (u >= p // 2)) % p).astype(np.int32)


def bernoulli_spikes(seed, T, count, prob):
    return (rng(seed).random((T, count)) < prob).astype(np.int32)


def uniform_weights(seed, shape, lo, hi):
    return rng(seed).integers(lo, hi + 1, size=shape, dtype=np.int64).astype(np.int32)


def _divide_round_away(w, d):
    w = np.asarray(w, np.int64)
    q = (np.abs(w) * 2 + d) // (2 * d)
    return (np.sign(w) * q).astype(np.int32)


def stroke_images(seed, count, size=28, levels=4, sigma=1.2):
    """MNIST-shaped images: 2-4 Gaussian strokes on a zero background.

    Each stroke is a segment between two uniform points in [4, 24]^2 rendered
    as exp(-d^2 / (2 sigma^2)) of the pixel's distance d to the segment; the
    image is the pixelwise max, normalised to max 1 and quantised to
    min(levels-1, floor(levels * x)).  Returns (count, size, size) int32.
    """
    g = rng(seed)
    yy, xx = np.mgrid[0:size, 0:size].astype(np.float64)
    out = np.zeros((count, size, size), np.int32)
    for i in range(count):
        img = np.zeros((size, size))
        for _ in range(int(g.integers(2, 5))):
            p0 = g.uniform(4, 24, size=2)
            p1 = g.uniform(4, 24, size=2)
            d = p1 - p0
            L2 = float(d @ d) + 1e-12
            t = np.clip(((yy - p0[0]) * d[0] + (xx - p0[1]) * d[1]) / L2, 0.0, 1.0)
            dist2 = (yy - (p0[0] + t * d[0])) ** 2 + (xx - (p0[1] + t * d[1])) ** 2
            img = np.maximum(img, np.exp(-dist2 / (2 * sigma * sigma)))
        img /= max(img.max(), 1e-12)
        out[i] = np.minimum(levels - 1, np.floor(levels * img)).astype(np.int32)
    return out


def toy_lif_net(seed=1, n_in=16, n_out=32, T=2, wmax=4):
    """16 binary inputs -> FC -> 32 LIF neurons, T steps (toy LIF layer)."""
    W = uniform_weights(seed, (n_out, n_in), -wmax, wmax)
    return {"layers": [{"type": "fc", "W": W}], "lif": dict(LIF_DEFAULT), "T": T,
            "static_input": False, "n_in": n_in}


def csnn_net(seed=2, T=4, divisors=CSNN_DIVISORS, raw=False):
    """MNIST-shaped conv-SNN: conv 1->8 5x5 s2 (1152 LIF) -> FC 1152->128 LIF
    -> FC 128->10 LIF, spike-count scores.  Pixels are encrypted once and the
    conv output is reused every step (static input)."""
    g = rng(seed)
    Wc = g.integers(-15, 16, size=(8, 1, 5, 5), dtype=np.int64)
    W1 = g.integers(-15, 16, size=(128, 8 * 12 * 12), dtype=np.int64)
    W2 = g.integers(-15, 16, size=(10, 128), dtype=np.int64)
    if not raw:
        Wc = _divide_round_away(Wc, divisors[0])
        W1 = _divide_round_away(W1, divisors[1])
        W2 = _divide_round_away(W2, divisors[2])
    layers = [
        {"type": "conv", "W": np.asarray(Wc, np.int32), "cin": 1, "h": 28, "w": 28,
         "stride": 2, "pad": 0},
        {"type": "fc", "W": np.asarray(W1, np.int32)},
        {"type": "fc", "W": np.asarray(W2, np.int32)},
    ]
    return {"layers": layers, "lif": dict(LIF_DEFAULT), "T": T, "static_input": True,
            "n_in": 28 * 28}


def poisson_thresholds(seed, T, n, levels=POISSON_LEVELS):
    """The server's public random matrices M_t of the Poisson encoder (2.3):
    (T, n) int32, uniform in [0, levels)."""
    return rng(seed).integers(0, levels, size=(T, n), dtype=np.int64).astype(np.int32)


def poisson_fc_net(seed=7, T=20, levels=POISSON_LEVELS, divisors=POISSON_DIVISORS, raw=False,
                   hidden=160, lif_mode="multi"):
    """The Poisson-encoded fully connected SNN of the paper's comparison
    (5.1, Table Poisson): Poisson encoder of the 784 pixels (one comparison
    bootstrap per pixel and step) -> FC 784->hidden LIF -> FC hidden->10 LIF,
    spike-count scores, T steps (the paper's T_1 is 20..100).  Pixels are
    encrypted once (static input, quantised to `levels` levels)."""
    g = rng(seed)
    W1 = g.integers(-15, 16, size=(hidden, 784), dtype=np.int64)
    W2 = g.integers(-15, 16, size=(10, hidden), dtype=np.int64)
    if not raw:
        W1 = _divide_round_away(W1, divisors[0])
        W2 = _divide_round_away(W2, divisors[1])
    layers = [
        {"type": "poisson", "M": poisson_thresholds(seed + 1, T, 784, levels)},
        {"type": "fc", "W": np.asarray(W1, np.int32)},
        {"type": "fc", "W": np.asarray(W2, np.int32)},
    ]
    return {"layers": layers, "lif": dict(LIF_DEFAULT), "T": T, "static_input": True,
            "n_in": 28 * 28, "levels": levels, "lif_mode": lif_mode}


def paper_csnn_net(seed=6, T=2, wmax=3):
    """The paper's CSNN (3.1): conv 1->10, 8x8, stride 2, padding 1 (10x12x12
    LIF) -> 2x2 average pooling -> FC 360->160 LIF -> FC 160->10 LIF.

    The pooling layer is a WeightSum too; its division is moved into the next
    layer's weights (3.3, multi-level discretization: Discret(w, theta/n)), so
    pooling + FC compose into one integer FC 1440->160 whose weight for input
    (c, y, x) is the FC weight of the pooled cell (c, y//2, x//2).  Weights are
    seeded integers in [-wmax, wmax] (the trained weights are not available).
    """
    g = rng(seed)
    Wc = g.integers(-wmax, wmax + 1, size=(10, 1, 8, 8), dtype=np.int64)
    Wfc = g.integers(-wmax, wmax + 1, size=(160, 10, 6, 6), dtype=np.int64)
    W2 = g.integers(-wmax, wmax + 1, size=(10, 160), dtype=np.int64)
    # compose the 2x2 sum pooling (division folded into Wfc) with FC 360->160
    W1 = np.repeat(np.repeat(Wfc, 2, axis=2), 2, axis=3).reshape(160, 10 * 12 * 12)
    layers = [
        {"type": "conv", "W": Wc.astype(np.int32), "cin": 1, "h": 28, "w": 28, "stride": 2,
         "pad": 1},
        {"type": "fc", "W": W1.astype(np.int32)},
        {"type": "fc", "W": W2.astype(np.int32)},
    ]
    return {"layers": layers, "lif": dict(LIF_DEFAULT), "T": T, "static_input": True,
            "n_in": 28 * 28}


def ragged_batch_sizes(seed, total, lo=1, hi=64):
    """Arrival batch sizes uniform in [lo, hi] that sum to `total`."""
    g = rng(seed)
    sizes = []
    left = total
    while left > 0:
        s = int(min(left, g.integers(lo, hi + 1)))
        sizes.append(s)
        left -= s
    return sizes
