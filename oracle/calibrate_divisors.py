"""Choose the per-layer weight divisors of the MNIST-shaped conv-SNN.

Runs only the oracle's plaintext DiCSNN (Thm 3.2) on seeded calibration images
and, layer by layer, picks the smallest integer divisor d_l such that every
synaptic sum stays within Thm 4.1's bound: V_th + max|I| <= p/2.  This mirrors
the paper's empirical estimate of the maximum input of each spiking activation
layer (5.2, Table SIZE_P) on synthetic data.  The printed tuple is stored as
the workload constant CSNN_DIVISORS.

Usage: python -m oracle.calibrate_divisors
"""
import numpy as np

from oracle import oracle as O
from paper_2309_09025_gb300 import synth


def max_abs_inputs(P, net, images):
    p = 1 << P["log2_p"]
    worst = np.zeros(len(net["layers"]), np.int64)
    for img in images:
        res = O.snn_plain(P, net, img.reshape(-1))
        for li in range(len(net["layers"])):
            if net["layers"][li]["type"] == "poisson":
                continue  # no WeightSum, no membrane
            # I[t] = H[t] - V[t-1]; V[-1] = 0
            H = res["h"][li].astype(np.int64)
            V = np.zeros_like(H)
            V[1:] = O.plain_bootstrap(O.lif_luts(P, **net["lif"])[1], H[:-1], p)
            worst[li] = max(worst[li], np.abs(H - V).max())
    return worst


def calibrate(P=synth.P630, n_images=64, seed=1000):
    p = 1 << P["log2_p"]
    images = synth.stroke_images(seed, n_images)
    v_th = synth.LIF_DEFAULT["v_th"]
    divisors = [1, 1, 1]
    for li in range(3):
        while True:
            net = synth.csnn_net(divisors=tuple(divisors))
            worst = max_abs_inputs(P, net, images)
            if v_th + worst[li] <= p // 2:
                break
            divisors[li] += 1
    return tuple(divisors), worst


def calibrate_poisson(P=synth.P630, n_images=16, seed=1000, T=20):
    """Divisors of the Poisson-encoded network's two FC layers (the encoder
    has no weights), on images quantised to POISSON_LEVELS levels."""
    p = 1 << P["log2_p"]
    images = synth.stroke_images(seed, n_images, levels=synth.POISSON_LEVELS)
    v_th = synth.LIF_DEFAULT["v_th"]
    divisors = [1, 1]
    for li in (1, 2):
        while True:
            net = synth.poisson_fc_net(T=T, divisors=tuple(divisors))
            worst = max_abs_inputs(P, net, images)
            if v_th + worst[li] <= p // 2:
                break
            divisors[li - 1] += 1
    return tuple(divisors), worst


if __name__ == "__main__":
    d, w = calibrate()
    print("CSNN_DIVISORS =", d, "max|I| per layer =", w.tolist())
    d, w = calibrate_poisson()
    print("POISSON_DIVISORS =", d, "max|I| per layer =", w.tolist())
