"""FP64-FFT blind rotation against the exact paths at scale (one JSON line).

    python -m paper_2309_09025_gb300.fft_report [--params P750] [--total 1000000]
                                                [--batch 16384]

Uniform random messages of Z_64 are bootstrapped with the identity-plus-
threshold table by the FP64 negacyclic-FFT variant and, on the same
ciphertexts, by the exact tensor-core variant (bit-identical to the CUDA-core
path and to the oracle).  Reported: FFT PBS/s, the largest distance of an FFT
product output to an integer (torus rounding error, in 2^-32 units), the
number of FFT outputs that decrypt differently from the exact path
(decryption failures of the FFT product), the number of exact outputs that
differ from the table value (intrinsic modulus-switch failures of the
parameter set), and the fraction of FFT outputs bit-identical to the exact
ones.  It also measures the device's FP64 peak (cuBLAS DGEMM through torch,
best of several 4096^3 products) and reports the FFT blind rotation's FP64
rate against it: per CMux step, (k+1) l forward and k+1 inverse complex
transforms of M = N/2 points at 5 M log2 M flops each (the conventional
radix-2 count; the kernel's radix-4 passes execute fewer) plus (k+1)^2 l M
complex multiply-adds of 8 flops.
"""
import argparse
import json

import numpy as np


def fft_flops_per_pbs(P):
    """Algorithmic FP64 flops of one FFT blind rotation (n CMux steps)."""
    import math
    M, k, l = P["N"] // 2, P["k"], P["l"]
    transform = 5 * M * math.log2(M)
    per_step = ((k + 1) * l + (k + 1)) * transform + (k + 1) ** 2 * l * M * 8
    return P["n"] * per_step


def fp64_peak_tflops(n=4096, reps=5):
    """Measured FP64 rate of cuBLAS DGEMM on this device (TFLOP/s)."""
    import torch
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    best = 0.0
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        e1.synchronize()
        best = max(best, 2.0 * n ** 3 / (e0.elapsed_time(e1) / 1e3) / 1e12)
    return best


def main():
    import torch

    from paper_2309_09025_gb300 import build, fhe, synth

    ap = argparse.ArgumentParser()
    ap.add_argument("--params", default="P750")
    ap.add_argument("--total", type=int, default=1000000)
    ap.add_argument("--batch", type=int, default=16384)
    ap.add_argument("--seed", type=int, default=4)
    args = ap.parse_args()
    build.build()
    P = dict(synth.PRESETS[args.params])
    p = 1 << P["log2_p"]
    keys = fhe.keygen_from_seed(P, seed=args.seed, max_batch=args.batch)
    table = synth.identity_plus_threshold_lut(p)
    lut = fhe.lut_create(keys, table[None])
    keys.fft_max_error(reset=True)
    fft_ms = 0.0
    done = fail = intrinsic = identical = 0
    stream = torch.cuda.current_stream()
    while done < args.total:
        b = min(args.batch, args.total - done)
        m = synth.uniform_messages(args.seed * 1000003 + done, b, p)
        ct = fhe.encrypt(keys, m, seed=done + 1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out_f = fhe.pbs_batch(keys, ct, lut, fhe.VARIANT_FFT)
        e1.record(stream)
        out_x = fhe.pbs_batch(keys, ct, lut, fhe.VARIANT_TC)
        e1.synchronize()
        fft_ms += e0.elapsed_time(e1)
        dec_f = fhe.decrypt(keys, out_f[0]).cpu().numpy() % (2 * p)
        dec_x = fhe.decrypt(keys, out_x[0]).cpu().numpy() % (2 * p)
        fail += int(np.sum(dec_f != dec_x))
        intrinsic += int(np.sum(dec_x != table[m]))
        identical += int(torch.sum(torch.all(out_f == out_x, dim=-1)).item())
        done += b
    rate = done / (fft_ms / 1e3)
    flops = fft_flops_per_pbs(P)
    peak = fp64_peak_tflops()
    print(json.dumps({
        "params": args.params, "pbs": done, "fft_pbs_per_s": rate,
        "fft_fp64_flops_per_pbs": flops, "fft_fp64_tflops": rate * flops / 1e12,
        "fp64_peak_tflops_measured": peak, "fft_fp64_frac": rate * flops / 1e12 / peak,
        "fft_max_rounding_error": keys.fft_max_error(),
        "fft_decryption_failures_vs_exact": fail,
        "exact_intrinsic_failures": intrinsic,
        "fft_bit_identical_fraction": identical / done,
    }), flush=True)
    assert keys.status() == fhe.FHE_OK


if __name__ == "__main__":
    main()
