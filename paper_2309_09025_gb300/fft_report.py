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
ones.
"""
import argparse
import json

import numpy as np


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
    print(json.dumps({
        "params": args.params, "pbs": done, "fft_pbs_per_s": done / (fft_ms / 1e3),
        "fft_max_rounding_error": keys.fft_max_error(),
        "fft_decryption_failures_vs_exact": fail,
        "exact_intrinsic_failures": intrinsic,
        "fft_bit_identical_fraction": identical / done,
    }), flush=True)
    assert keys.status() == fhe.FHE_OK


if __name__ == "__main__":
    main()
