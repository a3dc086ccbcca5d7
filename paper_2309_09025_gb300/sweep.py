"""Batched-PBS throughput sweep (one JSON line per batch size and variant).

    python -m paper_2309_09025_gb300.sweep [--params P630] [--batches 256,1024,4096,16384,65536]
                                           [--variants exact,tc,fft,auto] [--reps 3]
                                           [--tc-cluster 0|4|8|16] [--tc-multicast -1|0|1]
                                           [--tc-l2-hints -1|0|1]

Uniform random messages of Z_64 bootstrapped with the identity-plus-threshold
table f(u) = (u + [u >= p/2]) mod p through fhe_pbs_batch; the ciphertexts
are resident on the device and the time is measured with CUDA events on the
launching stream (median of `reps` runs after one warm-up).  Batches above the
key handle's workspace run in chunks of 16384.
"""
import argparse
import json

import numpy as np


def main():
    import torch

    from paper_2309_09025_gb300 import build, fhe, synth

    ap = argparse.ArgumentParser()
    ap.add_argument("--params", default="P630")
    ap.add_argument("--batches", default="256,1024,4096,16384,65536")
    ap.add_argument("--variants", default="exact,tc")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--tc-cluster", type=int, default=0,
                    help="tensor-core tile shape: 4, 8 or 16 CTAs per tile (0: tuned rule)")
    ap.add_argument("--tc-multicast", type=int, default=-1,
                    help="clusters of 16: 1 multicast, 0 per-CTA digit-tile copies, -1 default")
    ap.add_argument("--tc-l2-hints", type=int, default=-1,
                    help="1: L2 evict-last policy on the digit operand, 0: none, -1: default")
    args = ap.parse_args()
    build.build()
    P = dict(synth.PRESETS[args.params])
    p = 1 << P["log2_p"]
    batches = [int(b) for b in args.batches.split(",")]
    # workspace for the largest batch, so that no batch is split into chunks
    keys = fhe.keygen_from_seed(P, seed=args.seed, max_batch=max(16384, -(-max(batches) // 256) * 256))
    lut = fhe.lut_create(keys, synth.identity_plus_threshold_lut(p)[None])
    keys.set_tc_option(fhe.TC_OPT_CLUSTER, args.tc_cluster)
    keys.set_tc_option(fhe.TC_OPT_MULTICAST, args.tc_multicast)
    keys.set_tc_option(fhe.TC_OPT_L2_HINTS, args.tc_l2_hints)
    macs = P["n"] * (P["k"] + 1) ** 2 * P["l"] * P["N"] ** 2
    for variant in args.variants.split(","):
        v = {"exact": fhe.VARIANT_EXACT, "tc": fhe.VARIANT_TC, "fft": fhe.VARIANT_FFT,
             "auto": fhe.VARIANT_AUTO}[variant]
        if variant == "auto":
            print(json.dumps({"params": args.params, "autotune_tc_min_batch": keys.autotune()}), flush=True)
        for batch in batches:
            msgs = synth.uniform_messages(args.seed + batch, batch, p)
            ct = fhe.encrypt(keys, msgs, seed=1000 + batch)
            out = torch.empty((1, batch, P["n"] + 1), dtype=torch.int32, device="cuda")
            try:
                fhe.pbs_batch(keys, ct, lut, v, out=out)
            except fhe.FheError as e:
                print(json.dumps({"params": args.params, "variant": variant, "batch": batch,
                                  "unavailable": str(e)}), flush=True)
                break
            times = []
            stream = torch.cuda.current_stream()
            for _ in range(args.reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fhe.pbs_batch(keys, ct, lut, v, out=out)
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
            ms = float(np.median(times))
            dec = fhe.decrypt(keys, out[0]).cpu().numpy()
            exact = float(np.mean(dec % (2 * p) == synth.identity_plus_threshold_lut(p)[msgs]))
            print(json.dumps({"params": args.params, "variant": variant, "batch": batch,
                              "tc_cluster": args.tc_cluster, "tc_multicast": args.tc_multicast,
                              "tc_l2_hints": args.tc_l2_hints,
                              "ms": ms, "pbs_per_s": batch / (ms / 1e3),
                              "br_tmac_per_s": macs * batch / (ms / 1e3) / 1e12,
                              "decrypt_exact_fraction": exact}), flush=True)
            assert keys.status() == fhe.FHE_OK


if __name__ == "__main__":
    main()
