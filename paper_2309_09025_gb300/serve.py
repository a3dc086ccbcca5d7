"""Encrypted inference of images arriving in ragged batches (one JSON line).

    python -m paper_2309_09025_gb300.serve [--images 512] [--T 8] [--variant tc]
                                           [--coalesce 7] [--baseline-images 1]

Seeded MNIST-shaped stroke images (seed 5) arrive in batches whose sizes are
uniform in 1..64 (seed 55).  Each image is encrypted on the device (client
side, not timed), then served through the conv-SNN (conv 1->8 5x5 s2 -> FC
1152->128 -> FC 128->10, LIF, spike-count scores, P630) with T steps:

* "arrivals": every arrival batch is one inference call (CUDA graphs are
  captured once per batch size and reused);
* "coalesced": consecutive arrivals are regrouped into batches of --coalesce
  images that are streamed (fhe_snn_stream_push): each bootstrap launch holds
  every layer's neurons of two consecutive batches; a final partial batch
  runs as one inference call.

The per-image exact CUDA-core path (one image per call, FHE_VARIANT_EXACT) is
timed on --baseline-images images and reported per prediction.
"""
import argparse
import json
import time

import numpy as np


def main():
    import torch

    from paper_2309_09025_gb300 import build, fhe, synth

    ap = argparse.ArgumentParser()
    ap.add_argument("--images", type=int, default=512)
    ap.add_argument("--T", type=int, default=8)
    ap.add_argument("--variant", default="tc", choices=["tc", "exact", "fft"])
    ap.add_argument("--coalesce", type=int, default=7)
    ap.add_argument("--max-arrival", type=int, default=64)
    ap.add_argument("--baseline-images", type=int, default=1)
    args = ap.parse_args()
    build.build()
    P = dict(synth.P630)
    W = P["n"] + 1
    variant = {"tc": fhe.VARIANT_TC, "exact": fhe.VARIANT_EXACT, "fft": fhe.VARIANT_FFT}[args.variant]
    net = synth.csnn_net(T=args.T)
    keys = fhe.keygen_from_seed(P, seed=3, max_batch=max(16384, 1290 * args.max_arrival))
    images = synth.stroke_images(5, args.images)
    sizes = synth.ragged_batch_sizes(55, args.images, 1, args.max_arrival)
    ct = fhe.encrypt(keys, images.reshape(-1), seed=11).view(args.images, 28 * 28, W)
    cap = max(args.max_arrival, args.coalesce)
    snn = fhe.Snn(keys, net, max_images=cap, variant=variant, use_graph=True)
    per_image = snn.pbs_per_image()
    scores = torch.empty((args.images, 10, W), dtype=torch.int32, device="cuda")

    def run(batches):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        i0 = 0
        for b in batches:
            snn.infer(ct[i0:i0 + b].contiguous(), b, scores[i0:i0 + b])
            i0 += b
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    run(sizes[:2])  # warm up (captures the first sizes)
    t_arr = run(sizes)
    scores_arrivals = scores.clone()
    n_full, rest = divmod(args.images, args.coalesce)
    groups = [args.coalesce] * n_full + ([rest] if rest else [])

    def run_streamed():
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for gi in range(n_full):
            i0 = gi * args.coalesce
            snn.stream_push(ct[i0:i0 + args.coalesce].contiguous(), args.coalesce,
                            scores[i0:i0 + args.coalesce])
        snn.stream_flush()
        if rest:
            i0 = n_full * args.coalesce
            snn.infer(ct[i0:].contiguous(), rest, scores[i0:])
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    warm = torch.empty((args.coalesce, 10, W), dtype=torch.int32, device="cuda")
    snn.stream_push(ct[:args.coalesce].contiguous(), args.coalesce, warm)  # allocates the stream state
    snn.stream_flush()
    t_coal = run_streamed()
    same = bool(torch.equal(scores, scores_arrivals))  # deterministic: both schedules agree bit for bit
    pred = np.argmax(fhe.decrypt(keys, scores.view(-1, W)).cpu().numpy().reshape(-1, 10), axis=1)

    base = fhe.Snn(keys, net, max_images=1, variant=fhe.VARIANT_EXACT, use_graph=True)
    one = torch.empty((1, 10, W), dtype=torch.int32, device="cuda")
    base.infer(ct[:1].contiguous(), 1, one)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.baseline_images):
        base.infer(ct[i:i + 1].contiguous(), 1, one)
    torch.cuda.synchronize()
    t_base = (time.perf_counter() - t0) / args.baseline_images
    total = per_image * args.images
    print(json.dumps({
        "workload": "ragged arrivals of 1..%d images, conv-SNN P630, T=%d, %d images"
                    % (args.max_arrival, args.T, args.images),
        "variant": args.variant, "arrival_batches": len(sizes), "pbs_per_image": per_image,
        "arrivals": {"s": t_arr, "ms_per_prediction": 1e3 * t_arr / args.images,
                     "pbs_per_s": total / t_arr},
        "coalesced": {"batch": args.coalesce, "batches": len(groups), "streamed": True, "s": t_coal,
                      "ms_per_prediction": 1e3 * t_coal / args.images,
                      "pbs_per_s": total / t_coal},
        "per_image_exact": {"ms_per_prediction": 1e3 * t_base, "pbs_per_s": per_image / t_base,
                            "images_timed": args.baseline_images},
        "streamed_scores_bit_identical_to_arrivals": same,
        "predicted_class_histogram": np.bincount(pred, minlength=10).tolist(),
    }), flush=True)
    assert keys.status() == fhe.FHE_OK


if __name__ == "__main__":
    main()
