"""Streamed throughput of the network workloads (one JSON line each).

    python -m paper_2309_09025_gb300.workloads [--params P630] [--batches 3]
                                               [--only csnn,csnn_two_pbs,paper_csnn,poisson,csnn_spaces]

Each workload runs on the tensor-core blind rotation through the streamed
inference API (fhe_snn_stream_push): two warm-up batches fill the pipeline,
then --batches timed pushes (each exactly one batch of bootstraps), then a
flush outside the timed region.  Images per batch are chosen so that one
bootstrap launch holds about one wave of 36 clusters x 256 ciphertexts.

* csnn: conv 1->8 5x5 s2 -> FC 1152->128 -> FC 128->10, T = 4, one
  multi-value blind rotation per neuron-step;
* csnn_two_pbs: the same network with the paper's two bootstraps per
  neuron-step (4.2, Eq. FHE-Fire / FHE-Reset, spike value 2);
* paper_csnn: conv 1->10 8x8 s2 pad 1 -> pooling folded into FC 1440->160
  -> FC 160->10, T = 2 (3.1, 3.3);
* poisson: Poisson encoder of 784 pixels -> FC 784->160 -> FC 160->10,
  T = 20 (2.3, Table Poisson);
* csnn_spaces: the csnn network with per-layer message spaces p = 64, 32, 32
  (DiNN's dynamic message space, 5.2): one grouped table set, every launch
  still serving all active layers.
"""
import argparse
import json

import numpy as np


def main():
    import torch

    from paper_2309_09025_gb300 import build, fhe, synth

    ap = argparse.ArgumentParser()
    ap.add_argument("--params", default="P630")
    ap.add_argument("--batches", type=int, default=3)
    ap.add_argument("--only", default="csnn,csnn_two_pbs,paper_csnn,poisson,csnn_spaces")
    ap.add_argument("--latency", action="store_true",
                    help="one image per call through fhe_snn_infer (graphs, AUTO variant): "
                         "latency of a single encrypted prediction")
    args = ap.parse_args()
    build.build()
    P = dict(synth.PRESETS[args.params])
    W = P["n"] + 1
    two = synth.csnn_net(T=4)
    two["lif"] = dict(two["lif"], spike_scale=2)
    two["lif_mode"] = "two_pbs"  # spikes of value 2 stay inside Thm 4.1's doubled range
    px16 = lambda seed, n: synth.stroke_images(seed, n, levels=synth.POISSON_LEVELS)
    spaced = synth.csnn_net(T=4)
    for layer, lp in zip(spaced["layers"], (6, 5, 5)):
        layer["log2_p"] = lp
    nets = {  # network, neurons per image (one bootstrap input each), image generator
        "csnn": (synth.csnn_net(T=4), 1152 + 128 + 10, synth.stroke_images),
        "csnn_two_pbs": (two, 1152 + 128 + 10, synth.stroke_images),
        "paper_csnn": (synth.paper_csnn_net(T=2), 1440 + 160 + 10, synth.stroke_images),
        "poisson": (synth.poisson_fc_net(T=20), 784 + 160 + 10, px16),
        "csnn_spaces": (spaced, 1152 + 128 + 10, synth.stroke_images),
    }
    keys = fhe.keygen_from_seed(P, seed=3, max_batch=18432)
    stream = torch.cuda.current_stream()
    for name in args.only.split(","):
        net, neurons, gen = nets[name]
        if args.latency:
            keys.autotune()
            snn = fhe.Snn(keys, net, max_images=1, variant=fhe.VARIANT_AUTO, use_graph=True)
            img = gen(5, 1).reshape(1, -1)
            ct1 = fhe.encrypt(keys, img.reshape(-1), seed=11).view(1, 28 * 28, W)
            sc = torch.empty((1, 10, W), dtype=torch.int32, device="cuda")
            snn.infer(ct1, 1, sc)  # captures the graphs
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.batches):
                snn.infer(ct1, 1, sc)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / args.batches
            print(json.dumps({"workload": name, "params": args.params, "T": net["T"], "images": 1,
                              "pbs_per_image": snn.pbs_per_image(), "ms_per_prediction": ms,
                              "pbs_per_s": snn.pbs_per_image() / (ms / 1e3), "status": keys.status()}),
                  flush=True)
            snn.free()
            continue
        B = max(1, 9216 // neurons)
        snn = fhe.Snn(keys, net, max_images=B, variant=fhe.VARIANT_TC, use_graph=False, profile=True)
        per_image = snn.pbs_per_image()
        imgs = gen(5, B).reshape(B, -1)
        ct = fhe.encrypt(keys, imgs.reshape(-1), seed=11).view(B, 28 * 28, W)
        scores = [torch.empty((B, 10, W), dtype=torch.int32, device="cuda") for _ in range(2)]
        for k in range(2):
            snn.stream_push(ct, B, scores[k % 2])
        torch.cuda.synchronize()
        prof0 = snn.profile()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(args.batches):
            snn.stream_push(ct, B, scores[k % 2])
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        prof = snn.profile()
        snn.stream_flush()
        torch.cuda.synchronize()
        br_ms = prof[0] - prof0[0]
        br_cts = prof[2] - prof0[2]
        macs = P["n"] * (P["k"] + 1) ** 2 * P["l"] * P["N"] ** 2
        print(json.dumps({
            "workload": name, "params": args.params, "T": net["T"], "images_per_batch": B,
            "neurons_per_image": neurons, "pbs_per_image": per_image,
            "pbs_per_s": per_image * B * args.batches / (ms / 1e3),
            "ms_per_prediction": ms / (B * args.batches),
            "blind_rotation_tflops": 2.0 * 4 * macs * br_cts / (br_ms / 1e3) / 1e12,
            "status": keys.status(),
        }), flush=True)
        snn.free()


if __name__ == "__main__":
    main()
