"""Benchmark: encrypted MNIST-shaped conv-SNN inference on GB300.

Workload (one "step" = one encrypted prediction of a batch of images, all T
time steps, every hot-path stage): seeded 28x28 stroke images quantised to
4 levels, encrypted per pixel (LWE n=630); conv 1->8 5x5 s2 (1152 LIF) ->
FC 1152->128 LIF -> FC 128->10 LIF with spike-count scores; TFHE n=630, k=1,
N=1024, Bg=2^7 l=3, key switch 2^2 x 7, p=64 + padding; T=4 (5160
bootstraps per image, each LIF neuron-step one multi-value bootstrap giving
FHE-Fire and FHE-Reset).

Prints one JSON line (rank 0).  `value` is PBS/s over the whole job with the
encrypted inputs resident in HBM; `e2e` is the same metric through the C ABI
with host buffers (H2D of the encrypted images and D2H of the encrypted
scores inside the timed region).  `--impl reference` times the CPU oracle on
the host cores instead (bounded sample per step).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = ("PBS/s INT8-limb TC vs exact CUDA-core (bit-exact); "
          "ms per encrypted SNN prediction")
UNIT = "PBS/s"
SM_COUNT = 152
# INT32 multiply-add issue rate of one SM (4 SMSPs x 16 lanes per clock).
IMAD_PER_SM_CLK = 64
SM_MAX_MHZ = 2070.0
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one
# blind-rotation launch, recorded with the ncu command that measured it and
# a hash of the kernel's source file: a record whose hash no longer matches
# the source (the kernel changed since) reports no traffic.
TRAFFIC_RECORD = os.path.join(ROOT, "profiles", "dram_traffic.txt")
KERNEL_SOURCE = {"tc": "paper_2309_09025_gb300/csrc/fhe_pbs_tc.cu",
                 "exact": "paper_2309_09025_gb300/csrc/fhe_pbs_exact.cu"}


def source_sha16(rel):
    import hashlib
    with open(os.path.join(ROOT, rel), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def recorded_traffic(arm, cts_per_launch):
    """Bytes per launch from the traffic record, or (None, why)."""
    if not os.path.exists(TRAFFIC_RECORD):
        return None, "no traffic record"
    sha = source_sha16(KERNEL_SOURCE[arm])
    for line in open(TRAFFIC_RECORD):
        f = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
        if f.get("arm") != arm:
            continue
        if f.get("sha16") != sha:
            return None, "kernel source changed since the capture"
        if int(f.get("cts_per_launch", -1)) != int(round(cts_per_launch)):
            return None, "captured at %s ciphertexts per launch" % f.get("cts_per_launch")
        return float(f["bytes_per_launch"]), "ncu capture, " + f.get("capture", "")
    return None, "no record for this kernel"


def br_macs(P):
    return P["n"] * (P["k"] + 1) ** 2 * P["l"] * P["N"] ** 2


def workload_name(P, T, images):
    return ("mnist28-csnn conv8x5x5s2-fc128-fc10 LIF, TFHE n=%d N=%d Bg=2^%d l=%d "
            "ks=2^%dx%d p=%d, T=%d, %d images/step" % (
                P["n"], P["N"], P["log2_bg"], P["l"], P["log2_bks"], P["l_ks"],
                1 << P["log2_p"], T, images))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(ms, world, device):
    """Slowest rank's time (the job ends when the last replica ends)."""
    if world <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(pbs_per_rank, world, max_ms):
    """Whole-job bootstraps per second: every replica's work over the
    slowest replica's time (weak scaling, no exchange between replicas)."""
    return pbs_per_rank * world / (max_ms / 1e3)


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_oracle_rate(P, seed, images, n_pbs, nthreads):
    """Oracle PBS/s on the host cores: n_pbs LIF bootstraps of layer-1
    neurons (conv WeightSum + centring + multi-value FHE-Fire/FHE-Reset)."""
    from oracle import oracle as O
    from paper_2309_09025_gb300 import synth
    okeys = O.keygen(P, seed)
    net = synth.csnn_net(T=4)
    img = images[0].reshape(-1)
    ct = O.encrypt(P, okeys, img, 1000)
    conv = net["layers"][0]
    I = O.lwe_conv2d(P, conv["W"], ct, 1, 28, 28, 2, 0)
    H = O.lwe_add_const(P, I[:n_pbs], (1 << P["log2_p"]) // 2)
    luts = O.lif_luts(P, **net["lif"])
    t0 = time.perf_counter()
    O.pbs(P, okeys, H, luts, nthreads=nthreads)
    dt = time.perf_counter() - t0
    return n_pbs / dt, dt


def run_reference(args):
    """Reference arm: the CPU oracle as it stands, on the host cores."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    from paper_2309_09025_gb300 import synth
    P = dict(synth.P630)
    cores = os.cpu_count() or 1
    images = synth.stroke_images(5, 1)
    n_pbs = max(cores, 8)
    times = []
    for it in range(args.warmup + args.steps):
        rate, dt = cpu_oracle_rate(P, 3, images, n_pbs, cores)
        if it >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = n_pbs * len(times) / total
    sample = ("%d layer-1 LIF bootstraps (conv WeightSum + multi-value FHE-Fire/FHE-Reset, "
              "P630) per step on %d threads" % (n_pbs, cores))
    per_image = synth_pbs_per_image(T=4)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": workload_name(P, 4, args.images), "images_per_step": args.images,
                   "sample": "each step times a bounded sample of this workload (%d bootstraps)"
                             % n_pbs},
        "ms_per_prediction": 1e3 * per_image / value,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def synth_pbs_per_image(T):
    return (8 * 12 * 12 + 128 + 10) * T


def time_arm(fhe, keys, net, ct, B, variant, steps, warmup, streamed, world, local, flush, graphs=True):
    """Warm-up, then `steps` timed steps of one variant of the network on
    device-resident inputs: CUDA events on the launching stream around each
    step (an L2-flushing write before each, outside the events), nvidia-smi
    clocks sampled during the timed region, the blind-rotation launches
    bracketed by their own events for the roofline."""
    import torch
    snn = fhe.Snn(keys, net, max_images=B, variant=variant, use_graph=graphs, profile=True)
    P = keys.params
    scores = [torch.empty((B, 10, P["n"] + 1), dtype=torch.int32, device="cuda") for _ in range(2)]
    stream = torch.cuda.current_stream()

    def one_step(k):
        if streamed:
            snn.stream_push(ct, B, scores[k % 2])
        else:
            snn.infer(ct, B, scores[0])

    for k in range(warmup):  # streamed: fills the pipeline
        one_step(k)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    launches0 = fhe.kernel_launches()
    step_ms, br_ms, br_launches, br_cts = [], 0.0, 0, 0
    prof0 = snn.profile() if streamed else (0.0, 0, 0)
    for k in range(steps):
        flush.zero_()  # L2 flush (256 MiB > 129 MB L2), outside the timed events
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        one_step(warmup + k)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        if not streamed:
            ms, nl, nc = snn.profile()
            br_ms += ms
            br_launches += nl
            br_cts += nc
    barrier(world)
    launches = fhe.kernel_launches() - launches0
    clk = clocks.stop()
    if streamed:
        ms, nl, nc = snn.profile()
        br_ms, br_launches, br_cts = ms - prof0[0], nl - prof0[1], nc - prof0[2]
        snn.stream_flush()  # completes the last batch, after the timed region
        torch.cuda.synchronize()
    return {"snn": snn, "total_ms": max_over_ranks(sum(step_ms), world, "cuda"),
            "br_ms": br_ms, "br_launches": br_launches, "br_cts": br_cts,
            "launches": int(launches), "clocks": clk, "per_image": snn.pbs_per_image()}


def barrier(world):
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()


def roofline(P, arm, res):
    """Achieved rate of the dominant kernel (blind rotation) from its launch
    durations measured inside the timed region, against its peak."""
    br_avg_ms = res["br_ms"] / max(res["br_launches"], 1)
    cts = res["br_cts"] / max(res["br_launches"], 1)
    macs_per_launch = br_macs(P) * cts
    traffic, why = recorded_traffic(arm, cts)
    if arm == "exact":
        achieved = macs_per_launch / (br_avg_ms / 1e3) / 1e12
        peak = SM_COUNT * IMAD_PER_SM_CLK * SM_MAX_MHZ * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TIMAD/s",
                "kernel": "k_blind_rotate_exact<1024,4>",
                "peak_basis": "152 SMs x 64 INT32 multiply-adds/clk x 2070 MHz (derived)"}
    else:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        flops = 2.0 * 4 * macs_per_launch  # 4 eight-bit limbs on fp16 tensor cores
        achieved = flops / (br_avg_ms / 1e3) / 1e12
        peak = float(peaks["bf16_tflops_sustained"])
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "kernel": "k_blind_rotate_tc<1024,4>",
                "peak_basis": "measured bf16 sustained (fp16 same rate), of measured"}
    roof["frac"] = achieved / peak
    roof["traffic"] = traffic
    roof["traffic_source"] = why
    roof["launch_ms"] = br_avg_ms
    roof["launches"] = res["br_launches"]
    roof["ciphertexts_per_launch"] = cts
    return roof


def run_ours(args):
    import torch
    from paper_2309_09025_gb300 import build, fhe, synth

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
        # replicas load the library built without cluster-multicast copies
        fhe.use_library(build.build(replica=True))
    else:
        build.build()
    P = dict(synth.P630)
    T = 4
    B = args.images
    streamed = args.schedule == "stream"
    net = synth.csnn_net(T=T)
    # workspace: one bootstrap launch holds every layer's neurons of a batch
    keys = fhe.keygen_from_seed(P, seed=3 + rank, max_batch=max(16384, -(-B * 1290 // 256) * 256))
    keys.set_tc_option(fhe.TC_OPT_L2_HINTS, args.tc_l2_hints)
    if world == 1:
        keys.set_tc_option(fhe.TC_OPT_MULTICAST, args.tc_multicast)
    images = synth.stroke_images(5 + rank, B)
    ct = fhe.encrypt(keys, images.reshape(-1), seed=11 + rank).view(B, 28 * 28, P["n"] + 1)
    variant = fhe.VARIANT_TC if args.variant == "tc" else fhe.VARIANT_EXACT
    if args.variant == "auto":
        variant = fhe.VARIANT_EXACT
        try:
            probe = fhe.Snn(keys, net, max_images=1, variant=fhe.VARIANT_TC, use_graph=False)
            sc = torch.empty((1, 10, P["n"] + 1), dtype=torch.int32, device="cuda")
            probe.infer(ct[:1].contiguous(), 1, sc)
            torch.cuda.synchronize()
            variant = fhe.VARIANT_TC
            probe.free()
        except fhe.FheError:
            pass
    arm = "tc" if variant == fhe.VARIANT_TC else "exact"
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")
    res = time_arm(fhe, keys, net, ct, B, variant, args.steps, args.warmup, streamed, world,
                   local, flush, graphs=not args.no_graphs)
    snn, per_image, total_ms = res["snn"], res["per_image"], res["total_ms"]
    value = job_rate(per_image * B * args.steps, world, total_ms)

    # end to end through the C ABI with pinned host buffers
    e2e = None
    e2e_steps = args.e2e_steps if args.e2e_steps is not None else args.steps
    if not args.no_e2e and e2e_steps > 0:
        h_in = torch.empty(ct.shape, dtype=torch.int32, pin_memory=True)
        h_in.copy_(ct.cpu())
        h_out = [torch.empty((B, 10, P["n"] + 1), dtype=torch.int32, pin_memory=True)
                 for _ in range(2)]

        def host_step(k):
            if streamed:
                snn.stream_push(h_in, B, h_out[k % 2], on_host=True)
                torch.cuda.synchronize()  # the previous batch's scores are on the host now
            else:
                snn.infer(h_in, B, h_out[0], on_host=True)

        for k in range(2 if streamed else 1):  # warm the host path (streamed: fill)
            host_step(k)
        barrier(world)
        e2e_ms = []
        for k in range(e2e_steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            host_step(k)
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
        if streamed:
            snn.stream_flush()
        barrier(world)
        e2e_total = max_over_ranks(sum(e2e_ms), world, "cuda")
        e2e = {"value": job_rate(per_image * B * e2e_steps, world, e2e_total), "unit": UNIT,
               "steps": e2e_steps,
               "h2d_bytes_per_step": int(h_in.numel() * 4),
               "d2h_bytes_per_step": int(h_out[0].numel() * 4)}
    snn.free()

    # the CUDA-core arm of the metric: same workload, schedule and keys
    exact = None
    if arm == "tc" and args.exact_steps > 0 and world == 1:
        xres = time_arm(fhe, keys, net, ct, B, fhe.VARIANT_EXACT, args.exact_steps,
                        args.exact_warmup, streamed, world, local, flush, graphs=not args.no_graphs)
        xres["snn"].free()
        xvalue = per_image * B * args.exact_steps / (xres["total_ms"] / 1e3)
        exact = {"value": xvalue, "unit": UNIT, "steps": args.exact_steps,
                 "warmup": args.exact_warmup, "ms_per_step": xres["total_ms"] / args.exact_steps,
                 "ms_per_prediction": xres["total_ms"] / args.exact_steps / B,
                 "tc_over_exact": value / xvalue,
                 "roofline": roofline(P, "exact", xres), "clocks": xres["clocks"],
                 "gpu_launches": xres["launches"]}

    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cores = os.cpu_count() or 1
        n_pbs = max(cores, 8)
        rate, dt = cpu_oracle_rate(P, 3, images, n_pbs, cores)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "%d layer-1 LIF bootstraps at P630 (%.1f s of CPU work)" % (n_pbs, dt)}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": workload_name(P, T, B), "images_per_step": B,
                   "variant": arm,
                   "schedule": ("streamed: each timed step starts one batch and, in the same "
                                "bootstrap launches, finishes the batch before it (pipeline "
                                "filled by the warm-up steps, drained after the timed region); "
                                "one bootstrap launch per layer-skewed iteration, "
                                + ("each iteration a replayed CUDA graph" if not args.no_graphs
                                   else "launched directly"))
                               if streamed else
                               "one batch per step: layer-skewed, one bootstrap launch per "
                               "iteration, CUDA graph per iteration",
                   "l2": "256 MiB buffer written before every timed step",
                   "tc_l2_hints": args.tc_l2_hints, "tc_multicast": args.tc_multicast,
                   "parallelism": "replicas" if world > 1 else "single-gpu"},
        "ms_per_prediction": total_ms / args.steps / B,
        "pbs_per_image": per_image,
        "roofline": roofline(P, arm, res),
        "exact": exact,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": res["launches"],
        "clocks": res["clocks"],
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    # 7 images: a full layer-skewed iteration bootstraps 7 x 1290 = 9030
    # ciphertexts = 36 tiles of 256, one wave of the 36 co-resident 4-CTA
    # clusters
    ap.add_argument("--images", type=int, default=7)
    ap.add_argument("--variant", default="auto", choices=["auto", "exact", "tc"])
    ap.add_argument("--no-graphs", action="store_true",
                    help="launch every iteration's kernels directly instead of replaying "
                         "one captured CUDA graph per iteration")
    ap.add_argument("--schedule", default="stream", choices=["stream", "batch"],
                    help="stream: batches pipelined across steps; batch: one batch per step")
    ap.add_argument("--e2e-steps", type=int, default=None,
                    help="end-to-end steps (default: --steps)")
    # the CUDA-core arm is ~10x slower per step: a few steps of the same
    # workload keep the run within minutes
    ap.add_argument("--exact-steps", type=int, default=2,
                    help="timed steps of the CUDA-core arm (0: skip it)")
    ap.add_argument("--exact-warmup", type=int, default=1)
    ap.add_argument("--tc-l2-hints", type=int, default=-1,
                    help="tensor-core option: L2 evict-last policy on the digit operand "
                         "(1 on, 0 off, -1 library default)")
    ap.add_argument("--tc-multicast", type=int, default=-1,
                    help="tensor-core option: digit tiles by multicast (1) or per-CTA (0) copies "
                         "(-1 library default)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
