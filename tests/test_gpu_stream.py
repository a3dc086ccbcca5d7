"""GPU parity of the streamed inference (fhe_snn_stream_push / flush): a
sequence of batches whose layers overlap in the same bootstrap launches gives,
batch by batch and image by image, exactly the oracle's encrypted network
(and the one-batch fhe_snn_infer result).
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2309_09025_gb300 import synth

pytestmark = pytest.mark.gpu

NTHREADS = os.cpu_count() or 1


@pytest.fixture(scope="module")
def fhe():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_09025_gb300 import build, fhe as F
    build.build()
    return F


_GPU_KEYS = {}


def gpu_keys(fhe, name, seed, **over):
    key = (name, seed, tuple(sorted(over.items())))
    if key not in _GPU_KEYS:
        P = dict(synth.PRESETS[name])
        P.update(over)
        _GPU_KEYS[key] = (P, fhe.keygen_from_seed(P, seed))
    return _GPU_KEYS[key]


def u32(t):
    return t.detach().cpu().numpy().view(np.uint32)


def small_net(seed, T, lif_mode="multi"):
    g = np.random.default_rng(seed)
    return {"layers": [{"type": "fc", "W": g.integers(-1, 2, (5, 6)).astype(np.int32)},
                       {"type": "fc", "W": g.integers(-1, 2, (4, 5)).astype(np.int32)},
                       {"type": "fc", "W": g.integers(-1, 2, (3, 4)).astype(np.int32)}],
            "lif": dict(v_th=2, leak_shift=1, spike_scale=2 if lif_mode == "two_pbs" else 1),
            "T": T, "static_input": False, "lif_mode": lif_mode}


def run_stream(fhe, snn, batches, W, n_out, host, n_images=2):
    outs = []
    for ct in batches:
        if host:
            sc = np.zeros((n_images, n_out, W), np.uint32)
            snn.stream_push(np.ascontiguousarray(ct), n_images, sc, on_host=True)
        else:
            sc = torch.empty((n_images, n_out, W), dtype=torch.int32, device="cuda")
            snn.stream_push(torch.from_numpy(np.ascontiguousarray(ct).view(np.int32)).cuda(), n_images, sc)
        outs.append(sc)
    snn.stream_flush()
    torch.cuda.synchronize()
    return [o if isinstance(o, np.ndarray) else u32(o) for o in outs]


@pytest.mark.parametrize("T,variant,host", [(2, "EXACT", False), (1, "EXACT", True), (3, "TC", False)])
def test_stream_matches_oracle_per_batch(fhe, oracle_keys, T, variant, host):
    """Three layers with T = 1, 2, 3 (three, two and two batches in flight at
    once), four batches of two images each."""
    P, K = gpu_keys(fhe, "T0", 31)
    _, OK = oracle_keys("T0", 31)
    W = P["n"] + 1
    net = small_net(7, T)
    try:
        snn = fhe.Snn(K, net, max_images=2, variant=getattr(fhe, "VARIANT_" + variant))
    except fhe.FheError as e:
        if e.code == fhe.FHE_EUNSUPPORTED:
            pytest.skip("variant does not cover this parameter set")
        raise
    batches = []
    for b in range(4):
        x = synth.bernoulli_spikes(40 + b, T, 2 * 6, 0.5).reshape(T, 2, 6)
        batches.append(O.encrypt(P, OK, x.reshape(-1), 500 + b).reshape(T, 2, 6, W))
    got = run_stream(fhe, snn, batches, W, 3, host)
    for b, ct in enumerate(batches):
        for i in range(2):
            ref = O.snn_encrypted(P, OK, net, ct[:, i], nthreads=NTHREADS)
            assert np.array_equal(got[b][i], ref["scores"]), f"batch {b} image {i}"
    # the one-batch path gives the same ciphertexts
    one = torch.empty((2, 3, W), dtype=torch.int32, device="cuda")
    snn.infer(torch.from_numpy(np.ascontiguousarray(batches[2]).view(np.int32)).cuda(), 2, one)
    assert np.array_equal(u32(one), got[2])
    assert K.status() == fhe.FHE_OK


@pytest.mark.parametrize("lif_mode", ["multi", "two_pbs"])
def test_stream_poisson_and_two_pbs(fhe, oracle_keys, lif_mode):
    """Poisson encoder + two LIF layers (static pixel input), both LIF modes,
    three batches of two images streamed on the tensor-core path."""
    P, K = gpu_keys(fhe, "T0", 32)
    _, OK = oracle_keys("T0", 32)
    W = P["n"] + 1
    g = np.random.default_rng(3)
    net = {"layers": [{"type": "poisson", "M": synth.poisson_thresholds(4, 2, 16, 8)},
                      {"type": "fc", "W": g.integers(-1, 2, (6, 16)).astype(np.int32)},
                      {"type": "fc", "W": g.integers(-1, 2, (3, 6)).astype(np.int32)}],
           "lif": dict(v_th=2, leak_shift=1, spike_scale=2 if lif_mode == "two_pbs" else 1),
           "T": 2, "static_input": True, "lif_mode": lif_mode}
    try:
        snn = fhe.Snn(K, net, max_images=2, variant=fhe.VARIANT_TC)
    except fhe.FheError as e:
        if e.code == fhe.FHE_EUNSUPPORTED:
            pytest.skip("variant does not cover this parameter set")
        raise
    batches = []
    for b in range(3):
        px = np.random.default_rng(60 + b).integers(0, 8, (2, 16)).astype(np.int32)
        batches.append(np.stack([O.encrypt(P, OK, px[i], 70 + 2 * b + i) for i in range(2)]))
    got = run_stream(fhe, snn, batches, W, 3, host=False)
    for b, ct in enumerate(batches):
        for i in range(2):
            ref = O.snn_encrypted(P, OK, net, ct[i], nthreads=NTHREADS)
            assert np.array_equal(got[b][i], ref["scores"]), f"batch {b} image {i}"


def test_stream_rejects_mixed_sizes_and_infer_while_running(fhe):
    P, K = gpu_keys(fhe, "T0", 31)
    W = P["n"] + 1
    net = small_net(7, 2)
    snn = fhe.Snn(K, net, max_images=2)
    x = torch.zeros((2, 2, 6, W), dtype=torch.int32, device="cuda")
    sc = torch.empty((2, 3, W), dtype=torch.int32, device="cuda")
    snn.stream_push(x, 2, sc)
    with pytest.raises(fhe.FheError) as e:
        snn.stream_push(x[:, :1].contiguous(), 1, sc[:1])
    assert e.value.code == fhe.FHE_EINVAL
    with pytest.raises(fhe.FheError) as e:
        snn.infer(x, 2, sc)
    assert e.value.code == fhe.FHE_EINVAL
    snn.stream_flush()
    snn.infer(x, 2, sc)  # usable again after the flush
    torch.cuda.synchronize()


def test_stream_graph_replays_equal_direct_launches(fhe, oracle_keys):
    """With graphs on, the steady-state iterations replay one captured graph
    per residue j mod (T x slots); six batches at T = 2 replay every residue
    at least once.  Scores, the profiled bootstrap launches and the kernel
    count equal those of the same stream launched directly; a second stream
    re-uses the graphs, a smaller batch size and a tuning change re-capture
    them, and sampled images still equal the oracle."""
    P, K = gpu_keys(fhe, "T0", 31)
    _, OK = oracle_keys("T0", 31)
    W = P["n"] + 1
    net = small_net(11, 2)
    variant = fhe.VARIANT_TC
    try:
        g_snn = fhe.Snn(K, net, max_images=2, variant=variant, use_graph=True, profile=True)
    except fhe.FheError as e:
        if e.code != fhe.FHE_EUNSUPPORTED:
            raise
        variant = fhe.VARIANT_EXACT
        g_snn = fhe.Snn(K, net, max_images=2, variant=variant, use_graph=True, profile=True)
    d_snn = fhe.Snn(K, net, max_images=2, variant=variant, use_graph=False, profile=True)
    batches = []
    for b in range(6):
        x = synth.bernoulli_spikes(80 + b, 2, 2 * 6, 0.5).reshape(2, 2, 6)
        batches.append(O.encrypt(P, OK, x.reshape(-1), 900 + b).reshape(2, 2, 6, W))

    def run(snn, bs, n_images=2):
        k0 = fhe.kernel_launches()
        out = run_stream(fhe, snn, [b[:, :n_images] for b in bs], W, 3, host=False, n_images=n_images)
        return out, fhe.kernel_launches() - k0, snn.profile()

    got, kg, pg = run(g_snn, batches)
    ref, kd, pd = run(d_snn, batches)
    for b in range(6):
        assert np.array_equal(got[b], ref[b]), f"batch {b}"
    assert kg == kd
    assert pg[1:] == pd[1:] and pg[1] == 2 * 6 + 3 - 1  # one bootstrap launch per iteration
    for b, i in ((0, 0), (5, 1)):
        want = O.snn_encrypted(P, OK, net, batches[b][:, i], nthreads=NTHREADS)["scores"]
        assert np.array_equal(got[b][i], want), f"oracle: batch {b} image {i}"
    again, _, _ = run(g_snn, batches[:3])  # cached graphs of the first stream
    for b in range(3):
        assert np.array_equal(again[b], ref[b])
    one, _, _ = run(g_snn, batches[:4], n_images=1)  # other batch size
    for b in range(4):
        assert np.array_equal(one[b][0], ref[b][0])
    if variant == fhe.VARIANT_TC:
        K.set_tc_option(fhe.TC_OPT_CLUSTER, 8)
        try:
            moved, _, _ = run(g_snn, batches[:4])
        finally:
            K.set_tc_option(fhe.TC_OPT_CLUSTER, 0)
        for b in range(4):
            assert np.array_equal(moved[b], ref[b])
    assert K.status() == fhe.FHE_OK
