"""GPU parity of the network variants beyond the multi-value LIF layer:
the paper's two separate bootstraps per neuron-step (4.2 as printed,
negacyclic tables, no centring) and the Poisson encoder (2.3), on the
CUDA-core and tensor-core blind rotations -- every spike and score
ciphertext bit-identical to the oracle's encrypted network.
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


def make_snn(fhe, K, net, n_images, variant):
    try:
        return fhe.Snn(K, net, max_images=n_images, variant=getattr(fhe, "VARIANT_" + variant),
                       use_graph=True)
    except fhe.FheError as e:
        if e.code == fhe.FHE_EUNSUPPORTED:
            pytest.skip("variant does not cover this parameter set")
        raise


def check_network(fhe, P, OK, snn, net, ct, n_images):
    """Run `n_images` images; compare scores and every layer's last-step
    spikes with the oracle, image by image."""
    W = P["n"] + 1
    n_out = net["layers"][-1]["W"].shape[0]
    scores = torch.empty((n_images, n_out, W), dtype=torch.int32, device="cuda")
    dev = torch.from_numpy(np.ascontiguousarray(ct).view(np.int32)).cuda()
    snn.infer(dev, n_images, scores)
    refs = []
    for i in range(n_images):
        x = ct[i] if net.get("static_input") else ct[:, i]
        refs.append(O.snn_encrypted(P, OK, net, x, nthreads=NTHREADS))
        assert np.array_equal(u32(scores)[i], refs[i]["scores"]), f"scores of image {i}"
    for li, layer in enumerate(net["layers"]):
        size = layer["M"].shape[1] if layer["type"] == "poisson" else layer["W"].shape[0]
        spk = torch.empty((n_images, size, W), dtype=torch.int32, device="cuda")
        snn.layer_spikes(li, spk)
        for i in range(n_images):
            assert np.array_equal(u32(spk)[i], refs[i]["spikes"][li][-1]), f"layer {li} image {i}"


def small_lif_net(seed, T=3):
    g = np.random.default_rng(seed)
    return {"layers": [{"type": "fc", "W": g.integers(-1, 2, (5, 6)).astype(np.int32)},
                       {"type": "fc", "W": g.integers(-1, 2, (3, 5)).astype(np.int32)}],
            "lif": dict(v_th=2, leak_shift=1, spike_scale=2), "T": T,
            "static_input": False, "lif_mode": "two_pbs"}


def small_poisson_net(seed, lif_mode, T=3, n_px=24, levels=8):
    g = np.random.default_rng(seed)
    return {"layers": [{"type": "poisson", "M": synth.poisson_thresholds(seed, T, n_px, levels)},
                       {"type": "fc", "W": g.integers(-1, 2, (7, n_px)).astype(np.int32)},
                       {"type": "fc", "W": g.integers(-1, 2, (3, 7)).astype(np.int32)}],
            "lif": dict(v_th=2, leak_shift=1, spike_scale=2 if lif_mode == "two_pbs" else 1),
            "T": T, "static_input": True, "lif_mode": lif_mode}


@pytest.mark.parametrize("variant", ["EXACT", "TC"])
def test_two_pbs_lif_network_bit_exact(fhe, oracle_keys, variant):
    """FHE-Fire = bootstrap_sign(H - V_th) + 1 and FHE-Reset = bootstrap_g(H),
    two blind rotations per neuron-step, 3 images x 3 steps."""
    P, K = gpu_keys(fhe, "T0", 21)
    _, OK = oracle_keys("T0", 21)
    net = small_lif_net(5)
    x = synth.bernoulli_spikes(6, 3, 3 * 6, 0.5).reshape(3, 3, 6)  # [T][images][inputs]
    ct = O.encrypt(P, OK, x.reshape(-1), 77).reshape(3, 3, 6, -1)
    snn = make_snn(fhe, K, net, 3, variant)
    assert snn.pbs_per_image() == 2 * (5 + 3) * 3
    check_network(fhe, P, OK, snn, net, ct, 3)
    assert K.status() == fhe.FHE_OK


@pytest.mark.parametrize("lif_mode", ["multi", "two_pbs"])
@pytest.mark.parametrize("variant", ["EXACT", "TC"])
def test_poisson_network_bit_exact(fhe, oracle_keys, variant, lif_mode):
    """Poisson encoder (one comparison bootstrap per pixel and step) -> two
    LIF layers, 2 images x 3 steps."""
    P, K = gpu_keys(fhe, "T0", 22)
    _, OK = oracle_keys("T0", 22)
    net = small_poisson_net(9, lif_mode)
    px = np.random.default_rng(10).integers(0, 8, (2, 24)).astype(np.int32)
    ct = np.stack([O.encrypt(P, OK, px[i], 12 + i) for i in range(2)])
    snn = make_snn(fhe, K, net, 2, variant)
    per_lif = 2 if lif_mode == "two_pbs" else 1
    assert snn.pbs_per_image() == (24 + per_lif * (7 + 3)) * 3
    check_network(fhe, P, OK, snn, net, ct, 2)
    assert K.status() == fhe.FHE_OK


def test_poisson_workload_small_ring_bit_exact(fhe, oracle_keys):
    """The Poisson-encoded comparison network at its full shape (784 pixels
    of 16 levels -> FC 160 LIF -> FC 10 LIF) on the small ring (N = 256,
    p = 64), 2 steps, scores bit-exact to the oracle."""
    P, K = gpu_keys(fhe, "P64", 9, log2_p=6)
    _, OK = oracle_keys("P64", 9, log2_p=6)
    net = synth.poisson_fc_net(T=2)
    img = synth.stroke_images(3, 1, levels=synth.POISSON_LEVELS).reshape(1, -1)
    ct = O.encrypt(P, OK, img[0], 100)[None]
    snn = make_snn(fhe, K, net, 1, "EXACT")
    assert snn.pbs_per_image() == (784 + 160 + 10) * 2
    W = P["n"] + 1
    scores = np.zeros((1, 10, W), np.uint32)
    snn.infer(np.ascontiguousarray(ct), 1, scores, on_host=True)
    ref = O.snn_encrypted(P, OK, net, ct[0], nthreads=NTHREADS)
    assert np.array_equal(scores[0], ref["scores"])


def test_two_pbs_requires_spike_value_two(fhe):
    P, K = gpu_keys(fhe, "T0", 21)
    net = small_lif_net(5)
    net["lif"] = dict(net["lif"], spike_scale=1)
    with pytest.raises(fhe.FheError) as e:
        fhe.Snn(K, net, max_images=1)
    assert e.value.code == fhe.FHE_EINVAL


def test_paper_csnn_small_ring_bit_exact(fhe, oracle_keys):
    """The paper's CSNN topology (3.1; conv 1->10 8x8 s2 pad 1 -> 2x2 pooling
    folded into FC 1440->160 (3.3) -> FC 160->10) on the small ring (N = 256,
    p = 64), T = 2, scores bit-exact to the oracle through host buffers."""
    P, K = gpu_keys(fhe, "P64", 9, log2_p=6)
    _, OK = oracle_keys("P64", 9, log2_p=6)
    net = synth.paper_csnn_net(T=2)
    img = synth.stroke_images(3, 1).reshape(1, -1)
    ct = O.encrypt(P, OK, img[0], 100)[None]
    snn = make_snn(fhe, K, net, 1, "EXACT")
    assert snn.pbs_per_image() == (1440 + 160 + 10) * 2
    scores = np.zeros((1, 10, P["n"] + 1), np.uint32)
    snn.infer(np.ascontiguousarray(ct), 1, scores, on_host=True)
    ref = O.snn_encrypted(P, OK, net, ct[0], nthreads=NTHREADS)
    assert np.array_equal(scores[0], ref["scores"])
