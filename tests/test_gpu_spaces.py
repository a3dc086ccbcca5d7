"""GPU parity of per-layer message spaces (the dynamic message space of
DiNN, which the paper adopts in 5.2): bootstraps that read one space and
write another, grouped tables whose group changes along one launch, and
networks whose layers have their own spaces -- every ciphertext
bit-identical to the oracle on the CUDA-core and tensor-core blind rotations.
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


def gpu_keys(fhe, name, seed, max_batch=0):
    key = (name, seed, max_batch)
    if key not in _GPU_KEYS:
        P = dict(synth.PRESETS[name])
        _GPU_KEYS[key] = (P, fhe.keygen_from_seed(P, seed, max_batch=max_batch))
    return _GPU_KEYS[key]


def u32(t):
    return t.detach().cpu().numpy().view(np.uint32)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def variant_of(fhe, name):
    return getattr(fhe, "VARIANT_" + name)


@pytest.mark.parametrize("variant", ["EXACT", "TC", "FFT"])
@pytest.mark.parametrize("L,lp_in,lp_out", [(1, 3, (6,)), (2, 4, (2, 6)), (2, 6, (5, 5))])
def test_pbs_between_spaces(fhe, oracle_keys, variant, L, lp_in, lp_out):
    """300 inputs of Z_{2 p_in} (three tensor-core tiles and a ragged tail)
    bootstrapped into the output spaces: EXACT and TC bit-identical to the
    oracle, FFT decrypting the same."""
    P, K = gpu_keys(fhe, "T0", 23)
    _, OK = oracle_keys("T0", 23)
    Pi = dict(P, log2_p=lp_in)
    p_in = 1 << lp_in
    g = np.random.default_rng(lp_in + 10 * L)
    f = g.integers(-3, 4, (L, p_in)).astype(np.int32)
    m = g.integers(0, 2 * p_in, 300).astype(np.int32)
    ct = O.encrypt(Pi, OK, m, 400 + lp_in)
    lut = fhe.Lut(K, [f], log2_p_in=[lp_in], log2_p_out=[list(lp_out)])
    try:
        got = u32(fhe.pbs_batch(K, dev(ct), lut, variant=variant_of(fhe, variant)))
    except fhe.FheError as e:
        if e.code == fhe.FHE_EUNSUPPORTED:
            pytest.skip("variant does not cover this parameter set")
        raise
    ref = O.pbs(Pi, OK, ct, f, nthreads=NTHREADS, log2_p_out=list(lp_out))
    if variant == "FFT":
        for j, lo in enumerate(lp_out):
            Po = dict(P, log2_p=lo)
            assert np.array_equal(O.decrypt(Po, OK, got[j]), O.decrypt(Po, OK, ref[j]))
    else:
        assert np.array_equal(got, ref)
    assert K.status() == fhe.FHE_OK


GROUPS = [(5, (3, 6)), (3, (4, 4)), (6, (6, 2)), (4, (2, 5))]  # (log2 p_in, log2 p_out per table)


@pytest.mark.parametrize("variant,max_batch", [("EXACT", 0), ("TC", 0), ("EXACT", 256),
                                               ("TC", 256), ("FFT", 0)])
def test_grouped_tables_along_one_launch(fhe, oracle_keys, variant, max_batch):
    """Four table groups over 400 inputs with boundaries 130, 130 (an empty
    group), 300: each segment bootstrapped with its own group, in one launch
    (max_batch 0) or two chunks that split the third group (max_batch 256).
    Bit-identical to the oracle per segment (FFT: same decryptions)."""
    P, K = gpu_keys(fhe, "T0", 24, max_batch=max_batch)
    _, OK = oracle_keys("T0", 24)
    seg = [0, 130, 130, 300, 400]
    g = np.random.default_rng(5)
    tabs, cts = [], []
    for gi, (lp_in, _) in enumerate(GROUPS):
        p_in = 1 << lp_in
        tabs.append(g.integers(-3, 4, (2, p_in)).astype(np.int32))
        m = g.integers(0, 2 * p_in, seg[gi + 1] - seg[gi]).astype(np.int32)
        cts.append(O.encrypt(dict(P, log2_p=lp_in), OK, m, 500 + gi).reshape(-1, P["n"] + 1))
    ct = np.concatenate(cts)
    lut = fhe.Lut(K, tabs, log2_p_in=[lp for lp, _ in GROUPS],
                  log2_p_out=[list(lo) for _, lo in GROUPS])
    try:
        got = u32(fhe.pbs_batch_groups(K, dev(ct), lut, seg[1:4], variant=variant_of(fhe, variant)))
    except fhe.FheError as e:
        if e.code == fhe.FHE_EUNSUPPORTED:
            pytest.skip("variant does not cover this parameter set")
        raise
    for gi, (lp_in, lp_out) in enumerate(GROUPS):
        a, b = seg[gi], seg[gi + 1]
        if a == b:
            continue
        ref = O.pbs(dict(P, log2_p=lp_in), OK, cts[gi], tabs[gi], nthreads=NTHREADS,
                    log2_p_out=list(lp_out))
        if variant == "FFT":
            for j, lo in enumerate(lp_out):
                Po = dict(P, log2_p=lo)
                assert np.array_equal(O.decrypt(Po, OK, got[j, a:b]), O.decrypt(Po, OK, ref[j]))
        else:
            assert np.array_equal(got[:, a:b], ref), f"group {gi}"
    assert K.status() == fhe.FHE_OK


def test_grouped_tables_reject_bad_use(fhe):
    P, K = gpu_keys(fhe, "T0", 24)
    tabs = [np.zeros((2, 1 << lp), np.int32) for lp, _ in GROUPS]
    lut = fhe.Lut(K, tabs, log2_p_in=[lp for lp, _ in GROUPS],
                  log2_p_out=[list(lo) for _, lo in GROUPS])
    ct = torch.zeros((10, P["n"] + 1), dtype=torch.int32, device="cuda")
    for bad in ([5, 3, 8], [2, 4, 11]):  # decreasing; beyond the batch
        with pytest.raises(fhe.FheError) as e:
            fhe.pbs_batch_groups(K, ct, lut, bad)
        assert e.value.code == fhe.FHE_EINVAL
    with pytest.raises(fhe.FheError) as e:  # a grouped set needs its boundaries
        fhe.pbs_batch(K, ct, lut)
    assert e.value.code == fhe.FHE_EINVAL
    with pytest.raises(fhe.FheError) as e:  # 2 p_in > N
        fhe.Lut(K, [np.zeros((1, 1024), np.int32)], log2_p_in=[10], log2_p_out=[[4]])
    assert e.value.code == fhe.FHE_EINVAL
    with pytest.raises(fhe.FheError) as e:  # one table cannot have groups
        fhe.Lut(K, [np.zeros((1, 8), np.int32)] * 2, log2_p_in=[3, 3], log2_p_out=[[3], [3]])
    assert e.value.code == fhe.FHE_EINVAL


def spaces_net(seed, lps, T=3, sizes=(6, 40, 20, 5)):
    g = np.random.default_rng(seed)
    layers = [{"type": "fc", "W": g.integers(-1, 2, (sizes[i + 1], sizes[i])).astype(np.int32),
               "log2_p": lp} for i, lp in enumerate(lps)]
    return {"layers": layers, "lif": dict(v_th=1, leak_shift=1, spike_scale=1), "T": T,
            "static_input": False}


def make_snn(fhe, K, net, n_images, variant, use_graph=True):
    try:
        return fhe.Snn(K, net, max_images=n_images, variant=variant_of(fhe, variant),
                       use_graph=use_graph)
    except fhe.FheError as e:
        if e.code == fhe.FHE_EUNSUPPORTED:
            pytest.skip("variant does not cover this parameter set")
        raise


@pytest.mark.parametrize("variant", ["EXACT", "TC"])
@pytest.mark.parametrize("lps", [(4, 3, 2), (3, 2, 5)])
def test_network_with_layer_spaces_bit_exact(fhe, oracle_keys, variant, lps):
    """3 images x 3 steps of FC 6->40->20->5 whose layers have their own
    spaces (the first below the input's, so its weights are scaled): scores
    and every layer's last-step spikes bit-identical to the oracle; all
    layers share each iteration's bootstrap launch."""
    P, K = gpu_keys(fhe, "T0", 25)
    _, OK = oracle_keys("T0", 25)
    net = spaces_net(7, lps)
    x = synth.bernoulli_spikes(8, 3, 3 * 6, 0.5).reshape(3, 3, 6)  # [T][images][inputs]
    ct = O.encrypt(P, OK, x.reshape(-1), 81).reshape(3, 3, 6, -1)
    snn = make_snn(fhe, K, net, 3, variant)
    W = P["n"] + 1
    scores = torch.empty((3, 5, W), dtype=torch.int32, device="cuda")
    snn.infer(dev(ct), 3, scores)
    for i in range(3):
        ref = O.snn_encrypted(P, OK, net, ct[:, i], nthreads=NTHREADS)
        assert np.array_equal(u32(scores)[i], ref["scores"]), f"scores of image {i}"
        for li, size in enumerate((40, 20, 5)):
            spk = torch.empty((3, size, W), dtype=torch.int32, device="cuda")
            snn.layer_spikes(li, spk)
            assert np.array_equal(u32(spk)[i], ref["spikes"][li][-1]), f"layer {li} image {i}"
    assert K.status() == fhe.FHE_OK


@pytest.mark.parametrize("variant", ["EXACT", "TC"])
def test_stream_with_layer_spaces(fhe, oracle_keys, variant):
    """Streamed inference (layers of different batches share launches, some
    layers idle while the pipeline fills) with per-layer spaces: each batch's
    scores equal the oracle's."""
    P, K = gpu_keys(fhe, "T0", 25)
    _, OK = oracle_keys("T0", 25)
    net = spaces_net(9, (4, 2, 3), T=2)
    W = P["n"] + 1
    snn = make_snn(fhe, K, net, 2, variant, use_graph=False)
    batches, outs = [], []
    for b in range(3):
        x = synth.bernoulli_spikes(20 + b, 2, 2 * 6, 0.5).reshape(2, 2, 6)
        ct = O.encrypt(P, OK, x.reshape(-1), 90 + b).reshape(2, 2, 6, -1)
        batches.append(ct)
        sc = torch.empty((2, 5, W), dtype=torch.int32, device="cuda")
        snn.stream_push(dev(ct), 2, sc)
        outs.append(sc)
    snn.stream_flush()
    torch.cuda.synchronize()
    for b, ct in enumerate(batches):
        for i in range(2):
            ref = O.snn_encrypted(P, OK, net, ct[:, i], nthreads=NTHREADS)
            assert np.array_equal(u32(outs[b])[i], ref["scores"]), f"batch {b} image {i}"
    assert K.status() == fhe.FHE_OK


def test_poisson_first_layer_with_spaces(fhe, oracle_keys):
    """Poisson encoder in the key's space writing its spikes in the next
    layer's smaller space, 2 images x 3 steps, bit-exact scores."""
    P, K = gpu_keys(fhe, "T0", 26)
    _, OK = oracle_keys("T0", 26)
    g = np.random.default_rng(11)
    net = {"layers": [{"type": "poisson", "M": synth.poisson_thresholds(11, 3, 24, 8)},
                      {"type": "fc", "W": g.integers(-1, 2, (7, 24)).astype(np.int32), "log2_p": 3},
                      {"type": "fc", "W": g.integers(-1, 2, (3, 7)).astype(np.int32), "log2_p": 2}],
           "lif": dict(v_th=1, leak_shift=1, spike_scale=1), "T": 3, "static_input": True}
    px = g.integers(0, 8, (2, 24)).astype(np.int32)
    ct = np.stack([O.encrypt(P, OK, px[i], 30 + i) for i in range(2)])
    snn = make_snn(fhe, K, net, 2, "TC")
    W = P["n"] + 1
    scores = torch.empty((2, 3, W), dtype=torch.int32, device="cuda")
    snn.infer(dev(ct), 2, scores)
    for i in range(2):
        ref = O.snn_encrypted(P, OK, net, ct[i], nthreads=NTHREADS)
        assert np.array_equal(u32(scores)[i], ref["scores"]), f"image {i}"


def test_layer_spaces_rejected_where_they_cannot_be_encoded(fhe):
    P, K = gpu_keys(fhe, "T0", 25)
    bad = [spaces_net(7, (6, 3, 3)),  # first layer above the input's space
           dict(spaces_net(7, (4, 3, 3)), lif_mode="two_pbs"),
           spaces_net(7, (5, 10, 3))]  # 2 p > N
    bad[1]["lif"] = dict(bad[1]["lif"], spike_scale=2)
    for net in bad:
        with pytest.raises(fhe.FheError) as e:
            fhe.Snn(K, net, max_images=1)
        assert e.value.code == fhe.FHE_EINVAL


def test_csnn_layer_spaces_full_size_tc_equals_exact(fhe):
    """The MNIST-shaped conv-SNN at the production ring (n = 630, N = 1024)
    with layer spaces p = 64, 32, 32 (grouped tables in every launch of
    1152 + 128 + 10 neurons): the tensor-core path's scores and spikes equal
    the CUDA-core path's bit for bit, 2 images, T = 2."""
    P, K = gpu_keys(fhe, "P630", 3)
    net = synth.csnn_net(T=2)
    for layer, lp in zip(net["layers"], (6, 5, 5)):
        layer["log2_p"] = lp
    W = P["n"] + 1
    imgs = synth.stroke_images(5, 2).reshape(2, -1)
    ct = fhe.encrypt(K, imgs.reshape(-1), seed=11).view(2, 28 * 28, W)
    res = {}
    for variant in ("EXACT", "TC"):
        snn = make_snn(fhe, K, net, 2, variant)
        sc = torch.empty((2, 10, W), dtype=torch.int32, device="cuda")
        snn.infer(ct, 2, sc)
        spk = torch.empty((2, 128, W), dtype=torch.int32, device="cuda")
        snn.layer_spikes(1, spk)
        res[variant] = (u32(sc), u32(spk))
        snn.free()
    assert np.array_equal(res["EXACT"][0], res["TC"][0])
    assert np.array_equal(res["EXACT"][1], res["TC"][1])
    assert K.status() == fhe.FHE_OK


def test_layer_spaces_cut_bootstrap_failures(fhe, oracle_keys):
    """Measured per-layer bootstrap failures of the conv-SNN at the
    production ring, one step, 8 images: every layer's decrypted spikes
    against the plaintext layer applied to the spikes it actually received
    (so layer l's count holds only its own bootstrap failures).  With the
    key-switching precision of this set (2^-14) the noise of a WeightSum over
    hundreds of inputs spans about a message box at p = 64; halving p for
    layers 1 and 2 (their spaces p = 32) doubles the box and must cut layer
    1's failures."""
    import json

    P, K = gpu_keys(fhe, "P630", 3)
    _, OK = oracle_keys("P630", 3)
    W = P["n"] + 1
    B = 8
    imgs = synth.stroke_images(5, B).reshape(B, -1)
    ct = fhe.encrypt(K, imgs.reshape(-1), seed=11).view(B, 28 * 28, W)
    sizes = (1152, 128, 10)
    rates = {}
    for lps in ((6, 6, 6), (6, 5, 5)):
        net = synth.csnn_net(T=1)
        for layer, lp in zip(net["layers"], lps):
            layer["log2_p"] = lp
        snn = make_snn(fhe, K, net, B, "TC")
        sc = torch.empty((B, 10, W), dtype=torch.int32, device="cuda")
        snn.infer(ct, B, sc)
        spk = []
        for li, size in enumerate(sizes):
            t = torch.empty((B, size, W), dtype=torch.int32, device="cuda")
            snn.layer_spikes(li, t)
            reads = lps[li + 1] if li + 1 < 3 else P["log2_p"]
            spk.append(O.decrypt(dict(P, log2_p=reads), OK, u32(t).reshape(-1, W)).reshape(B, size))
        snn.free()
        miss = [0, 0, 0]
        for i in range(B):
            for li, layer in enumerate(net["layers"]):
                one = dict(net, layers=[layer], static_input=(li == 0))
                x = imgs[i] if li == 0 else spk[li - 1][i][None]
                ref = O.snn_plain(P, one, x)["spikes"][0][0]
                miss[li] += int(np.count_nonzero(ref != spk[li][i]))
        rates[str(lps)] = [m / (B * s) for m, s in zip(miss, sizes)]
    print(json.dumps({"bootstrap_failure_rate_per_layer": rates}))
    uni, spaced = rates["(6, 6, 6)"], rates["(6, 5, 5)"]
    assert spaced[1] < uni[1]
    assert K.status() == fhe.FHE_OK
