"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Exact paths must be bit-identical to the oracle for the same seeds (keys,
encryptions, WeightSums, bootstraps).  Sizes span several CTAs and a ragged
tail; the full-size P630/P750 cases compare sampled outputs that the oracle
computes one by one.
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


def gpu_keys(fhe, name, seed, max_batch=0, **over):
    key = (name, seed, max_batch, tuple(sorted(over.items())))
    if key not in _GPU_KEYS:
        P = dict(synth.PRESETS[name])
        P.update(over)
        _GPU_KEYS[key] = (P, fhe.keygen_from_seed(P, seed, max_batch=max_batch))
    return _GPU_KEYS[key]


def u32(t):
    return t.detach().cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("name,seed", [("P64", 1), ("T0", 2), ("P630", 3)])
def test_keygen_bit_exact(fhe, oracle_keys, name, seed):
    P, K = gpu_keys(fhe, name, seed)
    _, OK = oracle_keys(name, seed)
    assert np.array_equal(K.export(fhe.KEY_LWE), OK["lwe_key"])
    assert np.array_equal(K.export(fhe.KEY_GLWE), OK["glwe_key"])
    assert np.array_equal(K.export(fhe.KEY_BSK), OK["bsk"])
    assert np.array_equal(K.export(fhe.KEY_KSK), OK["ksk"])


@pytest.mark.parametrize("name", ["P64", "P630"])
def test_encrypt_decrypt_bit_exact(fhe, oracle_keys, name):
    P, K = gpu_keys(fhe, name, 5)
    _, OK = oracle_keys(name, 5)
    p = 1 << P["log2_p"]
    m = np.concatenate([np.arange(-p, p), synth.uniform_messages(9, 997, p)]).astype(np.int32)
    ct = fhe.encrypt(K, m, seed=44)
    assert np.array_equal(u32(ct), O.encrypt(P, OK, m, 44))
    assert np.array_equal(fhe.decrypt(K, ct).cpu().numpy(), ((m + p) % (2 * p)) - p)
    # empty batches are no-ops
    fhe.encrypt(K, np.zeros(0, np.int32), seed=1)


def test_lwe_linear_bit_exact(fhe, oracle_keys):
    P = dict(synth.P630)
    g = np.random.default_rng(3)
    K_in, M, batch = 67, 45, 3  # ragged against the 32 x 128 tiles
    W = g.integers(-15, 16, (M, K_in)).astype(np.int32)
    bias = g.integers(-5, 6, M).astype(np.int32)
    ct = g.integers(0, 2 ** 32, (batch, K_in, P["n"] + 1), dtype=np.uint64).astype(np.uint32)
    out = fhe.lwe_linear(P, torch.from_numpy(W).cuda(), ct, bias=torch.from_numpy(bias).cuda())
    for b in range(batch):
        assert np.array_equal(u32(out[b]), O.lwe_linear(P, W, ct[b], bias))


def test_lwe_conv2d_bit_exact(fhe):
    P = dict(synth.P630)
    g = np.random.default_rng(4)
    W = g.integers(-15, 16, (8, 1, 5, 5)).astype(np.int32)
    ct = g.integers(0, 2 ** 32, (2, 28 * 28, P["n"] + 1), dtype=np.uint64).astype(np.uint32)
    out = fhe.lwe_conv2d(P, torch.from_numpy(W).cuda(), ct, 1, 28, 28, 2, 0, batch=2)
    for b in range(2):
        assert np.array_equal(u32(out[b]), O.lwe_conv2d(P, W, ct[b], 1, 28, 28, 2, 0))
    W2 = g.integers(-3, 4, (3, 2, 3, 3)).astype(np.int32)
    ct2 = g.integers(0, 2 ** 32, (1, 2 * 7 * 6, P["n"] + 1), dtype=np.uint64).astype(np.uint32)
    out2 = fhe.lwe_conv2d(P, torch.from_numpy(W2).cuda(), ct2, 2, 7, 6, 2, 1)
    assert np.array_equal(u32(out2[0]), O.lwe_conv2d(P, W2, ct2[0], 2, 7, 6, 2, 1))


def _luts(P, L):
    p = 1 << P["log2_p"]
    if L == 1:
        return synth.identity_plus_threshold_lut(p)[None]
    return O.lif_luts(P, v_th=8 if p >= 32 else 2, leak_shift=1, spike_scale=1)


VARIANTS = ["EXACT", "TC"]  # bit-exact variants


def pbs(fhe, K, ct, lut, variant):
    """pbs_batch through the C ABI; variants without coverage of a parameter
    set (FHE_EUNSUPPORTED) are skipped, never replaced."""
    try:
        return fhe.pbs_batch(K, ct, lut, getattr(fhe, "VARIANT_" + variant))
    except fhe.FheError as e:
        if e.code == fhe.FHE_EUNSUPPORTED:
            pytest.skip("%s variant does not cover this parameter set" % variant)
        raise


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("L", [1, 2])
def test_pbs_p64_bit_exact_all_messages(fhe, oracle_keys, variant, L):
    P, K = gpu_keys(fhe, "P64", 1)
    _, OK = oracle_keys("P64", 1)
    p = 1 << P["log2_p"]
    m = np.concatenate([np.arange(2 * p), synth.uniform_messages(2, 37, 2 * p)]).astype(np.int32)
    ct = O.encrypt(P, OK, m, 123)  # 101 ciphertexts: ragged against 8 per CTA
    luts = _luts(P, L)
    lut = fhe.lut_create(K, luts)
    out = pbs(fhe, K, ct, lut, variant)
    torch.cuda.synchronize()
    ref = O.pbs(P, OK, ct, luts, nthreads=NTHREADS)
    assert np.array_equal(u32(out), ref)
    assert K.status() == fhe.FHE_OK


@pytest.mark.parametrize("variant", VARIANTS)
def test_pbs_t0_brute_force_and_bit_exact(fhe, oracle_keys, variant):
    P, K = gpu_keys(fhe, "T0", 2)
    _, OK = oracle_keys("T0", 2)
    p = 1 << P["log2_p"]
    m = np.arange(2 * p, dtype=np.int32)
    ct = O.encrypt(P, OK, m, 5)
    for L in (1, 2):
        luts = _luts(P, L)
        out = pbs(fhe, K, ct, fhe.lut_create(K, luts), variant)
        got = u32(out)
        for j in range(L):
            dec = O.decrypt(P, OK, got[j])
            fe = np.concatenate([luts[j], -luts[j]]).astype(np.int64)
            assert np.array_equal(dec, ((fe + p) % (2 * p)) - p)
        ref = O.pbs(P, OK, ct, luts, nthreads=NTHREADS)
        assert np.array_equal(got, ref)


def test_pbs_chunked_workspace_and_edges(fhe, oracle_keys):
    """Batches above the workspace capacity run in chunks; 0 and 1 items."""
    P, K = gpu_keys(fhe, "P64", 1, max_batch=24)
    _, OK = oracle_keys("P64", 1)
    p = 1 << P["log2_p"]
    m = synth.uniform_messages(17, 61, p)
    ct = O.encrypt(P, OK, m, 8)
    luts = _luts(P, 2)
    lut = fhe.lut_create(K, luts)
    out = fhe.pbs_batch(K, ct, lut, fhe.VARIANT_EXACT)
    assert np.array_equal(u32(out), O.pbs(P, OK, ct, luts, nthreads=NTHREADS))
    one = fhe.pbs_batch(K, ct[:1], lut, fhe.VARIANT_EXACT)
    assert np.array_equal(u32(one), O.pbs(P, OK, ct[:1], luts))
    empty = torch.empty((2, 0, P["n"] + 1), dtype=torch.int32, device="cuda")
    fhe.pbs_batch(K, torch.empty((0, P["n"] + 1), dtype=torch.int32, device="cuda"), lut,
                  fhe.VARIANT_EXACT, out=empty)


@pytest.mark.parametrize("name,count", [("P630", 1523), ("P750", 613)])
@pytest.mark.parametrize("variant", VARIANTS)
def test_pbs_full_size_sampled(fhe, oracle_keys, name, count, variant):
    """Full-size parameter sets: a batch spanning many CTAs with a ragged
    tail; sampled outputs bit-exact to the oracle, every output decrypting to
    the table value or a neighbouring box (modulus-switch failures)."""
    P, K = gpu_keys(fhe, name, 3)
    _, OK = oracle_keys(name, 3)
    p = 1 << P["log2_p"]
    m = synth.uniform_messages(31, count, p)
    ct = fhe.encrypt(K, m, seed=99)
    luts = _luts(P, 1)
    out = pbs(fhe, K, ct, fhe.lut_create(K, luts), variant)
    got = u32(out)[0]
    octs = O.encrypt(P, OK, m, 99)
    assert np.array_equal(u32(ct), octs)
    idx = np.array([0, 1, 2, 3, count // 2, count - 3, count - 2, count - 1])
    ref = O.pbs(P, OK, octs[idx], luts, nthreads=NTHREADS)[0]
    assert np.array_equal(got[idx], ref)
    dec = O.decrypt(P, OK, got).astype(np.int64) % (2 * p)
    f = luts[0].astype(np.int64)

    def table(u):  # bootstrap value of message u in Z_2p (negacyclic half)
        u = u % (2 * p)
        return np.where(u < p, f[np.minimum(u, p - 1)], -f[np.maximum(u - p, 0)]) % (2 * p)

    m64 = m.astype(np.int64)
    exact = dec == table(m64)
    neighbour = (dec == table(m64 - 1)) | (dec == table(m64 + 1))
    assert np.all(exact | neighbour)
    assert np.mean(~exact) < 0.25


def test_snn_toy_layer_bit_exact(fhe, oracle_keys):
    """16 Bernoulli(0.3) spikes -> 32 LIF neurons, T = 2 (64 bootstraps)."""
    P, K = gpu_keys(fhe, "P64", 1)
    _, OK = oracle_keys("P64", 1)
    net = synth.toy_lif_net(seed=1)
    x = synth.bernoulli_spikes(1, 2, 16, 0.3)
    ct = O.encrypt(P, OK, x.reshape(-1), 7).reshape(1, 2, 16, -1)
    for use_graph in (False, True):
        snn = fhe.Snn(K, net, max_images=1, use_graph=use_graph)
        assert snn.pbs_per_image() == 64
        scores = torch.empty((1, 32, P["n"] + 1), dtype=torch.int32, device="cuda")
        snn.infer(torch.from_numpy(ct.view(np.int32)).cuda(), 1, scores)
        ref = O.snn_encrypted(P, OK, net, ct[0], nthreads=NTHREADS)
        assert np.array_equal(u32(scores)[0], ref["scores"])


def test_snn_csnn_topology_small_params_bit_exact(fhe, oracle_keys):
    """The MNIST-shaped conv-SNN (conv 5x5 s2 -> 1152 LIF -> FC 128 LIF ->
    FC 10 LIF) end to end on 2 images with the small ring (N=256, p=64),
    scores bit-exact to the oracle; host buffers through the C ABI."""
    P, K = gpu_keys(fhe, "P64", 9, log2_p=6)
    _, OK = oracle_keys("P64", 9, log2_p=6)
    net = synth.csnn_net(seed=2, T=2)
    imgs = synth.stroke_images(3, 2).reshape(2, -1)
    ct = np.stack([O.encrypt(P, OK, imgs[i], 100 + i) for i in range(2)])
    snn = fhe.Snn(K, net, max_images=2, use_graph=True)
    scores = np.zeros((2, 10, P["n"] + 1), np.uint32)
    snn.infer(np.ascontiguousarray(ct), 2, scores, on_host=True)
    for i in range(2):
        ref = O.snn_encrypted(P, OK, net, ct[i], nthreads=NTHREADS)
        assert np.array_equal(scores[i], ref["scores"])


@pytest.mark.parametrize("name,count", [("P630", 389), ("P750", 613), ("P630", 3999), ("P750", 3999)])
def test_tc_matches_exact_full_batch(fhe, oracle_keys, name, count):
    """Tensor-core blind rotation: every output of a multi-cluster batch
    (ragged against 256-ciphertext cluster tiles) bit-identical to the
    CUDA-core path, outputs at the tile edges bit-identical to the oracle, for
    both table counts (P750: N = 2048 with split sub-digits).  With the
    default rule, the small batches run on clusters of 16 CTAs and 16 tiles
    (3999 ciphertexts) on clusters of 4 (every shape is forced in
    test_tc_every_tile_shape_bit_exact)."""
    P, K = gpu_keys(fhe, name, 3)
    _, OK = oracle_keys(name, 3)
    p = 1 << P["log2_p"]
    m = synth.uniform_messages(41, count, p)
    ct = fhe.encrypt(K, m, seed=7)
    for L in (1, 2):
        luts = _luts(P, L)
        lut = fhe.lut_create(K, luts)
        ref_gpu = u32(fhe.pbs_batch(K, ct, lut, fhe.VARIANT_EXACT))
        got = u32(pbs(fhe, K, ct, lut, "TC"))
        assert np.array_equal(got, ref_gpu)
        idx = np.array([0, 255, 256, count - 1])
        ref = O.pbs(P, OK, u32(ct)[idx], luts, nthreads=NTHREADS)
        assert np.array_equal(got[:, idx], ref)
    assert K.status() == fhe.FHE_OK


@pytest.mark.parametrize("name,count", [("P630", 389), ("P750", 613)])
def test_tc_every_tile_shape_bit_exact(fhe, oracle_keys, name, count):
    """Every shape of the tensor-core kernel forced in turn (fhe_pbs_set_tc_option):
    256-ciphertext tiles on clusters of 4, 8 and 16 CTAs and spread over two
    clusters of 16 (the two pairs of each block adding into it), each shape
    with multicast and with per-CTA digit-tile copies, with and without the
    L2 policy on the digit operand; all outputs of both
    LIF tables bit-identical to the CUDA-core path, tile-edge outputs to the
    oracle."""
    P, K = gpu_keys(fhe, name, 3)
    _, OK = oracle_keys(name, 3)
    p = 1 << P["log2_p"]
    m = synth.uniform_messages(47, count, 2 * p)
    ct = fhe.encrypt(K, m, seed=23)
    luts = _luts(P, 2)
    lut = fhe.lut_create(K, luts)
    ref_gpu = u32(fhe.pbs_batch(K, ct, lut, fhe.VARIANT_EXACT))
    idx = np.array([0, 255, 256, count - 1])
    ref = O.pbs(P, OK, u32(ct)[idx], luts, nthreads=NTHREADS)
    assert np.array_equal(ref_gpu[:, idx], ref)
    try:
        for cluster, mc, hint in [(4, -1, 0), (8, -1, 0), (16, 1, 0), (16, 0, 0), (32, -1, 0),
                                  (4, 0, 0), (8, 0, 0), (4, -1, 1), (16, 1, 1)]:
            K.set_tc_option(fhe.TC_OPT_CLUSTER, cluster)
            K.set_tc_option(fhe.TC_OPT_MULTICAST, mc)
            K.set_tc_option(fhe.TC_OPT_L2_HINTS, hint)
            got = u32(pbs(fhe, K, ct, lut, "TC"))
            assert np.array_equal(got, ref_gpu), f"clusters of {cluster}, multicast {mc}, L2 {hint}"
            if cluster == 32:  # the split shape really ran (not a fallback to 16)
                assert K.tuning()[3] >= -(-count // 256), "two-cluster tiles were not launched"
    finally:
        for opt, v in ((fhe.TC_OPT_CLUSTER, 0), (fhe.TC_OPT_MULTICAST, -1), (fhe.TC_OPT_L2_HINTS, -1)):
            K.set_tc_option(opt, v)
    assert K.status() == fhe.FHE_OK


def test_tc_matches_exact_across_workspace_chunks(fhe, oracle_keys):
    """A batch larger than the key handle's workspace (16384 ciphertexts)
    runs in two chunks (a full wave-sized chunk, then a ragged one of 2000):
    every output of both tables bit-identical between the tensor-core and
    CUDA-core paths, the outputs on both sides of the chunk edge and at the
    ends bit-identical to the oracle."""
    P, K = gpu_keys(fhe, "P630", 3)
    _, OK = oracle_keys("P630", 3)
    count = 16384 + 2000
    m = synth.uniform_messages(43, count, 1 << P["log2_p"])
    ct = fhe.encrypt(K, m, seed=9)
    luts = _luts(P, 2)
    lut = fhe.lut_create(K, luts)
    ref_gpu = u32(fhe.pbs_batch(K, ct, lut, fhe.VARIANT_EXACT))
    got = u32(pbs(fhe, K, ct, lut, "TC"))
    assert np.array_equal(got, ref_gpu)
    idx = np.array([0, 16383, 16384, count - 1])
    ref = O.pbs(P, OK, u32(ct)[idx], luts, nthreads=NTHREADS)
    assert np.array_equal(got[:, idx], ref)
    assert K.status() == fhe.FHE_OK


def test_csnn_full_size_layer_chain_tc(fhe, oracle_keys):
    """The bench's network at full size (P630, conv 1->8 5x5 s2 -> FC
    1152->128 -> FC 128->10, 7 images, tensor cores), T = 1 so that every
    layer's spikes are observable: sampled neurons of each layer are
    recomputed by the oracle from the GPU's spikes of the layer before
    (WeightSum + centring + multi-value bootstrap) and must match bit for
    bit; the scores are the last layer's spikes."""
    P, K = gpu_keys(fhe, "P630", 3)
    _, OK = oracle_keys("P630", 3)
    W = P["n"] + 1
    p = 1 << P["log2_p"]
    B = 7
    net = synth.csnn_net(T=1)
    imgs = synth.stroke_images(5, B).reshape(B, -1)
    ct = fhe.encrypt(K, imgs.reshape(-1), seed=11).view(B, 28 * 28, W)
    snn = fhe.Snn(K, net, max_images=B, variant=fhe.VARIANT_TC, use_graph=True)
    scores = torch.empty((B, 10, W), dtype=torch.int32, device="cuda")
    snn.infer(ct, B, scores)
    sizes = [1152, 128, 10]
    spk = []
    for li, size in enumerate(sizes):
        t = torch.empty((B, size, W), dtype=torch.int32, device="cuda")
        snn.layer_spikes(li, t)
        spk.append(u32(t))
    assert np.array_equal(spk[2], u32(scores))
    luts = O.lif_luts(P, **net["lif"])
    x_img = u32(ct)
    picks = [(0, 0), (3, 577), (6, 1151)]  # (image, neuron) per layer, scaled to its size
    for li, size in enumerate(sizes):
        rows = []
        for img, nrn in picks:
            nrn = nrn * size // 1152
            layer = net["layers"][li]
            if layer["type"] == "conv":
                I = O.lwe_conv2d(P, layer["W"], x_img[img], layer["cin"], layer["h"], layer["w"],
                                 layer["stride"], layer["pad"])[nrn:nrn + 1]
            else:
                I = O.lwe_linear(P, layer["W"][nrn:nrn + 1], spk[li - 1][img])
            rows.append((img, nrn, O.lwe_add_const(P, I, p // 2)))
        ref = O.pbs(P, OK, np.concatenate([r[2] for r in rows]), luts, nthreads=NTHREADS)[0]
        for k, (img, nrn, _) in enumerate(rows):
            assert np.array_equal(spk[li][img, nrn], ref[k]), f"layer {li} image {img} neuron {nrn}"
    assert K.status() == fhe.FHE_OK


def test_snn_toy_layer_tc_bit_exact(fhe, oracle_keys):
    """Encrypted LIF layer on the tensor-core path (low-noise ring N=1024)."""
    P, K = gpu_keys(fhe, "T0", 2)
    _, OK = oracle_keys("T0", 2)
    net = synth.toy_lif_net(seed=4)
    net["lif"] = dict(v_th=3, leak_shift=1, spike_scale=1)
    x = synth.bernoulli_spikes(5, 2, 16, 0.3)
    ct = O.encrypt(P, OK, x.reshape(-1), 9).reshape(2, 1, 16, -1)
    try:
        snn = fhe.Snn(K, net, max_images=1, variant=fhe.VARIANT_TC, use_graph=True)
    except fhe.FheError as e:
        if e.code == fhe.FHE_EUNSUPPORTED:
            pytest.skip("TC variant does not cover this parameter set")
        raise
    scores = torch.empty((1, 32, P["n"] + 1), dtype=torch.int32, device="cuda")
    snn.infer(torch.from_numpy(ct.view(np.int32)).cuda(), 1, scores)
    ref = O.snn_encrypted(P, OK, net, ct[:, 0], nthreads=NTHREADS)
    assert np.array_equal(u32(scores)[0], ref["scores"])


@pytest.mark.parametrize("name,count", [("P630", 389), ("P750", 257)])
def test_fft_variant_decrypts_like_exact(fhe, oracle_keys, name, count):
    """FP64 FFT blind rotation (not bit-exact by design): every output decrypts
    to the exact path's message; most outputs are even bit-identical (the
    rounded doubles hit the exact integers); the rounding-error report is set."""
    P, K = gpu_keys(fhe, name, 3)
    _, OK = oracle_keys(name, 3)
    p = 1 << P["log2_p"]
    m = synth.uniform_messages(43, count, p)
    ct = fhe.encrypt(K, m, seed=17)
    for L in (1, 2):
        luts = _luts(P, L)
        lut = fhe.lut_create(K, luts)
        ref = u32(fhe.pbs_batch(K, ct, lut, fhe.VARIANT_EXACT))
        K.fft_max_error(reset=True)
        got = u32(pbs(fhe, K, ct, lut, "FFT"))
        err = K.fft_max_error()
        assert 0.0 < err < 0.5
        for j in range(L):
            assert np.array_equal(O.decrypt(P, OK, got[j]), O.decrypt(P, OK, ref[j]))
        assert np.mean(np.all(got == ref, axis=-1)) > 0.9


def test_snn_toy_layer_fft_decrypts_like_plain(fhe, oracle_keys):
    """Encrypted LIF layer on the FFT path: decrypted spike counts equal the
    plaintext network (low-noise ring N=1024)."""
    P, K = gpu_keys(fhe, "T0", 2)
    _, OK = oracle_keys("T0", 2)
    net = synth.toy_lif_net(seed=4)
    net["lif"] = dict(v_th=3, leak_shift=1, spike_scale=1)
    x = synth.bernoulli_spikes(5, 2, 16, 0.3)
    ct = O.encrypt(P, OK, x.reshape(-1), 9).reshape(2, 1, 16, -1)
    snn = fhe.Snn(K, net, max_images=1, variant=fhe.VARIANT_FFT, use_graph=True)
    scores = torch.empty((1, 32, P["n"] + 1), dtype=torch.int32, device="cuda")
    snn.infer(torch.from_numpy(ct.view(np.int32)).cuda(), 1, scores)
    plain = O.snn_plain(P, net, x)
    assert np.array_equal(O.decrypt(P, OK, u32(scores)[0]), plain["scores"])


@pytest.mark.parametrize("name", ["P630", "P64"])
def test_autotuned_variant_is_bit_exact(fhe, oracle_keys, name):
    """FHE_VARIANT_AUTO picks the CUDA-core or tensor-core blind rotation by
    batch size (crossover measured by fhe_pbs_autotune); on both sides of the
    crossover the outputs equal the CUDA-core path's bit for bit.  The tuner
    also times the two tile shapes of the tensor-core path (clusters of 4 or
    8 SMs per 256-ciphertext tile) and reports the limit it keeps.  P64 has no
    tensor-core path: the tuner reports none and AUTO stays on CUDA cores."""
    P, K = gpu_keys(fhe, name, 3)
    p = 1 << P["log2_p"]
    cross = K.autotune()
    tuned, cl8_tiles, cl16_tiles, split_tiles = K.tuning()
    assert tuned == cross
    if name == "P64":
        assert cross is None
    else:
        assert cross is not None and 1 <= cross <= 8192
        assert 0 <= cl8_tiles <= 152 // 8
        assert 0 <= cl16_tiles <= 152 // 16
        assert 0 <= split_tiles <= 152 // 32
        print("autotune %s: tensor cores from %d ciphertexts, clusters of 8 up to %d tiles, "
              "of 16 up to %d tiles, two clusters of 16 per tile up to %d tiles"
              % (name, cross, cl8_tiles, cl16_tiles, split_tiles))
    luts = _luts(P, 2)
    lut = fhe.lut_create(K, luts)
    for count in (100, 1500):
        m = synth.uniform_messages(51 + count, count, p)
        ct = fhe.encrypt(K, m, seed=13)
        ref = u32(fhe.pbs_batch(K, ct, lut, fhe.VARIANT_EXACT))
        got = u32(fhe.pbs_batch(K, ct, lut, fhe.VARIANT_AUTO))
        assert np.array_equal(got, ref)
    assert K.status() == fhe.FHE_OK


def test_p750_thousand_bootstraps_match_oracle_hashes(fhe):
    """1000 bootstraps at P750 (N = 2048; keys, messages and encryption from
    seed 4; identity-plus-threshold table) on both integer blind-rotation
    paths: every output ciphertext equals the oracle's, compared through the
    SHA-256 prefixes that tests/golden/make_p750_pbs_hashes.py wrote from the
    oracle alone."""
    import hashlib
    path = os.path.join(os.path.dirname(__file__), "golden", "p750_pbs_1000.txt")
    golden = [l.split()[1] for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(golden) == 1000
    P, K = gpu_keys(fhe, "P750", 4)
    p = 1 << P["log2_p"]
    m = synth.uniform_messages(4, 1000, p)
    ct = fhe.encrypt(K, m, seed=4)
    lut = fhe.lut_create(K, synth.identity_plus_threshold_lut(p)[None])
    for variant in VARIANTS:
        out = u32(pbs(fhe, K, ct, lut, variant))[0]
        got = [hashlib.sha256(np.ascontiguousarray(out[i], dtype="<u4").tobytes()).hexdigest()[:16]
               for i in range(1000)]
        bad = [i for i in range(1000) if got[i] != golden[i]]
        assert not bad, f"{variant}: {len(bad)} outputs differ from the oracle, first {bad[:5]}"
    assert K.status() == fhe.FHE_OK
