"""GPU parity of the configuration the benchmark times, at full size.

The benchmark runs the MNIST-shaped conv-SNN (P630: n=630, N=1024, Bg=2^7
l=3, key switch 2^2 x 7, p=64; conv 1->8 5x5 s2 -> FC 1152->128 -> FC 128->10;
T=4) streamed on tensor cores, every neuron-step one multi-value bootstrap with
the LIF table pair (Thm 3.2; Eq. FHE-Fire and Eq. FHE-Reset of 4.2).  Here:

* 1000 bootstraps of that table pair at P630 on inputs spread over all of
  Z_2p, each output ciphertext of both integer blind rotations compared with
  the oracle's (stored SHA-256 prefixes written by the oracle alone);
* the streamed network itself, two batches through all T=4 steps, observed
  one layer-skewed step at a time: sampled neurons of every layer at every
  step are recomputed by the oracle from the GPU's spikes of the layer below
  and its own membranes of the step before (WeightSum, H = V + I, centring,
  bootstrap), and the scores are the sum of the last layer's spikes.
"""
import hashlib
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


def u32(t):
    return t.detach().cpu().numpy().view(np.uint32)


def sha16(row):
    return hashlib.sha256(np.ascontiguousarray(row, dtype="<u4").tobytes()).hexdigest()[:16]


@pytest.mark.parametrize("variant", ["EXACT", "TC"])
def test_p630_lif_thousand_bootstraps_match_oracle_hashes(fhe, variant):
    """1000 multi-value bootstraps at P630 with the LIF pair (V_th 8, leak
    >>1, spike 1), messages uniform in Z_128 (both halves of the test
    polynomial), keys seed 2, messages and encryption seed 6: every output
    ciphertext of both tables equals the oracle's, compared through the
    SHA-256 prefixes tests/golden/make_p630_lif_pbs_hashes.py wrote."""
    path = os.path.join(os.path.dirname(__file__), "golden", "p630_lif_pbs_1000.txt")
    golden = [l.split()[1:] for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(golden) == 1000 and all(len(g) == 2 for g in golden)
    P = dict(synth.P630)
    p = 1 << P["log2_p"]
    K = fhe.keygen_from_seed(P, 2)
    m = synth.uniform_messages(6, 1000, 2 * p)
    ct = fhe.encrypt(K, m, seed=6)
    lif = synth.LIF_DEFAULT
    lut = fhe.lut_create(K, O.lif_luts(P, lif["v_th"], lif["leak_shift"], lif["spike_scale"]))
    out = u32(fhe.pbs_batch(K, ct, lut, getattr(fhe, "VARIANT_" + variant)))
    bad = [(j, i) for i in range(1000) for j in range(2) if sha16(out[j, i]) != golden[i][j]]
    assert not bad, f"{variant}: {len(bad)} outputs differ from the oracle, first {bad[:5]}"
    assert K.status() == fhe.FHE_OK


def test_streamed_csnn_t4_full_size_every_step(fhe, oracle_keys):
    """The bench's network and schedule at full size on tensor cores: three
    batches of 2 images pushed into one stream (each batch's first steps
    share bootstrap launches with the previous batch's deeper layers), all
    T = 4 steps of all three layers checked neuron by neuron on a sample,
    through fhe_snn_stream_stage / fhe_snn_stream_iterate, the same
    iteration code as fhe_snn_stream_push.  As in the bench, the iterations
    with every layer active run as CUDA graphs, one per residue of the step
    mod 8: the third batch's iterations replay graphs captured during the
    first two."""
    P, OK = oracle_keys("P630", 3)
    K = fhe.keygen_from_seed(P, 3)
    W = P["n"] + 1
    p = 1 << P["log2_p"]
    T, B, NB = 4, 2, 3
    net = synth.csnn_net(T=T)
    sizes = [1152, 128, 10]
    nl = len(sizes)
    imgs = synth.stroke_images(5, B * NB).reshape(NB, B, -1)
    cts = [fhe.encrypt(K, imgs[b].reshape(-1), seed=11 + b).view(B, 28 * 28, W) for b in range(NB)]
    snn = fhe.Snn(K, net, max_images=B, variant=fhe.VARIANT_TC, use_graph=True)
    scores = [torch.empty((B, 10, W), dtype=torch.int32, device="cuda") for _ in range(NB)]

    def snap(batches):
        """Spikes and membranes of every layer of the batches in flight."""
        st = {}
        for b in batches:
            for l in range(nl):
                for kind in (fhe.STATE_SPIKES, fhe.STATE_MEMBRANES):
                    t = torch.empty((B, sizes[l], W), dtype=torch.int32, device="cuda")
                    snn.stream_state(b, l, kind, t)
                    st[(b, l, kind)] = t
        torch.cuda.synchronize()
        return {k: u32(v) for k, v in st.items()}

    # run the stream step by step, keeping the state before and after each step
    states = []  # (step j, batches staged, state before, state after)
    j, staged = 0, 0
    while True:
        if staged < NB and j == staged * T:
            snn.stream_stage(cts[staged], B, scores[staged])
            staged += 1
        in_flight = [b for b in range(staged) if staged <= b + 2]
        before = snap(in_flight) if j > 0 else {}
        left = snn.stream_iterate()
        after = snap(in_flight)
        states.append((j, in_flight, before, after))
        j += 1
        if left == 0 and staged == NB:
            break
    assert j == NB * T + nl - 1
    snn.stream_flush()
    torch.cuda.synchronize()

    luts = O.lif_luts(P, **net["lif"])
    conv = net["layers"][0]
    x_img = [u32(c) for c in cts]
    # oracle bootstrap inputs of the sampled neurons, then one oracle batch
    items, H_in = [], []
    last_spikes = {}
    for j, in_flight, before, after in states:
        for l in range(nl):
            if j < l or (j - l) // T >= NB:
                continue
            b, t = (j - l) // T, (j - l) % T
            assert b in in_flight
            for k in range(2):
                img = (j + k) % B
                nrn = (97 * (j + 1) + 31 * k + 13 * l) % sizes[l]
                if l == 0:
                    I = O.lwe_conv2d(P, conv["W"], x_img[b][img], conv["cin"], conv["h"], conv["w"],
                                     conv["stride"], conv["pad"])[nrn:nrn + 1]
                else:
                    x = before[(b, l - 1, fhe.STATE_SPIKES)][img]
                    I = O.lwe_linear(P, net["layers"][l]["W"][nrn:nrn + 1], x)
                if t > 0:
                    V = before[(b, l, fhe.STATE_MEMBRANES)][img, nrn:nrn + 1]
                    I = (I.astype(np.uint64) + V).astype(np.uint32)
                H_in.append(O.lwe_add_const(P, I, p // 2))
                items.append((j, l, b, t, img, nrn))
            if l == nl - 1:
                last_spikes[(b, t)] = after[(b, l, fhe.STATE_SPIKES)]
    ref = O.pbs(P, OK, np.concatenate(H_in), luts, nthreads=NTHREADS)
    by_step = {j: after for j, _, _, after in states}
    for k, (j, l, b, t, img, nrn) in enumerate(items):
        after = by_step[j]
        what = f"step {j} layer {l} batch {b} t {t} image {img} neuron {nrn}"
        assert np.array_equal(after[(b, l, fhe.STATE_SPIKES)][img, nrn], ref[0, k]), "spike " + what
        assert np.array_equal(after[(b, l, fhe.STATE_MEMBRANES)][img, nrn], ref[1, k]), "membrane " + what
    # scores = the last layer's spikes summed over the T steps (5.3)
    for b in range(NB):
        s = sum(last_spikes[(b, t)].astype(np.uint64) for t in range(T)) % (1 << 32)
        assert np.array_equal(u32(scores[b]), s.astype(np.uint32)), f"scores of batch {b}"
    assert K.status() == fhe.FHE_OK
