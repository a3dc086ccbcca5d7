"""GPU tests of two measured workloads.

* FP64 negacyclic-FFT blind rotation against the exact integer path over one
  million bootstraps at P750 (n=750, N=2048, Bg=2^10 l=2, p=64; messages
  uniform in Z_64): no output decrypts differently from the exact path's
  output for the same input (a decryption failure, read as in the design
  notes), and the largest rounding distance of the FFT products stays below
  half a torus step.  The exact side is the tensor-core path, bit-identical
  to the CUDA-core path and to the oracle (other tests).
* Ragged arrivals: one network object serves batches of different sizes
  (uniform in 1..64, one CUDA graph set captured per size and reused when a
  size recurs), each batch's scores bit-exact to the oracle's encrypted
  network on sampled images, on the small ring.
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


def u32(t):
    return t.detach().cpu().numpy().view(np.uint32)


def test_fft_million_bootstraps_no_decryption_failure(fhe):
    P = dict(synth.P750)
    p = 1 << P["log2_p"]
    total, chunk = 1_000_000, 125_000
    K = fhe.keygen_from_seed(P, 4, max_batch=chunk)
    lut = fhe.lut_create(K, synth.identity_plus_threshold_lut(p)[None])
    f = synth.identity_plus_threshold_lut(p).astype(np.int64)
    m_all = synth.uniform_messages(4, total, p)
    K.fft_max_error(reset=True)
    failures = identical = intrinsic = 0
    for c0 in range(0, total, chunk):
        m = m_all[c0:c0 + chunk]
        ct = fhe.encrypt(K, m, seed=1000 + c0 // chunk)
        exact = fhe.pbs_batch(K, ct, lut, fhe.VARIANT_TC)
        fft = fhe.pbs_batch(K, ct, lut, fhe.VARIANT_FFT)
        d_exact = fhe.decrypt(K, exact[0]).cpu().numpy().astype(np.int64)
        d_fft = fhe.decrypt(K, fft[0]).cpu().numpy().astype(np.int64)
        failures += int(np.sum(d_fft != d_exact))
        identical += int(torch.sum(torch.all(fft[0] == exact[0], dim=1)).item())
        want = ((f[m] + p) % (2 * p)) - p
        intrinsic += int(np.sum(d_exact != want))
    err = K.fft_max_error()
    print("FFT vs exact over %d bootstraps at P750: %d decryption failures, %d bit-identical "
          "outputs, %d intrinsic modulus-switch failures (%.3f%%), max rounding distance %.4f"
          % (total, failures, identical, intrinsic, 100.0 * intrinsic / total, err))
    assert failures == 0
    assert 0.0 < err < 0.5
    # the parameter set's own modulus-switch failures, for scale (about 0.4%)
    assert intrinsic < 0.01 * total
    assert K.status() == fhe.FHE_OK


def test_ragged_arrivals_one_network_every_batch_matches_oracle(fhe, oracle_keys):
    """Batch sizes uniform in 1..64 (seed 5; the first size recurs at the
    end, replaying its cached graphs), the conv-SNN topology (conv 1->8 5x5
    s2 -> FC 1152->128 -> FC 128->10) on the small ring (n=64, N=256, p=64),
    T = 2: the first and last image of every batch bit-exact to the oracle,
    and every image of a batch equal to the same image inferred alone."""
    P, OK = oracle_keys("P64", 9, log2_p=6)
    K = fhe.keygen_from_seed(P, 9)
    W = P["n"] + 1
    net = synth.csnn_net(seed=2, T=2)
    sizes = [int(s) for s in synth.rng(5).integers(1, 65, size=5)]
    sizes.append(sizes[0])
    imgs = synth.stroke_images(55, sum(sizes)).reshape(sum(sizes), -1)
    snn = fhe.Snn(K, net, max_images=64, use_graph=True)
    one = fhe.Snn(K, net, max_images=1, use_graph=True)
    start = 0
    for bi, n in enumerate(sizes):
        batch = imgs[start:start + n]
        ct = np.stack([O.encrypt(P, OK, batch[i], 7000 + start + i) for i in range(n)])
        d_ct = torch.from_numpy(ct.view(np.int32)).cuda()
        scores = torch.empty((n, 10, W), dtype=torch.int32, device="cuda")
        snn.infer(d_ct, n, scores)
        got = u32(scores)
        for i in sorted({0, n - 1}):
            ref = O.snn_encrypted(P, OK, net, ct[i], nthreads=NTHREADS)
            assert np.array_equal(got[i], ref["scores"]), f"batch {bi} (size {n}) image {i}"
        for i in range(n):
            alone = torch.empty((1, 10, W), dtype=torch.int32, device="cuda")
            one.infer(d_ct[i:i + 1].contiguous(), 1, alone)
            assert np.array_equal(got[i], u32(alone)[0]), f"batch {bi} image {i} vs alone"
        start += n
    assert K.status() == fhe.FHE_OK
