"""GPU parity of the replica library (libfhe_dicsnn_replica.so).

Runs with one process per GPU load the library built with FHE_NO_MULTICAST:
its tensor-core blind rotation copies every digit tile into each CTA itself
and commits MMA completion to each CTA's barrier separately, with no
cluster-multicast instruction compiled in.  Its outputs must equal the same
library's CUDA-core path bit for bit (on both cluster shapes and both table
counts), and sampled outputs the oracle's.  The replica library is loaded
through a second instance of the binding, beside the single-GPU library.
"""
import importlib.util
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2309_09025_gb300 import synth

pytestmark = pytest.mark.gpu

NTHREADS = os.cpu_count() or 1
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rfhe():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_09025_gb300 import build
    path = build.build(replica=True)
    spec = importlib.util.spec_from_file_location(
        "fhe_replica_binding", os.path.join(ROOT, "paper_2309_09025_gb300", "fhe.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.use_library(path)
    return mod


def u32(t):
    return t.detach().cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("count", [389, 3999])
def test_replica_tensor_cores_bit_exact(rfhe, oracle_keys, count):
    """389 ciphertexts run on clusters of 8 CTAs, 3999 on clusters of 4."""
    P, OK = oracle_keys("P630", 3)
    K = rfhe.keygen_from_seed(P, 3)
    p = 1 << P["log2_p"]
    m = synth.uniform_messages(61, count, 2 * p)
    ct = rfhe.encrypt(K, m, seed=19)
    for L in (1, 2):
        luts = (synth.identity_plus_threshold_lut(p)[None] if L == 1
                else O.lif_luts(P, v_th=8, leak_shift=1, spike_scale=1))
        lut = rfhe.lut_create(K, luts)
        ref = u32(rfhe.pbs_batch(K, ct, lut, rfhe.VARIANT_EXACT))
        got = u32(rfhe.pbs_batch(K, ct, lut, rfhe.VARIANT_TC))
        assert np.array_equal(got, ref), f"L={L}: tensor-core outputs differ from CUDA cores"
        idx = np.array([0, 255, 256, count - 1])
        assert np.array_equal(got[:, idx], O.pbs(P, OK, u32(ct)[idx], luts, nthreads=NTHREADS))
    assert K.status() == rfhe.FHE_OK
