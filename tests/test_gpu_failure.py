"""Failure detection on the GPU without a fault: a bounded device wait that
nothing completes gives up after a short limit and reports FHE_ETIMEOUT
through the status word; the context stays usable afterwards."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fhe():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_09025_gb300 import build, fhe as F
    build.build()
    return F


def test_bounded_wait_reports_timeout_and_context_survives(fhe):
    from paper_2309_09025_gb300 import synth
    P = dict(synth.P64)
    keys = fhe.keygen_from_seed(P, seed=31)
    assert keys.status() == fhe.FHE_OK
    assert keys.selftest_timeout(20000) == fhe.FHE_ETIMEOUT
    assert keys.status() == fhe.FHE_OK  # the status word was cleared by the read
    # the device still works: a bootstrap after the timeout decrypts correctly
    p = 1 << P["log2_p"]
    lut = fhe.lut_create(keys, synth.identity_plus_threshold_lut(p)[None])
    m = np.arange(p, dtype=np.int32)
    out = fhe.pbs_batch(keys, fhe.encrypt(keys, m, seed=3), lut, fhe.VARIANT_EXACT)
    dec = fhe.decrypt(keys, out[0]).cpu().numpy() % (2 * p)
    assert np.mean(dec == synth.identity_plus_threshold_lut(p)[m]) > 0.8
    assert keys.status() == fhe.FHE_OK


def test_invalid_arguments_are_rejected(fhe):
    from paper_2309_09025_gb300 import synth
    keys = fhe.keygen_from_seed(dict(synth.P64), seed=32)
    assert keys.selftest_timeout(0) == fhe.FHE_EINVAL
    lut = fhe.lut_create(keys, synth.identity_plus_threshold_lut(32)[None])
    with pytest.raises(fhe.FheError) as e:
        fhe.pbs_batch(keys, torch.zeros((4, 65), dtype=torch.int32, device="cuda"), lut, 7)
    assert e.value.code == fhe.FHE_EINVAL
