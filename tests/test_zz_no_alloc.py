"""fhe_pbs_batch_noalloc: bootstrapping for callers that cannot allocate.

Callers whose device memory is owned by another allocator, or whose serving
loop must not risk an allocation, call fhe_pbs_batch_noalloc; it uses a fixed
scratch array compiled into the library instead of the key handle's
workspace.  Its outputs must equal fhe_pbs_batch's (exact variant) bit for bit,
on consecutive calls that share that array.  This file is self-contained so it
also passes alone in a fresh process.
"""
import ctypes

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


def test_noalloc_matches_pbs_batch_on_consecutive_calls(fhe):
    from paper_2309_09025_gb300 import synth
    P = dict(synth.P64)
    keys = fhe.keygen_from_seed(P, seed=21)
    p = 1 << P["log2_p"]
    v = np.arange(p) - p // 2
    luts = np.stack([(v >= 8).astype(np.int32),
                     np.where(v >= 8, 0, np.where(v >= 0, v >> 1, 0)).astype(np.int32)])
    lut = fhe.lut_create(keys, luts)
    for call, (count, seed) in enumerate([(300, 5), (77, 6)]):
        msgs = synth.uniform_messages(seed, count, 2 * p)
        ct = fhe.encrypt(keys, msgs, seed=100 + seed)
        ref = fhe.pbs_batch(keys, ct, lut, fhe.VARIANT_EXACT)
        got = fhe.pbs_batch_noalloc(keys, ct, lut)
        torch.cuda.synchronize()
        assert got.shape == ref.shape, call
        assert torch.equal(got, ref), "call %d differs from fhe_pbs_batch" % call
    assert keys.status() == fhe.FHE_OK


def test_noalloc_rejects_batches_above_the_scratch_limit(fhe):
    from paper_2309_09025_gb300 import synth
    P = dict(synth.P64)
    keys = fhe.keygen_from_seed(P, seed=22)
    lut = fhe.lut_create(keys, synth.identity_plus_threshold_lut(1 << P["log2_p"])[None])
    limit = fhe.PBS_NOALLOC_MAX_WORDS // (P["k"] * P["N"] + 1)
    ct = torch.zeros((limit + 1, P["n"] + 1), dtype=torch.int32, device="cuda")
    out = torch.empty((1, limit + 1, P["n"] + 1), dtype=torch.int32, device="cuda")
    rc = fhe.lib().fhe_pbs_batch_noalloc(keys.handle, ctypes.c_void_p(ct.data_ptr()), limit + 1,
                                         lut.handle, ctypes.c_void_p(out.data_ptr()),
                                         ctypes.c_void_p(0))
    assert rc == fhe.FHE_EINVAL
    ok = fhe.pbs_batch_noalloc(keys, ct[:limit], lut)
    ref = fhe.pbs_batch(keys, ct[:limit], lut, fhe.VARIANT_EXACT)
    assert torch.equal(ok, ref)


def test_noalloc_at_the_n1024_limit_allocates_nothing(fhe):
    """The documented limit at N = 1024 (511 ciphertexts with two tables, the
    LIF pair of a conv-SNN layer) on two calls in a row, bit-identical to
    fhe_pbs_batch; free device memory is the same after the later calls as
    after the first one (which resolves the array's address), and one
    ciphertext more is rejected."""
    from paper_2309_09025_gb300 import synth
    P = dict(synth.P630)
    keys = fhe.keygen_from_seed(P, seed=23)
    p = 1 << P["log2_p"]
    v = np.arange(p) - p // 2
    luts = np.stack([(v >= 8).astype(np.int32),
                     np.where(v >= 8, 0, np.where(v >= 0, v >> 1, 0)).astype(np.int32)])
    lut = fhe.lut_create(keys, luts)
    limit = fhe.PBS_NOALLOC_MAX_WORDS // (2 * (P["k"] * P["N"] + 1))
    assert limit == 511
    cts, refs, outs = [], [], []
    for seed in (7, 8):
        msgs = synth.uniform_messages(seed, limit, 2 * p)
        ct = fhe.encrypt(keys, msgs, seed=200 + seed)
        cts.append(ct)
        refs.append(fhe.pbs_batch(keys, ct, lut, fhe.VARIANT_EXACT))
        outs.append(torch.empty_like(refs[-1]))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call(i, count=limit):
        return fhe.lib().fhe_pbs_batch_noalloc(keys.handle, ctypes.c_void_p(cts[i].data_ptr()),
                                               count, lut.handle,
                                               ctypes.c_void_p(outs[i].data_ptr()), stream)

    assert call(0) == fhe.FHE_OK  # first call on this device in this test's order
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    assert call(1) == fhe.FHE_OK
    assert call(0) == fhe.FHE_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0, "a call changed the free device memory"
    for i in range(2):
        assert torch.equal(outs[i], refs[i]), "call on input %d differs from fhe_pbs_batch" % i
    big = torch.zeros((limit + 1, P["n"] + 1), dtype=torch.int32, device="cuda")
    rc = fhe.lib().fhe_pbs_batch_noalloc(keys.handle, ctypes.c_void_p(big.data_ptr()), limit + 1,
                                         lut.handle, ctypes.c_void_p(outs[0].data_ptr()), stream)
    assert rc == fhe.FHE_EINVAL
    # 2 * 1025 * 2^63 wraps to 0 in 64 bits: the limit check must not overflow
    rc = fhe.lib().fhe_pbs_batch_noalloc(keys.handle, ctypes.c_void_p(big.data_ptr()), 1 << 63,
                                         lut.handle, ctypes.c_void_p(outs[0].data_ptr()), stream)
    assert rc == fhe.FHE_EINVAL
    assert keys.status() == fhe.FHE_OK
