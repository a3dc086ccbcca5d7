"""Python face of the CPU oracle (TEST INFRASTRUCTURE ONLY).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may import
this module.  It never imports the product package (paper_2309_09025_gb300) and
the product package never imports it.  Parameters are passed as plain dicts
with the keys of ``PARAM_KEYS``.

The TFHE primitives are the plain C functions of tfhe_oracle.c (schoolbook,
integer exact); the spiking-network compositions below follow the paper's
equations directly:

* plaintext DiCSNN (Thm 3.2, Eq. DiscretEquation) in Z_{2p} with the same wrap
  semantics as the ciphertext path;
* encrypted DiCSNN (4.1 WeightSum, 4.2 FHE-Fire / FHE-Reset, 5.3 protocol).
"""
import ctypes
import os

import numpy as np

from . import build_oracle

PARAM_KEYS = ("n", "k", "N", "log2_bg", "l", "log2_bks", "l_ks", "log2_p",
              "lwe_noise_log2", "glwe_noise_log2")


class _Params(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint32) for k in PARAM_KEYS[:8]] + [
        ("lwe_noise_log2", ctypes.c_int32), ("glwe_noise_log2", ctypes.c_int32)]


_lib = None


def lib():
    """Load (building if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = build_oracle.build()
        L = ctypes.CDLL(path)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        i32p = ctypes.POINTER(ctypes.c_int32)
        pp = ctypes.POINTER(_Params)
        u64, u32, i32 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32
        sig = {
            "orc_splitmix_out": (u64, [u64, u64]),
            "orc_draw": (u64, [u64, u32, u64]),
            "orc_noise": (u32, [u64, u32, u64, i32]),
            "orc_negacyclic_mul": (None, [u32p, u32p, u32, u32p]),
            "orc_poly_rotate": (None, [u32p, u32, u32, u32p]),
            "orc_decompose": (None, [u32, u32, u32, i32p]),
            "orc_mod_switch": (u32, [u32, u32]),
            "orc_keygen": (None, [pp, u64, u32p, u32p, u32p, u32p]),
            "orc_encrypt": (None, [pp, u32p, i32p, u64, u64, u32p]),
            "orc_phase": (None, [u32, u32p, u32p, u64, u32p]),
            "orc_decrypt": (None, [pp, u32p, u32p, u64, i32p]),
            "orc_glwe_phase": (None, [pp, u32p, u32p, u32p]),
            "orc_lut_coeffs": (None, [pp, i32p, i32p]),
            "orc_test_poly": (None, [pp, i32p, u32p]),
            "orc_external_product": (None, [pp, u32p, u32p, u32p]),
            "orc_blind_rotate": (None, [pp, u32p, u32p, u32p, u32p]),
            "orc_sample_extract": (None, [pp, u32p, u32p]),
            "orc_key_switch": (None, [pp, u32p, u32p, u32p]),
            "orc_pbs": (None, [pp, u32p, u32p, u32p, i32p, u32, u32p]),
            "orc_pbs_batch": (None, [pp, u32p, u32p, u32p, u64, i32p, u32, u32p, u32p,
                                     ctypes.c_int]),
            "orc_lwe_linear": (None, [u32, u32, i32p, u64, u64, i32p, u32p, u32p]),
            "orc_lwe_conv2d": (None, [u32, u32, u32, u32, u32, u32, u32, u32, u32, u32,
                                      i32p, i32p, u32p, u32p]),
            "orc_lwe_add_const": (None, [u32, u32, u32p, u64, i32]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _p(P):
    return ctypes.byref(_Params(*[int(P[k]) for k in PARAM_KEYS]))


def _u32(a):
    a = np.ascontiguousarray(a, dtype=np.uint32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _null_i32():
    return ctypes.POINTER(ctypes.c_int32)()


def delta(P):
    """Delta = q / (2p): one padding bit above the message (2.1, Fig. ZP)."""
    return 1 << (31 - P["log2_p"])


# ---------------------------------------------------------------- randomness
def splitmix_out(state, i):
    return int(lib().orc_splitmix_out(state, i))


def draw(seed, domain, index):
    return int(lib().orc_draw(seed, domain, index))


def noise(seed, domain, index, noise_log2):
    return int(lib().orc_noise(seed, domain, index, noise_log2))


# ---------------------------------------------------------------- ring ops
def negacyclic_mul(a, b):
    a, pa = _u32(a)
    b, pb = _u32(b)
    out = np.zeros(a.shape[0], np.uint32)
    _, po = _u32(out)
    lib().orc_negacyclic_mul(pa, pb, a.shape[0], po)
    return out


def poly_rotate(P_, e):
    P_, pp = _u32(P_)
    out = np.zeros_like(P_)
    lib().orc_poly_rotate(pp, P_.shape[0], e, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    return out


def decompose(x, log2_base, levels):
    d = np.zeros(levels, np.int32)
    lib().orc_decompose(int(x) & 0xFFFFFFFF, log2_base, levels,
                        d.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return d


def mod_switch(a, N):
    return int(lib().orc_mod_switch(int(a) & 0xFFFFFFFF, N))


# ---------------------------------------------------------------- keys, LWE
def keygen(P, seed):
    n, k, N, l = P["n"], P["k"], P["N"], P["l"]
    s = np.zeros(n, np.uint32)
    S = np.zeros(k * N, np.uint32)
    bsk = np.zeros(n * (k + 1) * l * (k + 1) * N, np.uint32)
    ksk = np.zeros(k * N * P["l_ks"] * (n + 1), np.uint32)
    lib().orc_keygen(_p(P), seed, _u32(s)[1], _u32(S)[1], _u32(bsk)[1], _u32(ksk)[1])
    return {"lwe_key": s, "glwe_key": S, "bsk": bsk, "ksk": ksk}


def encrypt(P, keys, msgs, seed):
    msgs, pm = _i32(np.asarray(msgs).reshape(-1))
    ct = np.zeros((msgs.shape[0], P["n"] + 1), np.uint32)
    lib().orc_encrypt(_p(P), _u32(keys["lwe_key"])[1], pm, msgs.shape[0], seed, _u32(ct)[1])
    return ct


def phase(P, keys, ct):
    ct, pc = _u32(np.asarray(ct).reshape(-1, P["n"] + 1))
    out = np.zeros(ct.shape[0], np.uint32)
    lib().orc_phase(P["n"], _u32(keys["lwe_key"])[1], pc, ct.shape[0], _u32(out)[1])
    return out


def decrypt(P, keys, ct):
    ct, pc = _u32(np.asarray(ct).reshape(-1, P["n"] + 1))
    out = np.zeros(ct.shape[0], np.int32)
    lib().orc_decrypt(_p(P), _u32(keys["lwe_key"])[1], pc, ct.shape[0], _i32(out)[1])
    return out


def glwe_phase(P, keys, glwe):
    glwe, pg = _u32(glwe)
    out = np.zeros(P["N"], np.uint32)
    lib().orc_glwe_phase(_p(P), _u32(keys["glwe_key"])[1], pg, _u32(out)[1])
    return out


# ---------------------------------------------------------------- bootstrapping
def lut_coeffs(P, f):
    f, pf = _i32(f)
    out = np.zeros(P["N"], np.int32)
    lib().orc_lut_coeffs(_p(P), pf, _i32(out)[1])
    return out


def test_poly(P, f):
    f, pf = _i32(f)
    out = np.zeros(P["N"], np.uint32)
    lib().orc_test_poly(_p(P), pf, _u32(out)[1])
    return out


def external_product(P, ggsw, glwe):
    out = np.zeros((P["k"] + 1) * P["N"], np.uint32)
    lib().orc_external_product(_p(P), _u32(ggsw)[1], _u32(glwe)[1], _u32(out)[1])
    return out


def blind_rotate(P, keys, ct, tv):
    acc = np.zeros((P["k"] + 1) * P["N"], np.uint32)
    lib().orc_blind_rotate(_p(P), _u32(keys["bsk"])[1], _u32(ct)[1], _u32(tv)[1], _u32(acc)[1])
    return acc


def sample_extract(P, acc):
    out = np.zeros(P["k"] * P["N"] + 1, np.uint32)
    lib().orc_sample_extract(_p(P), _u32(acc)[1], _u32(out)[1])
    return out


def key_switch(P, keys, big):
    out = np.zeros(P["n"] + 1, np.uint32)
    lib().orc_key_switch(_p(P), _u32(keys["ksk"])[1], _u32(big)[1], _u32(out)[1])
    return out


def pbs(P, keys, ct, luts, nthreads=None, log2_p_out=None):
    """Batched bootstrapping; luts is (L, p) with p = 2^P['log2_p'], the
    input's message space; table j is written with Delta = 2^(31 -
    log2_p_out[j]) (default: the input's space).  Returns (L, count, n+1)."""
    luts, pl = _i32(np.asarray(luts).reshape(-1, 1 << P["log2_p"]))
    L = luts.shape[0]
    ct, pc = _u32(np.asarray(ct).reshape(-1, P["n"] + 1))
    count = ct.shape[0]
    out = np.zeros((L, count, P["n"] + 1), np.uint32)
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    po = ctypes.POINTER(ctypes.c_uint32)()
    if log2_p_out is not None:
        lp = np.asarray(log2_p_out, np.uint32).reshape(-1)
        assert lp.shape[0] == L and lp.min() >= 1 and lp.max() <= 30
        lp, po = _u32(lp)
    lib().orc_pbs_batch(_p(P), _u32(keys["bsk"])[1], _u32(keys["ksk"])[1], pc, count, pl, L,
                        po, _u32(out)[1], int(nthreads))
    return out


# ---------------------------------------------------------------- WeightSum
def lwe_linear(P, W, ct_in, bias=None):
    W, pw = _i32(W)
    M, K = W.shape
    ct_in, pc = _u32(np.asarray(ct_in).reshape(K, P["n"] + 1))
    out = np.zeros((M, P["n"] + 1), np.uint32)
    pb = _i32(bias)[1] if bias is not None else _null_i32()
    lib().orc_lwe_linear(P["n"], P["log2_p"], pw, M, K, pb, pc, _u32(out)[1])
    return out


def conv_out_hw(h, w, kh, kw, stride, pad):
    return (h + 2 * pad - kh) // stride + 1, (w + 2 * pad - kw) // stride + 1


def lwe_conv2d(P, W, ct_in, cin, h, w, stride, pad, bias=None):
    W, pw = _i32(W)
    cout, cin_, kh, kw = W.shape
    assert cin_ == cin
    ho, wo = conv_out_hw(h, w, kh, kw, stride, pad)
    ct_in, pc = _u32(np.asarray(ct_in).reshape(cin * h * w, P["n"] + 1))
    out = np.zeros((cout * ho * wo, P["n"] + 1), np.uint32)
    pb = _i32(bias)[1] if bias is not None else _null_i32()
    lib().orc_lwe_conv2d(P["n"], P["log2_p"], cin, h, w, cout, kh, kw, stride, pad, pw, pb, pc,
                         _u32(out)[1])
    return out


def lwe_add_const(P, ct, value):
    ct = np.ascontiguousarray(ct, dtype=np.uint32).copy()
    lib().orc_lwe_add_const(P["n"], P["log2_p"], _u32(ct)[1], ct.size // (P["n"] + 1), int(value))
    return ct


def lwe_add_consts(P, ct, values):
    """Trivial plaintext addition, one message per ciphertext: b_i += m_i * Delta
    (mod 2^32), a unchanged (2.1: LWE is additively homomorphic)."""
    w = P["n"] + 1
    ct = np.array(ct, dtype=np.uint32, copy=True).reshape(-1, w)
    m = (np.asarray(values, np.int64).reshape(-1) % (1 << 32)).astype(np.uint64)
    b = (ct[:, -1].astype(np.uint64) + m * np.uint64(delta(P))) % np.uint64(1 << 32)
    ct[:, -1] = b.astype(np.uint32)
    return ct


# ---------------------------------------------------------------- LIF (4.2)
def lif_luts(P, v_th, leak_shift, spike_scale):
    """FHE-Fire and FHE-Reset program functions as LUTs over u in [0, p).

    The bootstrap input is centred: u = H + p/2, so v = u - p/2 is the signed
    membrane value H in [-p/2, p/2).  Fire (Eq. FHE-Fire, with the tie read as
    firing, Thm 3.2 '>='): spike_scale * [v >= V_th].  Reset (Eq. FHE-Reset /
    Thm 3.2): 0 if v >= V_th, leak(v) if 0 <= v < V_th, 0 if v < 0, with
    leak(v) = floor(v / 2^leak_shift) (leak_shift = 0 is the IF model).
    """
    p = 1 << P["log2_p"]
    v = np.arange(p, dtype=np.int64) - p // 2
    fire = np.where(v >= v_th, spike_scale, 0)
    reset = np.where(v >= v_th, 0, np.where(v >= 0, v >> leak_shift, 0))
    return np.stack([fire, reset]).astype(np.int32)


def lif_luts_two_pbs(P, v_th, leak_shift):
    """The paper's two program functions for separate bootstraps (4.2), as
    tables over u in [0, p); the bootstrap's negacyclic half gives -g(u) for
    messages in [-p, 0) (the paper's plaintext modulus is 2p here, with
    Delta = q / 2p, so g(v + p) = -g(v) holds by construction).

    Sign (Eq. FHE-Fire): g = 1, so bootstrap(H - V_th) + 1 = 2 Spike.
    Reset (Eq. FHE-Reset): 0 for u >= V_th, leak(u) for 0 <= u < V_th.
    """
    p = 1 << P["log2_p"]
    u = np.arange(p, dtype=np.int64)
    sign = np.ones(p, np.int64)
    reset = np.where(u >= v_th, 0, u >> leak_shift)
    return np.stack([sign, reset]).astype(np.int32)


def poisson_spikes(x, M_t, spike):
    """Poisson encoding (2.3, Eq. Poisson-coding): a spike of value `spike`
    where the pixel exceeds the step's random value, none where it does not."""
    return np.where(np.asarray(x, np.int64) > np.asarray(M_t, np.int64), spike, 0)


def wrap2p(x, p):
    """Signed representative in [-p, p) of x mod 2p."""
    x = np.asarray(x, dtype=np.int64)
    return ((x + p) % (2 * p)) - p


def plain_bootstrap(f, v, p, centre=True, p_out=None):
    """What a bootstrap of a message v (mod 2p, centred by +p/2 unless
    centre is False) decrypts to, read in the output space p_out (default p).

    u = (v + p/2) mod 2p; f(u) for u < p, -f(u - p) otherwise (negacyclic half,
    Thm 2.1), reduced mod 2 p_out.
    """
    u = (np.asarray(v, dtype=np.int64) + (p // 2 if centre else 0)) % (2 * p)
    f = np.asarray(f, dtype=np.int64)
    out = np.where(u < p, f[np.minimum(u, p - 1)], -f[np.maximum(u - p, 0)])
    return wrap2p(out, p if p_out is None else p_out)


def layer_spaces(P, net):
    """log2 of each layer's message space p_l (the dynamic message space of
    DiNN carried over in 5.2): layer['log2_p'] where given, else the key's
    P['log2_p'].  Layer l's currents, membranes and bootstrap boxes live in
    Z_{2 p_l}; its spikes are written in the space of the layer that reads
    them (the key's space for the last layer, whose spikes form the
    scores).  The network input is encrypted in the key's space, so a
    WeightSum first layer needs p_0 <= p (its weights are multiplied by
    p / p_0 in the ciphertext domain); a Poisson first layer compares pixels
    in the key's space itself.  Only the multi-value mode changes spaces."""
    lps = [int(layer.get("log2_p", P["log2_p"])) for layer in net["layers"]]
    for li, (layer, lp) in enumerate(zip(net["layers"], lps)):
        if not 1 <= lp or (2 << lp) > P["N"]:
            raise ValueError("layer %d: message space 2^%d does not fit N" % (li, lp))
        if li == 0 and (lp > P["log2_p"] or (layer["type"] == "poisson" and lp != P["log2_p"])):
            raise ValueError("first layer: message space must not exceed the input's")
    if net.get("lif_mode") == "two_pbs" and any(lp != P["log2_p"] for lp in lps):
        raise ValueError("the two-bootstrap mode keeps the key's message space")
    return lps


def _plain_layer(layer, x):
    x = np.asarray(x, dtype=np.int64)
    if layer["type"] == "fc":
        y = np.asarray(layer["W"], np.int64) @ x
    else:
        W = np.asarray(layer["W"], np.int64)
        cout, cin, kh, kw = W.shape
        h, w, s, pad = layer["h"], layer["w"], layer["stride"], layer["pad"]
        ho, wo = conv_out_hw(h, w, kh, kw, s, pad)
        xi = np.zeros((cin, h + 2 * pad, w + 2 * pad), np.int64)
        xi[:, pad:pad + h, pad:pad + w] = x.reshape(cin, h, w)
        y = np.zeros((cout, ho, wo), np.int64)
        for oy in range(ho):
            for ox in range(wo):
                patch = xi[:, oy * s:oy * s + kh, ox * s:ox * s + kw]
                y[:, oy, ox] = np.tensordot(W, patch, axes=([1, 2, 3], [0, 1, 2]))
        y = y.reshape(-1)
    if layer.get("bias") is not None:
        y = y + np.asarray(layer["bias"], np.int64)
    return y


def snn_plain(P, net, inputs):
    """Plaintext DiCSNN (Thm 3.2) with Z_{2p} wrap semantics.

    inputs: (T, n_in) per-step inputs, or (n_in,) when net['static_input'].
    Returns dict(spikes=[per layer (T, size)], h=[per layer (T, size)],
    scores=(n_out,)).  H[t] = V[t-1] + I[t]; S = Fire(H); V = Reset(H);
    scores = sum_t S_last[t] (5.3, step 4).

    net['lif_mode'] = 'two_pbs' evaluates the paper's separate negacyclic
    bootstraps (4.2): S = sign(H - V_th) + 1, V = g(H) without centring.  A
    'poisson' first layer (2.3) spikes where the pixel exceeds M[t]; its 'h'
    entry is x - M[t].  Layers with their own message space (layer_spaces)
    wrap their currents and membranes mod 2 p_l and write their spikes mod
    2 p of the reading layer.
    """
    p = 1 << P["log2_p"]
    T = net["T"]
    lif = net["lif"]
    two = net.get("lif_mode") == "two_pbs"
    lps = layer_spaces(P, net)
    nl = len(net["layers"])
    # p_l of each layer and the space its spikes are written in
    pl = [1 << lp for lp in lps]
    pn = [1 << (lps[li + 1] if li + 1 < nl else P["log2_p"]) for li in range(nl)]
    f = [lif_luts(dict(P, log2_p=lp), lif["v_th"], lif["leak_shift"], lif["spike_scale"])
         for lp in lps]
    g = lif_luts_two_pbs(P, lif["v_th"], lif["leak_shift"])
    V = [None] * nl
    spikes = [[] for _ in net["layers"]]
    hs = [[] for _ in net["layers"]]
    static_I0 = None
    for t in range(T):
        x = inputs if net.get("static_input") else inputs[t]
        for li, layer in enumerate(net["layers"]):
            if layer["type"] == "poisson":
                S = wrap2p(poisson_spikes(x, layer["M"][t], 2 if two else lif["spike_scale"]),
                           pn[li])
                spikes[li].append(S)
                hs[li].append(np.asarray(x, np.int64) - np.asarray(layer["M"][t], np.int64))
                x = S
                continue
            if li == 0 and net.get("static_input"):
                if static_I0 is None:
                    static_I0 = wrap2p(_plain_layer(layer, x), pl[li])
                I = static_I0
            else:
                I = wrap2p(_plain_layer(layer, x), pl[li])
            if V[li] is None:
                V[li] = np.zeros_like(I)
            H = wrap2p(V[li] + I, pl[li])
            if two:
                S = wrap2p(plain_bootstrap(g[0], H - lif["v_th"], p, centre=False) + 1, p)
                V[li] = plain_bootstrap(g[1], H, p, centre=False)
            else:
                S = plain_bootstrap(f[li][0], H, pl[li], p_out=pn[li])
                V[li] = plain_bootstrap(f[li][1], H, pl[li])
            spikes[li].append(S)
            hs[li].append(H)
            x = S
    scores = wrap2p(np.sum(np.stack(spikes[-1]), axis=0), p)
    return {"spikes": [np.stack(s) for s in spikes], "h": [np.stack(h) for h in hs],
            "scores": scores}


def snn_encrypted(P, keys, net, ct_inputs, nthreads=None):
    """Encrypted DiCSNN (4.1 WeightSum + 4.2 FHE-Fire/FHE-Reset, 5.3 flow).

    ct_inputs: (T, n_in, n+1) or (n_in, n+1) when static.  Per layer and step:
    I = WeightSum(x); H = V + I; (S, V) = bootstrap(H + p/2) with the two LIF
    LUTs (one blind rotation, multi-value); the last layer's spikes are summed
    into the encrypted scores.  With net['lif_mode'] = 'two_pbs':
    S = bootstrap(H - V_th; sign) + 1 and V = bootstrap(H; g), no centring
    (4.2).  A 'poisson' first layer bootstraps the comparison x > M[t] (2.3):
    the Fire table on x - M[t] + V_th - 1 (multi-value; its Reset output is
    not used) or the sign table on x - M[t] - 1, plus 1 (two bootstraps).
    Per-layer message spaces (layer_spaces): layer l centres by p_l/2, reads
    with p_l boxes and writes Fire in the reading layer's space, Reset in its
    own.  Returns dict(spikes=[per layer (T, size, n+1)], scores=(n_out, n+1)).
    """
    p = 1 << P["log2_p"]
    w = P["n"] + 1
    T = net["T"]
    lif = net["lif"]
    two = net.get("lif_mode") == "two_pbs"
    lps = layer_spaces(P, net)
    nl = len(net["layers"])
    lpn = [lps[li + 1] if li + 1 < nl else P["log2_p"] for li in range(nl)]
    Pl = [dict(P, log2_p=lp) for lp in lps]
    luts = [lif_luts(Q, lif["v_th"], lif["leak_shift"], lif["spike_scale"]) for Q in Pl]
    g = lif_luts_two_pbs(P, lif["v_th"], lif["leak_shift"])
    V = [None] * nl
    spikes = [[] for _ in net["layers"]]
    static_I0 = None
    scores = None
    for t in range(T):
        x = ct_inputs if net.get("static_input") else ct_inputs[t]
        for li, layer in enumerate(net["layers"]):
            if layer["type"] == "poisson":
                M = np.asarray(layer["M"][t], np.int64)
                if two:
                    Hf = lwe_add_consts(P, x, -M - 1)
                    S = lwe_add_const(P, pbs(P, keys, Hf, g[0:1], nthreads=nthreads)[0], 1)
                else:
                    Hc = lwe_add_consts(P, x, -M + lif["v_th"] - 1 + p // 2)
                    S = pbs(P, keys, Hc, luts[li], nthreads=nthreads,
                            log2_p_out=[lpn[li], lps[li]])[0]
                spikes[li].append(S)
                x = S
                continue
            # the input's Delta is p / p_0 times smaller than layer 0's
            Wl = np.asarray(layer["W"], np.int64) * (1 << (P["log2_p"] - lps[0]) if li == 0 else 1)
            if li == 0 and net.get("static_input") and static_I0 is not None:
                I = static_I0
            elif layer["type"] == "fc":
                I = lwe_linear(Pl[li], Wl, x, layer.get("bias"))
            else:
                I = lwe_conv2d(Pl[li], Wl, x, layer["cin"], layer["h"], layer["w"],
                               layer["stride"], layer["pad"], layer.get("bias"))
            if li == 0 and net.get("static_input"):
                static_I0 = I
            if V[li] is None:
                V[li] = np.zeros_like(I)
            H = (V[li] + I).astype(np.uint32)
            if two:
                Hf = lwe_add_const(P, H, -lif["v_th"])
                S = lwe_add_const(P, pbs(P, keys, Hf, g[0:1], nthreads=nthreads)[0], 1)
                V[li] = pbs(P, keys, H, g[1:2], nthreads=nthreads)[0]
            else:
                Hc = lwe_add_const(Pl[li], H, (1 << lps[li]) // 2)
                out = pbs(Pl[li], keys, Hc, luts[li], nthreads=nthreads,
                          log2_p_out=[lpn[li], lps[li]])
                S, V[li] = out[0], out[1]
            spikes[li].append(S)
            x = S
        scores = spikes[-1][-1].copy() if scores is None else (scores + spikes[-1][-1]).astype(np.uint32)
    return {"spikes": [np.stack(s) for s in spikes], "scores": scores.reshape(-1, w)}
