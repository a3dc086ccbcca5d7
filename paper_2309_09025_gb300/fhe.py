"""Thin Python binding of libfhe_dicsnn.so (argument marshalling only).

Every function maps one-to-one onto an entry point of include/fhe_dicsnn.h and
keeps its name without the ``fhe_`` prefix.  Device buffers are torch CUDA
tensors (int32 tensors carry the uint32 ciphertext words bit for bit); the
current torch stream is passed as the CUDA stream.  All compute runs in the
CUDA library: if it is missing this module raises instead of falling back.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfhe_dicsnn.so")

FHE_OK = 0
FHE_EINVAL = -1
FHE_ENOMEM = -2
FHE_ECUDA = -3
FHE_ETIMEOUT = -4
FHE_EUNSUPPORTED = -5
VARIANT_EXACT = 0
VARIANT_TC = 1
VARIANT_FFT = 2
VARIANT_AUTO = 3
KEY_LWE, KEY_GLWE, KEY_BSK, KEY_KSK = 0, 1, 2, 3
LAYER_FC, LAYER_CONV, LAYER_POISSON = 0, 1, 2
LIF_MULTI_VALUE, LIF_TWO_PBS = 0, 1
SNN_PROFILE = 2
STATE_SPIKES, STATE_MEMBRANES, STATE_CURRENTS = 0, 1, 2
TC_OPT_CLUSTER, TC_OPT_MULTICAST, TC_OPT_L2_HINTS = 0, 1, 2

# Every symbol the header declares (checked by the CPU test-suite).
EXPORTED = (
    "fhe_strerror", "fhe_keygen_from_seed", "fhe_keys_free", "fhe_keys_params",
    "fhe_keys_size", "fhe_keys_export", "fhe_encrypt", "fhe_decrypt", "fhe_lwe_linear",
    "fhe_lwe_conv2d", "fhe_lut_create", "fhe_lut_free", "fhe_pbs_batch", "fhe_status",
    "fhe_snn_create", "fhe_snn_free", "fhe_snn_pbs_per_image", "fhe_snn_infer",
    "fhe_snn_layer_spikes", "fhe_snn_profile", "fhe_kernel_launches",
    "fhe_pbs_batch_noalloc", "fhe_snn_begin", "fhe_snn_step", "fhe_snn_end",
    "fhe_snn_iterations", "fhe_selftest_timeout", "fhe_fft_max_error",
    "fhe_snn_stream_push", "fhe_snn_stream_flush", "fhe_pbs_autotune",
    "fhe_lut_create_spaces", "fhe_pbs_batch_groups", "fhe_pbs_tuning", "fhe_tc_plan_query",
    "fhe_snn_stream_stage", "fhe_snn_stream_iterate", "fhe_snn_stream_state",
    "fhe_pbs_set_tc_option",
)
LUT_MAX_GROUPS = 8
PBS_NOALLOC_MAX_WORDS = 1 << 20


class FheError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s failed: %s (%d)" % (what, strerror(code), code))
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("k", ctypes.c_uint32), ("N", ctypes.c_uint32),
                ("log2_bg", ctypes.c_uint32), ("l", ctypes.c_uint32),
                ("log2_bks", ctypes.c_uint32), ("l_ks", ctypes.c_uint32),
                ("log2_p", ctypes.c_uint32), ("lwe_noise_log2", ctypes.c_int32),
                ("glwe_noise_log2", ctypes.c_int32)]

    @classmethod
    def from_dict(cls, d):
        return cls(*[int(d[f]) for f, _ in cls._fields_])

    def to_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class LayerDesc(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("weights", ctypes.POINTER(ctypes.c_int32)),
                ("in_size", ctypes.c_uint32), ("out_size", ctypes.c_uint32),
                ("cin", ctypes.c_uint32), ("h", ctypes.c_uint32), ("w", ctypes.c_uint32),
                ("cout", ctypes.c_uint32), ("kh", ctypes.c_uint32), ("kw", ctypes.c_uint32),
                ("stride", ctypes.c_uint32), ("pad", ctypes.c_uint32),
                ("log2_p", ctypes.c_uint32)]


class TcPlan(ctypes.Structure):
    _fields_ = [("available", ctypes.c_int32), ("key_rows", ctypes.c_uint32),
                ("digit_rows", ctypes.c_uint32), ("sub_shift", ctypes.c_uint32),
                ("max_digit", ctypes.c_uint32), ("chunk_rows", ctypes.c_uint32),
                ("max_partial", ctypes.c_uint64)]


class SnnDesc(ctypes.Structure):
    _fields_ = [("n_layers", ctypes.c_uint32), ("layers", ctypes.POINTER(LayerDesc)),
                ("v_th", ctypes.c_int32), ("leak_shift", ctypes.c_int32),
                ("spike_scale", ctypes.c_int32), ("T", ctypes.c_uint32),
                ("static_input", ctypes.c_int32), ("max_images", ctypes.c_uint32),
                ("variant", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("lif_mode", ctypes.c_int32)]


_lib = None
_lib_path = None


def use_library(path):
    """Select the library file before its first use: the replica build
    (libfhe_dicsnn_replica.so, no cluster-multicast copies) for runs with one
    process per GPU.  The environment variable FHE_DICSNN_LIB does the same."""
    global _lib_path
    if _lib is not None and os.path.abspath(path) != os.path.abspath(_lib_path):
        raise RuntimeError("the CUDA library is already loaded from " + _lib_path)
    _lib_path = path


def lib():
    """Load the CUDA library (no fallback: raises if it was not built)."""
    global _lib, _lib_path
    if _lib is None:
        if _lib_path is None:
            _lib_path = os.environ.get("FHE_DICSNN_LIB") or LIB_PATH
        if not os.path.exists(_lib_path):
            raise RuntimeError("%s is missing: run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`" % _lib_path)
        L = ctypes.CDLL(_lib_path)
        vp, sz, u32, u64, i32 = (ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32,
                                 ctypes.c_uint64, ctypes.c_int32)
        sig = {
            "fhe_strerror": (ctypes.c_char_p, [ctypes.c_int]),
            "fhe_keygen_from_seed": (ctypes.c_int, [ctypes.POINTER(Params), u64, sz, vp,
                                                    ctypes.POINTER(vp)]),
            "fhe_keys_free": (None, [vp]),
            "fhe_keys_params": (ctypes.c_int, [vp, ctypes.POINTER(Params)]),
            "fhe_keys_size": (sz, [vp, ctypes.c_int]),
            "fhe_keys_export": (ctypes.c_int, [vp, ctypes.c_int, vp, sz]),
            "fhe_encrypt": (ctypes.c_int, [vp, vp, sz, u64, vp, vp]),
            "fhe_decrypt": (ctypes.c_int, [vp, vp, sz, vp, vp]),
            "fhe_lwe_linear": (ctypes.c_int, [u32, u32, vp, sz, sz, vp, vp, sz, vp, vp]),
            "fhe_lwe_conv2d": (ctypes.c_int, [u32, u32, vp] + [u32] * 8 + [vp, vp, sz, vp, vp]),
            "fhe_lut_create": (ctypes.c_int, [vp, vp, u32, ctypes.POINTER(vp)]),
            "fhe_lut_free": (None, [vp]),
            "fhe_pbs_batch": (ctypes.c_int, [vp, vp, sz, vp, vp, ctypes.c_int, vp]),
            "fhe_status": (ctypes.c_int, [vp, vp]),
            "fhe_snn_create": (ctypes.c_int, [vp, ctypes.POINTER(SnnDesc), ctypes.POINTER(vp)]),
            "fhe_snn_free": (None, [vp]),
            "fhe_snn_pbs_per_image": (u64, [vp]),
            "fhe_snn_infer": (ctypes.c_int, [vp, vp, sz, vp, ctypes.c_int, vp]),
            "fhe_snn_layer_spikes": (ctypes.c_int, [vp, u32, vp, vp]),
            "fhe_snn_profile": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_double),
                                               ctypes.POINTER(u64), ctypes.POINTER(u64)]),
            "fhe_kernel_launches": (u64, []),
            "fhe_pbs_batch_noalloc": (ctypes.c_int, [vp, vp, sz, vp, vp, vp]),
            "fhe_snn_begin": (ctypes.c_int, [vp, vp, sz, ctypes.c_int, vp]),
            "fhe_snn_step": (ctypes.c_int, [vp, vp]),
            "fhe_snn_end": (ctypes.c_int, [vp, vp, ctypes.c_int, vp]),
            "fhe_snn_iterations": (u32, [vp]),
            "fhe_selftest_timeout": (ctypes.c_int, [vp, u32, vp]),
            "fhe_fft_max_error": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
            "fhe_snn_stream_push": (ctypes.c_int, [vp, vp, sz, vp, ctypes.c_int, vp]),
            "fhe_snn_stream_flush": (ctypes.c_int, [vp, vp]),
            "fhe_pbs_autotune": (ctypes.c_int, [vp, ctypes.POINTER(u64), vp]),
            "fhe_lut_create_spaces": (ctypes.c_int, [vp, vp, u32, u32, vp, vp, ctypes.POINTER(vp)]),
            "fhe_pbs_batch_groups": (ctypes.c_int, [vp, vp, sz, vp, vp, vp, ctypes.c_int, vp]),
            "fhe_pbs_tuning": (ctypes.c_int, [vp, ctypes.POINTER(u64), ctypes.POINTER(i32),
                                              ctypes.POINTER(i32), ctypes.POINTER(i32)]),
            "fhe_pbs_set_tc_option": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int]),
            "fhe_tc_plan_query": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.POINTER(TcPlan)]),
            "fhe_snn_stream_stage": (ctypes.c_int, [vp, vp, sz, vp, ctypes.c_int, vp]),
            "fhe_snn_stream_iterate": (ctypes.c_int, [vp, vp]),
            "fhe_snn_stream_state": (ctypes.c_int, [vp, u64, u32, ctypes.c_int, vp, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def kernel_launches():
    return int(lib().fhe_kernel_launches())


def strerror(code):
    return lib().fhe_strerror(int(code)).decode()


def _check(rc, what):
    if rc != FHE_OK:
        raise FheError(rc, what)


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _dev_u32(x, shape=None):
    """Device int32 tensor holding uint32 words (numpy uint32 accepted)."""
    import torch
    if isinstance(x, np.ndarray):
        x = torch.from_numpy(np.ascontiguousarray(x).view(np.int32)).cuda()
    assert x.is_cuda and x.dtype == torch.int32 and x.is_contiguous()
    return x if shape is None else x.view(*shape)


def to_numpy_u32(t):
    return t.detach().cpu().numpy().view(np.uint32)


class Keys:
    """Handle of fhe_keygen_from_seed (device keys and PBS workspace)."""

    def __init__(self, params, seed, max_batch=0, stream=None):
        self.params = dict(params)
        self._p = Params.from_dict(params)
        h = ctypes.c_void_p()
        _check(lib().fhe_keygen_from_seed(ctypes.byref(self._p), int(seed), int(max_batch),
                                          _stream(stream), ctypes.byref(h)), "keygen_from_seed")
        self.handle = h

    def free(self):
        if self.handle:
            lib().fhe_keys_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def export(self, which):
        size = lib().fhe_keys_size(self.handle, which)
        out = np.zeros(size // 4, np.uint32)
        _check(lib().fhe_keys_export(self.handle, which, out.ctypes.data_as(ctypes.c_void_p),
                                     size), "keys_export")
        return out

    def fft_max_error(self, reset=False):
        """Largest rounding distance of the FFT variant's products so far."""
        v = ctypes.c_double()
        _check(lib().fhe_fft_max_error(self.handle, ctypes.byref(v), int(bool(reset))),
               "fft_max_error")
        return v.value

    def selftest_timeout(self, limit_us=20000, stream=None):
        """Bounded-wait self-test; returns FHE_ETIMEOUT when detection works."""
        return lib().fhe_selftest_timeout(self.handle, int(limit_us), _stream(stream))

    def status(self, stream=None):
        return lib().fhe_status(self.handle, _stream(stream))

    def autotune(self, stream=None):
        """fhe_pbs_autotune: smallest batch run on tensor cores by
        VARIANT_AUTO, measured on this device (None: not available)."""
        v = ctypes.c_uint64()
        _check(lib().fhe_pbs_autotune(self.handle, ctypes.byref(v), _stream(stream)), "pbs_autotune")
        return None if v.value == (1 << 64) - 1 else int(v.value)

    def tuning(self):
        """fhe_pbs_tuning: (smallest batch AUTO runs on tensor cores or None,
        most tiles run on clusters of 8, of 16, spread over two clusters of 16)."""
        v, c, c16, c32 = ctypes.c_uint64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().fhe_pbs_tuning(self.handle, ctypes.byref(v), ctypes.byref(c),
                                    ctypes.byref(c16), ctypes.byref(c32)), "pbs_tuning")
        return ((None if v.value == (1 << 64) - 1 else int(v.value)), int(c.value), int(c16.value),
                int(c32.value))

    def set_tc_option(self, option, value):
        """fhe_pbs_set_tc_option: TC_OPT_CLUSTER (0, 4, 8, 16),
        TC_OPT_MULTICAST (-1, 0, 1) or TC_OPT_L2_HINTS (-1, 0, 1)."""
        _check(lib().fhe_pbs_set_tc_option(self.handle, int(option), int(value)),
               "pbs_set_tc_option")


def tc_plan(params):
    """fhe_tc_plan_query: the tensor-core path's exactness plan for a
    parameter dict (host only)."""
    p = Params.from_dict(params)
    out = TcPlan()
    _check(lib().fhe_tc_plan_query(ctypes.byref(p), ctypes.byref(out)), "tc_plan_query")
    return {f: int(getattr(out, f)) for f, _ in TcPlan._fields_}


def keygen_from_seed(params, seed, max_batch=0, stream=None):
    return Keys(params, seed, max_batch, stream)


def encrypt(keys, msg, seed, out=None, stream=None):
    import torch
    msg = msg if isinstance(msg, torch.Tensor) else torch.as_tensor(np.asarray(msg, np.int32))
    msg = msg.to(device="cuda", dtype=torch.int32).contiguous().view(-1)
    w = keys.params["n"] + 1
    if out is None:
        out = torch.empty((msg.numel(), w), dtype=torch.int32, device="cuda")
    _check(lib().fhe_encrypt(keys.handle, _ptr(msg), msg.numel(), int(seed), _ptr(out),
                             _stream(stream)), "encrypt")
    return out


def decrypt(keys, ct, stream=None):
    import torch
    ct = _dev_u32(ct)
    w = keys.params["n"] + 1
    count = ct.numel() // w
    out = torch.empty(count, dtype=torch.int32, device="cuda")
    _check(lib().fhe_decrypt(keys.handle, _ptr(ct), count, _ptr(out), _stream(stream)), "decrypt")
    return out


def lwe_linear(params, W, ct_in, bias=None, out=None, stream=None):
    """ct_in: (batch, K, n+1) or (K, n+1) device int32; W: (M, K) device int32."""
    import torch
    n, log2_p = params["n"], params["log2_p"]
    M, K = W.shape
    ct_in = _dev_u32(ct_in)
    batch = ct_in.numel() // (K * (n + 1))
    if out is None:
        out = torch.empty((batch, M, n + 1), dtype=torch.int32, device="cuda")
    _check(lib().fhe_lwe_linear(n, log2_p, _ptr(W), M, K, _ptr(bias), _ptr(ct_in), batch,
                                _ptr(out), _stream(stream)), "lwe_linear")
    return out


def lwe_conv2d(params, W, ct_in, cin, h, w, stride, pad, bias=None, batch=1, out=None,
               stream=None):
    import torch
    n, log2_p = params["n"], params["log2_p"]
    cout, cin_, kh, kw = W.shape
    assert cin_ == cin
    ho, wo = (h + 2 * pad - kh) // stride + 1, (w + 2 * pad - kw) // stride + 1
    if out is None:
        out = torch.empty((batch, cout * ho * wo, n + 1), dtype=torch.int32, device="cuda")
    _check(lib().fhe_lwe_conv2d(n, log2_p, _ptr(W), cin, h, w, cout, kh, kw, stride, pad,
                                _ptr(bias), _ptr(_dev_u32(ct_in)), batch, _ptr(out),
                                _stream(stream)), "lwe_conv2d")
    return out


class Lut:
    """Bootstrap tables (fhe_lut_create).  With log2_p_in / log2_p_out
    (fhe_lut_create_spaces): f is a list of groups, group g an (L, 2^log2_p_in[g])
    array whose table j is written in the space 2^log2_p_out[g][j]."""

    def __init__(self, keys, f, log2_p_in=None, log2_p_out=None):
        h = ctypes.c_void_p()
        if log2_p_in is None:
            f = np.ascontiguousarray(np.asarray(f, np.int32).reshape(-1, 1 << keys.params["log2_p"]))
            self.L = f.shape[0]
            self.groups = 1
            _check(lib().fhe_lut_create(keys.handle, f.ctypes.data_as(ctypes.c_void_p), self.L,
                                        ctypes.byref(h)), "lut_create")
        else:
            lp_in = np.ascontiguousarray(np.asarray(log2_p_in, np.uint32).reshape(-1))
            self.groups = lp_in.shape[0]
            tabs = [np.asarray(fg, np.int32).reshape(-1, 1 << int(lp)) for fg, lp in zip(f, lp_in)]
            self.L = tabs[0].shape[0]
            flat = np.ascontiguousarray(np.concatenate([t.reshape(-1) for t in tabs]))
            lp_out = np.ascontiguousarray(np.asarray(log2_p_out, np.uint32).reshape(-1))
            if (len(tabs) != self.groups or lp_out.shape[0] != self.groups * self.L
                    or any(t.shape[0] != self.L for t in tabs)):
                raise ValueError("one group of L tables and L output spaces per input space")
            _check(lib().fhe_lut_create_spaces(keys.handle, flat.ctypes.data_as(ctypes.c_void_p),
                                               self.L, self.groups,
                                               lp_in.ctypes.data_as(ctypes.c_void_p),
                                               lp_out.ctypes.data_as(ctypes.c_void_p),
                                               ctypes.byref(h)), "lut_create_spaces")
        self.handle = h

    def free(self):
        if self.handle:
            lib().fhe_lut_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def lut_create(keys, f):
    return Lut(keys, f)


def pbs_batch(keys, ct_in, lut, variant=VARIANT_EXACT, out=None, stream=None):
    """Returns (L, count, n+1) device int32 (uint32 words)."""
    import torch
    w = keys.params["n"] + 1
    ct_in = _dev_u32(ct_in)
    count = ct_in.numel() // w
    if out is None:
        out = torch.empty((lut.L, count, w), dtype=torch.int32, device="cuda")
    _check(lib().fhe_pbs_batch(keys.handle, _ptr(ct_in), count, lut.handle, _ptr(out),
                               int(variant), _stream(stream)), "pbs_batch")
    return out


def pbs_batch_groups(keys, ct_in, lut, seg_end, variant=VARIANT_EXACT, out=None, stream=None):
    """fhe_pbs_batch_groups: inputs [seg_end[g-1], seg_end[g]) use table
    group g of a grouped Lut; (L, count, n+1) int32."""
    import torch
    w = keys.params["n"] + 1
    ct_in = _dev_u32(ct_in)
    count = ct_in.numel() // w
    if out is None:
        out = torch.empty((lut.L, count, w), dtype=torch.int32, device="cuda")
    ends = (ctypes.c_size_t * max(1, len(seg_end)))(*[int(e) for e in seg_end])
    _check(lib().fhe_pbs_batch_groups(keys.handle, _ptr(ct_in), count, lut.handle,
                                      ctypes.cast(ends, ctypes.c_void_p) if len(seg_end) else None,
                                      _ptr(out), int(variant), _stream(stream)),
           "pbs_batch_groups")
    return out


def pbs_batch_noalloc(keys, ct_in, lut, out=None, stream=None):
    """fhe_pbs_batch_noalloc: exact bootstrapping with the library's fixed
    scratch array (no allocation in the library); (L, count, n+1) int32."""
    import torch
    w = keys.params["n"] + 1
    ct_in = _dev_u32(ct_in)
    count = ct_in.numel() // w
    if out is None:
        out = torch.empty((lut.L, count, w), dtype=torch.int32, device="cuda")
    _check(lib().fhe_pbs_batch_noalloc(keys.handle, _ptr(ct_in), count, lut.handle, _ptr(out),
                                       _stream(stream)), "pbs_batch_noalloc")
    return out


class Snn:
    """Encrypted DiCSNN (fhe_snn_create / fhe_snn_infer).

    net: {"layers": [...], "lif": {"v_th", "leak_shift", "spike_scale"}, "T",
    "static_input", optional "lif_mode" ("multi" or "two_pbs")}; a layer is
    {"type": "fc", "W": [out][in]}, {"type": "conv", "W": [cout][cin][kh][kw],
    "h", "w", "stride", "pad"} or {"type": "poisson", "M": [T][pixels]}, with
    an optional "log2_p" giving the layer its own message space."""

    def __init__(self, keys, net, max_images, variant=VARIANT_EXACT, use_graph=True,
                 profile=False):
        self.keys = keys
        self._weights = []
        descs = (LayerDesc * len(net["layers"]))()
        for i, layer in enumerate(net["layers"]):
            Wt = np.ascontiguousarray(np.asarray(layer["M" if layer["type"] == "poisson" else "W"],
                                                 np.int32))
            self._weights.append(Wt)
            d = descs[i]
            d.weights = Wt.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            d.log2_p = int(layer.get("log2_p", 0))
            if layer["type"] == "poisson":
                d.type = LAYER_POISSON
                d.in_size = d.out_size = Wt.shape[1]
            elif layer["type"] == "fc":
                d.type = LAYER_FC
                d.out_size, d.in_size = Wt.shape
            else:
                d.type = LAYER_CONV
                d.cout, d.cin, d.kh, d.kw = Wt.shape
                d.h, d.w, d.stride, d.pad = layer["h"], layer["w"], layer["stride"], layer["pad"]
        lif = net["lif"]
        self.desc = SnnDesc(len(net["layers"]), descs, lif["v_th"], lif["leak_shift"],
                            lif["spike_scale"], net["T"], int(bool(net.get("static_input"))),
                            max_images, int(variant),
                            int(bool(use_graph)) | (SNN_PROFILE if profile else 0),
                            LIF_TWO_PBS if net.get("lif_mode") == "two_pbs" else LIF_MULTI_VALUE)
        self._descs = descs
        h = ctypes.c_void_p()
        _check(lib().fhe_snn_create(keys.handle, ctypes.byref(self.desc), ctypes.byref(h)),
               "snn_create")
        self.handle = h
        self.T = net["T"]
        self.static = bool(net.get("static_input"))
        self.n_out = (net["layers"][-1]["W"].shape[0] if net["layers"][-1]["type"] == "fc"
                      else None)

    def pbs_per_image(self):
        return int(lib().fhe_snn_pbs_per_image(self.handle))

    def infer(self, ct_input, n_images, scores, on_host=False, stream=None):
        """ct_input / scores: device tensors; if on_host, host numpy arrays or
        (pinned) CPU torch tensors."""
        if on_host:
            def hp(x):
                return (ctypes.c_void_p(x.data_ptr()) if hasattr(x, "data_ptr")
                        else x.ctypes.data_as(ctypes.c_void_p))
            pin, pout = hp(ct_input), hp(scores)
        else:
            pin, pout = _ptr(ct_input), _ptr(scores)
        _check(lib().fhe_snn_infer(self.handle, pin, n_images, pout, int(bool(on_host)),
                                   _stream(stream)), "snn_infer")
        return scores

    def iterations(self):
        return int(lib().fhe_snn_iterations(self.handle))

    def begin(self, ct_input, n_images, stream=None):
        """Stage a device input and reset the state (fhe_snn_begin)."""
        _check(lib().fhe_snn_begin(self.handle, _ptr(ct_input), n_images, 0, _stream(stream)),
               "snn_begin")

    def step(self, stream=None):
        """One layer-skewed step; returns the number of steps still to run."""
        rc = lib().fhe_snn_step(self.handle, _stream(stream))
        if rc < 0:
            _check(rc, "snn_step")
        return rc

    def end(self, scores, stream=None):
        _check(lib().fhe_snn_end(self.handle, _ptr(scores), 0, _stream(stream)), "snn_end")
        return scores

    def stream_push(self, ct_input, n_images, scores, on_host=False, stream=None):
        """Start one batch of a streamed inference (fhe_snn_stream_push);
        `scores` receives the batch's encrypted scores once it completes."""
        if on_host:
            def hp(x):
                return (ctypes.c_void_p(x.data_ptr()) if hasattr(x, "data_ptr")
                        else x.ctypes.data_as(ctypes.c_void_p))
            pin, pout = hp(ct_input), hp(scores)
        else:
            pin, pout = _ptr(ct_input), _ptr(scores)
        _check(lib().fhe_snn_stream_push(self.handle, pin, n_images, pout, int(bool(on_host)),
                                         _stream(stream)), "snn_stream_push")
        return scores

    def stream_stage(self, ct_input, n_images, scores, on_host=False, stream=None):
        """Stage the next batch without running a step (fhe_snn_stream_stage)."""
        if on_host:
            pin = ctypes.c_void_p(ct_input.data_ptr()) if hasattr(ct_input, "data_ptr") \
                else ct_input.ctypes.data_as(ctypes.c_void_p)
            pout = ctypes.c_void_p(scores.data_ptr()) if hasattr(scores, "data_ptr") \
                else scores.ctypes.data_as(ctypes.c_void_p)
        else:
            pin, pout = _ptr(ct_input), _ptr(scores)
        _check(lib().fhe_snn_stream_stage(self.handle, pin, n_images, pout, int(bool(on_host)),
                                          _stream(stream)), "snn_stream_stage")
        return scores

    def stream_iterate(self, stream=None):
        """Run the stream's next step; returns the steps that can still run."""
        rc = lib().fhe_snn_stream_iterate(self.handle, _stream(stream))
        if rc < 0:
            _check(rc, "snn_stream_iterate")
        return rc

    def stream_state(self, batch, layer, kind, dst, stream=None):
        """Copy a streamed batch's layer state (STATE_SPIKES, STATE_MEMBRANES
        or STATE_CURRENTS) into the device tensor dst."""
        _check(lib().fhe_snn_stream_state(self.handle, int(batch), int(layer), int(kind), _ptr(dst),
                                          _stream(stream)), "snn_stream_state")
        return dst

    def stream_flush(self, stream=None):
        """Complete every pushed batch and end the stream."""
        _check(lib().fhe_snn_stream_flush(self.handle, _stream(stream)), "snn_stream_flush")

    def profile(self):
        """(blind-rotation ms, launches, ciphertexts) of the last inference."""
        ms = ctypes.c_double()
        nl = ctypes.c_uint64()
        nc = ctypes.c_uint64()
        _check(lib().fhe_snn_profile(self.handle, ctypes.byref(ms), ctypes.byref(nl),
                                     ctypes.byref(nc)), "snn_profile")
        return ms.value, nl.value, nc.value

    def layer_spikes(self, layer, dst, stream=None):
        _check(lib().fhe_snn_layer_spikes(self.handle, layer, _ptr(dst), _stream(stream)),
               "snn_layer_spikes")
        return dst

    def free(self):
        if self.handle:
            lib().fhe_snn_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
