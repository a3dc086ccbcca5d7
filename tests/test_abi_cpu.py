"""CPU checks of the C ABI library: it builds, loads without a GPU and
exports every entry point the header declares (no compute calls)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "fhe_dicsnn.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fhe_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    from paper_2309_09025_gb300 import build, fhe
    path = build.build()
    L = ctypes.CDLL(path)
    declared = _declared()
    assert len(declared) >= 15
    missing = [s for s in declared if not hasattr(L, s)]
    assert not missing, missing
    assert sorted(fhe.EXPORTED) == declared


def test_strerror_without_gpu():
    from paper_2309_09025_gb300 import fhe
    assert fhe.strerror(0) == "ok"
    assert "invalid" in fhe.strerror(fhe.FHE_EINVAL)
    assert fhe.strerror(12345) == "unknown error"


def test_unsupported_params_rejected_before_any_device_work():
    from paper_2309_09025_gb300 import fhe, synth
    p = fhe.Params.from_dict(dict(synth.P64, k=2))
    h = ctypes.c_void_p()
    rc = fhe.lib().fhe_keygen_from_seed(ctypes.byref(p), 1, 0, None, ctypes.byref(h))
    assert rc == fhe.FHE_EINVAL and not h.value
    rc = fhe.lib().fhe_keygen_from_seed(None, 1, 0, None, ctypes.byref(h))
    assert rc == fhe.FHE_EINVAL


def test_ctypes_structs_match_the_header(tmp_path):
    """The binding's ctypes mirrors of the ABI structs have the header's
    size and field offsets (a C probe compiled with the host compiler
    against include/fhe_dicsnn.h prints them)."""
    import shutil
    import subprocess

    import pytest

    from paper_2309_09025_gb300 import fhe
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    mirrors = {"fhe_params": fhe.Params, "fhe_layer_desc": fhe.LayerDesc,
               "fhe_snn_desc": fhe.SnnDesc, "fhe_tc_plan": fhe.TcPlan}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "fhe_dicsnn.h"',
             "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append('  printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for field, _ in py._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));'
                         % (cname, field, cname, field))
    lines += ["  return 0;", "}"]
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "probe"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for field, _ in py._fields_:
            assert got[(cname, field)] == getattr(py, field).offset, (cname, field)


def test_binding_constants_match_the_header():
    """Every #define of the header has the same value in the binding
    (FHE_X there is FHE_X, X or a listed alias here)."""
    from paper_2309_09025_gb300 import fhe
    text = open(os.path.join(ROOT, "include", "fhe_dicsnn.h")).read()
    defines = dict(re.findall(r"#define (FHE_[A-Z0-9_]+) ([^/\n]+)", text))
    defines.pop("FHE_DICSNN_H", None)
    alias = {"FHE_KEY_LWE": "KEY_LWE", "FHE_KEY_GLWE": "KEY_GLWE", "FHE_KEY_BSK": "KEY_BSK",
             "FHE_KEY_KSK": "KEY_KSK", "FHE_LAYER_FC": "LAYER_FC", "FHE_LAYER_CONV": "LAYER_CONV",
             "FHE_LAYER_POISSON": "LAYER_POISSON", "FHE_LIF_MULTI_VALUE": "LIF_MULTI_VALUE",
             "FHE_LIF_TWO_PBS": "LIF_TWO_PBS", "FHE_SNN_PROFILE": "SNN_PROFILE",
             "FHE_LUT_MAX_GROUPS": "LUT_MAX_GROUPS",
             "FHE_PBS_NOALLOC_MAX_WORDS": "PBS_NOALLOC_MAX_WORDS"}
    assert len(defines) >= 20
    def value_of(expr):  # "0", "(-1)", "(1u << 20)"
        e = expr.strip().strip("()").replace("u", "")
        if "<<" in e:
            a, b = e.split("<<")
            return int(a) << int(b)
        return int(e)

    for name, expr in defines.items():
        value = value_of(expr)
        py = getattr(fhe, name, None)
        if py is None:
            py = getattr(fhe, alias.get(name, name[len("FHE_"):]))
        assert py == value, name


def test_plain_c_client_builds_links_and_fails_cleanly_without_gpu(tmp_path):
    """tests/c_abi_example.c, a plain C client of the ABI (keys, encryption,
    one multi-value bootstrap batch, decryption, check against the tables),
    compiles against the header and links against the library.  Without a
    GPU it must stop at the first call with the library's error code (exit 2,
    the failing call named), not crash; with one it must find every output
    equal to its table value (exit 0)."""
    import shutil
    import subprocess

    import pytest

    from paper_2309_09025_gb300 import build
    cc = shutil.which("gcc") or shutil.which("cc")
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    if cc is None or not os.path.exists(os.path.join(cuda, "include", "cuda_runtime.h")):
        pytest.skip("no C compiler or CUDA headers")
    lib = build.build()
    libdir = os.path.dirname(lib)
    cudalib = next((d for d in (os.path.join(cuda, "lib64"), os.path.join(cuda, "lib"))
                    if os.path.exists(d)), None)
    exe = tmp_path / "c_abi_example"
    cmd = [cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(cuda, "include"), os.path.join(ROOT, "tests", "c_abi_example.c"),
           "-o", str(exe), "-L", libdir, "-lfhe_dicsnn", "-Wl,-rpath," + libdir]
    if cudalib:
        cmd += ["-L", cudalib, "-Wl,-rpath," + cudalib]
    cmd += ["-lcudart"]
    subprocess.run(cmd, check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    try:
        import torch
        gpu = torch.cuda.is_available()
    except ImportError:
        gpu = False
    if gpu:
        assert r.returncode == 0, r.stdout + r.stderr
    else:
        assert r.returncode == 2, r.stdout + r.stderr
        assert "fhe_keygen_from_seed" in r.stderr


def test_replica_build_compiles_no_multicast():
    """Runs with one process per GPU load the replica library; every source
    it compiles, preprocessed with its flags, holds no multicast copy or
    multicast commit (the single-GPU forms live in fhe_tc_multicast.cuh,
    which the replica flags leave out)."""
    import subprocess
    from paper_2309_09025_gb300 import build
    try:
        nv = build.nvcc()
    except RuntimeError:
        pytest.skip("no nvcc")
    flags = [f for f in build._flags(False, replica=True) if not f.startswith("-gencode")
             and not f.startswith("arch=")]
    for src in build.SOURCES:
        r = subprocess.run([nv, "-E", "-x", "cu"] + build.ARCH + flags +
                           [os.path.join(build.CSRC, src)], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[-2000:]
        bad = [l for l in r.stdout.splitlines()
               if "multicast" in l and ("cp.async" in l or "tcgen05" in l or "asm" in l)]
        assert not bad, (src, bad[:3])
