"""Build the sm_103a shared library libfhe_dicsnn.so in-tree.

Each translation unit is compiled by nvcc in parallel (one -gencode for
sm_103a), then linked with -shared.  No cmake; the same command works on the
x86-64 build host (cross-compilation) and on the aarch64 GPU host.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfhe_dicsnn.so")
# Replica library for runs with one process per GPU: compiled with
# FHE_NO_MULTICAST, so no cluster-multicast copy is compiled into it (the
# tensor-core blind rotation copies its digit tiles per CTA).
BUILD_REPLICA = os.path.join(HERE, "_build_replica")
LIB_REPLICA = os.path.join(HERE, "libfhe_dicsnn_replica.so")
SOURCES = ["fhe_keys.cu", "fhe_linear.cu", "fhe_pbs_exact.cu", "fhe_pbs_tc.cu", "fhe_snn.cu",
           "fhe_noalloc.cu", "fhe_pbs_fft.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags(verbose, replica=False):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                "--expt-relaxed-constexpr", "-I", os.path.join(HERE, "..", "include")]
    if replica:
        f += ["-DFHE_NO_MULTICAST"]
    if verbose:
        f += ["-Xptxas", "-v"]
    return f


def _compile(src, verbose, replica=False):
    obj = os.path.join(BUILD_REPLICA if replica else BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc()] + _flags(verbose, replica) + ["-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    return obj, r.stderr


def _stale(lib):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(HERE, "..", "include", "fhe_dicsnn.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, replica=False):
    """Compile and link libfhe_dicsnn.so (replica: libfhe_dicsnn_replica.so)
    if needed; returns its path."""
    lib = LIB_REPLICA if replica else LIB
    if not force and not _stale(lib):
        return lib
    os.makedirs(BUILD_REPLICA if replica else BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose, replica), SOURCES))
    if verbose:
        for _, log in results:
            print(log)
    tmp = lib + ".tmp.%d" % os.getpid()
    # runtime API only (no driver-API calls), so no -lcuda
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv, replica="--replica" in sys.argv))
