"""The product path and the oracle share no code (CPU checks).

The CUDA library and its binding never import, include or link the oracle;
the oracle reaches into the product package only for the seeded input
generators and parameter presets of `synth`, which hold none of the method's
arithmetic.
"""
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2309_09025_gb300")


def _sources(top, exts):
    for d, _, files in os.walk(top):
        if "_build" in d or "__pycache__" in d:
            continue
        for f in files:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_product_never_reaches_the_oracle():
    bad = re.compile(r"^\s*(from\s+oracle\b|import\s+oracle\b)|#\s*include\s*[<\"].*oracle|"
                     r"tfhe_oracle|\borc_[a-z]", re.M)
    hits = [p for p in _sources(PKG, (".py", ".cu", ".cuh", ".h")) if bad.search(open(p).read())]
    hits += [p for p in _sources(os.path.join(ROOT, "include"), (".h",))
             if bad.search(open(p).read())]
    assert not hits, hits


def test_oracle_uses_only_the_input_generators_of_the_package():
    pat = re.compile(r"^\s*(?:from\s+paper_2309_09025_gb300(?:\.(\w+))?\s+import\s+([\w, ]+)|"
                     r"import\s+paper_2309_09025_gb300(?:\.(\w+))?)", re.M)
    for p in _sources(os.path.join(ROOT, "oracle"), (".py", ".c", ".h")):
        for m in pat.finditer(open(p).read()):
            names = {m.group(1) or "", m.group(3) or ""} | {
                n.strip() for n in (m.group(2) or "").split(",")}
            assert names - {"", "synth"} == set(), (p, m.group(0))


def test_importing_the_binding_loads_no_oracle_module():
    code = ("import sys; import paper_2309_09025_gb300.fhe, paper_2309_09025_gb300.synth; "
            "sys.exit(1 if any(m == 'oracle' or m.startswith('oracle.') for m in sys.modules) else 0)")
    assert subprocess.run([sys.executable, "-c", code], cwd=ROOT).returncode == 0
