"""The oracle and the CUDA path share no code: the library never imports,
links or reads anything under oracle/, and the oracle imports nothing of the
library except the seeded input generators (workloads.py, which holds none
of the method's arithmetic)."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2310_16668_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _files(d, exts):
    for base, _, names in os.walk(d):
        if "_build" in base or "__pycache__" in base:
            continue
        for f in names:
            if f.endswith(exts):
                yield os.path.join(base, f)


def _imports(path):
    tree = ast.parse(open(path).read())
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            yield from (a.name for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            yield ("." * node.level) + (node.module or "")


def test_library_does_not_use_the_oracle():
    for path in _files(PKG, (".py",)):
        for mod in _imports(path):
            assert not mod.split(".")[0] == "oracle", (path, mod)
    for path in _files(PKG, (".cu", ".cuh", ".cpp", ".h")):
        text = open(path).read()
        assert not re.search(r'#include\s*["<][^">]*oracle', text), path
    for path in _files(os.path.join(ROOT, "include"), (".h",)):
        assert "oracle" not in open(path).read(), path


def test_oracle_uses_only_the_input_generators():
    for path in _files(ORACLE, (".py",)):
        for mod in _imports(path):
            if mod.startswith("paper_2310_16668_gb300"):
                assert mod == "paper_2310_16668_gb300.workloads" or mod == "paper_2310_16668_gb300", (path, mod)
    for path in _files(ORACLE, (".c", ".h")):
        text = open(path).read()
        assert "paper_2310_16668_gb300" not in text and "skel.h" not in text, path


def test_input_generators_hold_no_method_arithmetic():
    # workloads.py draws points, charges and samples; it must not evaluate a
    # kernel, build a tree or call the library
    text = open(os.path.join(PKG, "workloads.py")).read()
    for word in ("import torch", "_lib", "skel_", "def kernel", "hankel", "exp(1j", "4 * np.pi", "4.0 * np.pi",
                 "4 * math.pi", "np.log(np.sqrt", "1.0 / (4"):
        assert word not in text, word


def test_product_fails_loudly_without_the_library():
    # no CPU fallback: with the shared library missing, loading raises
    import subprocess
    import sys
    code = ("import paper_2310_16668_gb300._lib as L\n"
            "L.LIB_PATH = '/nonexistent/libskel.so'\n"
            "L._lib = None\n"
            "try:\n"
            "    L.load()\n"
            "except ImportError as e:\n"
            "    print('raised', e)\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.startswith("raised"), r.stdout + r.stderr
