"""Static checks (no GPU) that the product path and the oracle stay apart:
the package and its CUDA sources never import, load or read the oracle, and
the oracle never imports the package.  The one shared module is the seeded
input generator (paper_1109_1027_gb300/workloads.py), which tests hand to
both sides; it holds none of the method's arithmetic, so it may not call
into the library either."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1109_1027_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _sources(top, exts):
    for dirpath, dirnames, files in os.walk(top):
        dirnames[:] = [d for d in dirnames if d not in ("__pycache__", "_build", "lib")]
        for f in files:
            if f.endswith(exts):
                yield os.path.join(dirpath, f)


def _code(path):
    with open(path, encoding="utf-8") as fh:
        text = fh.read()
    if path.endswith(".py"):
        text = re.sub(r'""".*?"""', "", text, flags=re.S)     # docstrings may name the oracle
        text = re.sub(r"#.*", "", text)
    else:
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//.*", "", text)
    return text


def test_package_never_references_the_oracle():
    for path in _sources(PKG, (".py", ".cu", ".cuh", ".h")):
        assert not re.search(r"\boracle\b", _code(path)), path
    for path in _sources(os.path.join(ROOT, "include"), (".h",)):
        assert not re.search(r"\boracle\b", _code(path)), path


def test_oracle_never_imports_the_package():
    for path in _sources(ORACLE, (".py", ".c", ".h")):
        code = _code(path)
        assert "paper_1109_1027_gb300" not in code, path
        assert not re.search(r"libnlse(?!_oracle)", code), path     # its own library is libnlse_oracle_*


def test_input_generators_hold_no_library_calls():
    code = _code(os.path.join(PKG, "workloads.py"))
    assert not re.search(r"\bimport\s+torch\b|\bfrom\s+\.\s+import\s+nlse\b|\bnlse\.", code)
