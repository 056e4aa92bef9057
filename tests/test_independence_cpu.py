"""The product and the oracle share no code: nothing in the package (Python,
CUDA, C++) imports, includes, loads or names the oracle, and the oracle imports
nothing from the package.  Only the tests, smoke() and bench.py's CPU legs use
the oracle."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2203_12866_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _sources(top, exts):
    for d, dirs, files in os.walk(top):
        dirs[:] = [x for x in dirs if x not in ("_build", "__pycache__")]
        for f in files:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_package_does_not_use_the_oracle():
    pat = re.compile(r"^\s*(import\s+oracle|from\s+oracle|#\s*include\s*[<\"].*oracle)|cosenu_oracle|"
                     r"liboracle|oracle/", re.M)
    for path in _sources(PKG, (".py", ".cu", ".cuh", ".inc", ".cpp", ".h")):
        text = open(path).read()
        assert not pat.search(text), path


def test_oracle_does_not_use_the_package():
    pat = re.compile(r"paper_2203_12866_gb300|cosenu\.h\b|libcosenu\.so|stage_kernel|cosenu_device")
    for path in _sources(ORACLE, (".py", ".c", ".h")):
        assert not pat.search(open(path).read()), path


def test_binding_fails_loudly_without_the_library(tmp_path):
    """No fallback: a missing CUDA library is an error, not a silent CPU path."""
    import subprocess
    import sys
    code = ("from paper_2203_12866_gb300 import binding\n"
            "try:\n"
            f"    binding.load({str(tmp_path / 'missing.so')!r})\n"
            "except ImportError:\n"
            "    print('raised')\n")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                         check=True, timeout=120).stdout
    assert out.strip() == "raised"
