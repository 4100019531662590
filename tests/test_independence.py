"""The oracle and the CUDA library are independent, and the library has no
fallback (no GPU needed).

* Nothing under oracle/ imports the package or reads its sources, and nothing
  in the package or its CUDA sources names the oracle: the two share only the
  seeded input generators in synth/, which hold none of the method's
  arithmetic (they import neither side).
* Importing the package where libdid.so is missing raises ImportError: no
  call can fall back to a CPU implementation.
"""

import os
import re
import shutil
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1802_08938_gb300")


def _sources(folder, exts):
    for base, dirs, files in os.walk(folder):
        dirs[:] = [d for d in dirs if d not in ("__pycache__", "_build")]
        for f in files:
            if f.endswith(exts):
                yield os.path.join(base, f)


def test_oracle_does_not_use_the_library():
    for path in _sources(os.path.join(ROOT, "oracle"), (".py", ".c", ".h")):
        text = open(path).read()
        assert "paper_1802_08938_gb300" not in text, path
        assert "libdid" not in text and "csrc" not in text, path


def test_library_does_not_use_the_oracle():
    for path in _sources(PKG, (".py", ".cu", ".cuh", ".h", ".cpp")):
        text = open(path).read()
        assert not re.search(r"\boracle\b", text), path
    for path in _sources(os.path.join(ROOT, "include"), (".h",)):
        assert not re.search(r"\boracle\b", open(path).read()), path


def test_generators_import_neither_side():
    for path in _sources(os.path.join(ROOT, "synth"), (".py",)):
        text = open(path).read()
        assert not re.search(r"^\s*(from|import)\s+(oracle|paper_1802_08938_gb300)", text, re.M), path


def test_missing_library_fails_loudly(tmp_path):
    # a copy of the package without libdid.so next to it
    dst = tmp_path / "paper_1802_08938_gb300"
    dst.mkdir()
    shutil.copy(os.path.join(PKG, "__init__.py"), dst / "__init__.py")
    code = ("import sys; sys.path.insert(0, %r)\n"
            "try:\n"
            "    import paper_1802_08938_gb300\n"
            "except ImportError as e:\n"
            "    print('ImportError:', e)\n"
            "    sys.exit(0)\n"
            "sys.exit(3)\n") % str(tmp_path)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=str(tmp_path), timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "libdid.so is not built" in r.stdout
