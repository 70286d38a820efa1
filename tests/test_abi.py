"""Host-side checks of the C ABI: the library builds, loads without a GPU and
exports every entry point declared in include/tflbm.h; the ctypes mirrors of
the structs match the header; the oracle and the library share no code."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1810_07642_gb300 import _lib as L
from paper_1810_07642_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tflbm.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tf_lbm_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("tf_lbm_init", "tf_lbm_step", "tf_lbm_moments", "tf_lbm_mass",
                     "tf_lbm_check", "tf_lbm_destroy", "tf_lbm_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(tf_lbm_\w+)", out))
    missing = set(declared_functions()) - exported
    assert not missing, missing
    lib = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(lib, name)


def test_binding_covers_header(libpath):
    assert set(L.EXPORTED) == set(declared_functions())
    for name in L.EXPORTED:
        assert callable(getattr(L, name))


def test_struct_mirrors_match_header_layout(tmp_path):
    """The ctypes mirrors have the sizes and field offsets the C compiler
    gives the structs of include/tflbm.h."""
    import subprocess
    structs = {"tf_lbm_params": L.Params, "tf_lbm_launch": L.Launch,
               "tf_lbm_batch_launch": L.BatchLaunch}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "tflbm.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0; }"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", f"-I{os.path.join(ROOT, 'include')}", str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {(a, b): int(c) for a, b, c in (l.split() for l in out if l.strip())}
    for cname, py in structs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_library_loads_without_gpu_and_reports_version(libpath):
    assert L.tf_lbm_version() >= 100
    assert L.tf_lbm_last_error() == ""


def test_oracle_and_library_share_no_code():
    """Neither side imports or includes the other; only the seeded input
    generators (paper_1810_07642_gb300/inputs.py, no arithmetic of the
    method) are shared, and only by the tests."""
    pkg = os.path.join(ROOT, "paper_1810_07642_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, fn)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), fn
                assert "tflbm_oracle" not in text, fn
    for fn in os.listdir(os.path.join(ROOT, "oracle")):
        if fn.endswith((".py", ".c", ".h")):
            text = open(os.path.join(ROOT, "oracle", fn)).read()
            assert not re.search(r"^\s*(import|from)\s+paper_1810_07642_gb300", text, re.M), fn
            assert not re.search(r"#\s*include\s+\S*tflbm", text), fn


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No CPU fallback: with the shared library absent every entry point
    raises instead of computing anything elsewhere."""
    from paper_1810_07642_gb300 import _lib as L
    from paper_1810_07642_gb300 import build
    monkeypatch.setattr(build, "LIB", str(tmp_path / "absent.so"))
    monkeypatch.setattr(L, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        L.tf_lbm_version()
    with pytest.raises(RuntimeError, match="not built"):
        L.tf_lbm_step(1, 1)
