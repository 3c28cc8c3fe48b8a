"""C-ABI boundary checks that need no GPU: every entry point declared in include/hjg.h is
exported by libhjg.so and bound by the Python layer; the ctypes structures match the C
layout; the product path never touches the oracle."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hjg.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hjg_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2605_18566_gb300 import build as B
    return B.build()


def test_every_declared_symbol_is_exported(lib_path):
    from paper_2605_18566_gb300 import _lib
    names = _declared()
    assert len(names) >= 14
    lib = C.CDLL(lib_path)
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(_lib.symbols()) == names
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (hjg_[a-z0-9_]+)", out))
    assert set(names) <= exported


def test_struct_layout_matches_header(tmp_path):
    from paper_2605_18566_gb300 import _lib
    prog = tmp_path / "layout.c"
    fields = {
        "hjg_dynamics": _lib.Dynamics, "hjg_target": _lib.Target,
        "hjg_options": _lib.Options, "hjg_diag": _lib.Diag,
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "hjg.h"', 'int main(void){']
    for cname, cls in fields.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines.append("return 0;}")
    prog.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for cname, cls in fields.items():
        assert int(got[cname]) == C.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert int(got["%s.%s" % (cname, f)]) == getattr(cls, f).offset, (cname, f)


def test_header_is_plain_c_and_cxx(tmp_path):
    """The boundary header compiles warning-free as strict C99 and as C++11, so C callers
    and C++ callers see the same declarations."""
    prog = tmp_path / "hdr.c"
    prog.write_text('#include "hjg.h"\nint main(void) { return sizeof(hjg_options) > 0 ? 0 : 1; }\n')
    inc = os.path.join(ROOT, "include")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", inc,
                    str(prog), "-o", str(tmp_path / "c99")], check=True)
    subprocess.run(["g++", "-std=c++11", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", inc,
                    "-x", "c++", str(prog), "-o", str(tmp_path / "cxx11")], check=True)


def test_missing_library_fails_loudly():
    from paper_2605_18566_gb300 import _lib
    saved = _lib._lib
    try:
        _lib._lib = None
        with pytest.raises(RuntimeError, match="libhjg.so not found"):
            _lib.load(os.path.join(ROOT, "does_not_exist", "libhjg.so"))
    finally:
        _lib._lib = saved


def test_product_never_imports_oracle():
    pkg = os.path.join(ROOT, "paper_2605_18566_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, fn)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", txt, re.M), fn
                assert "hjg_oracle" not in txt and "liboracle" not in txt, fn


def test_status_strings(lib_path):
    from paper_2605_18566_gb300 import _lib
    lib = _lib.load()
    assert lib.hjg_status_string(0) == b"ok"
    assert lib.hjg_status_string(4) == b"non-finite result"
    assert lib.hjg_last_error(None) == b"null context"
