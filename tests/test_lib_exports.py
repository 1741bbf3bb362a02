"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/rnnls.h declares (no compute call: no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rnnls.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rnnls_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_0812_4547_gb300 import build

    return build.build()


def test_header_lists_the_boundary():
    names = declared_functions()
    for must in ("rnnls_sketch", "rnnls_solve", "rnnls_solve_batched", "rnnls_create", "rnnls_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (rnnls_[a-z0-9_]+)\b", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_binding_names_match_header(libpath):
    from paper_0812_4547_gb300 import _binding

    assert sorted(_binding.EXPORTS) == declared_functions()
    lib = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(lib, name)


def test_struct_layouts_match_header(tmp_path):
    """Every field offset and struct size of the ctypes mirrors equals what a
    C compiler makes of include/rnnls.h."""
    from paper_0812_4547_gb300 import _binding

    structs = [_binding.rnnls_info, _binding.rnnls_problem, _binding.rnnls_sketch_job, _binding.rnnls_kernel_time,
               _binding.rnnls_tuning]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "rnnls.h"', "int main(void) {"]
    for st in structs:
        n = st.__name__
        lines.append(f'  printf("{n} %zu\\n", sizeof({n}));')
        for f in st._fields_:
            lines.append(f'  printf("{n}.{f[0]} %zu\\n", offsetof({n}, {f[0]}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    for st in structs:
        n = st.__name__
        assert int(got[n]) == ctypes.sizeof(st), n
        for f in st._fields_:
            assert int(got[f"{n}.{f[0]}"]) == getattr(st, f[0]).offset, (n, f[0])


def test_strerror_needs_no_device(libpath):
    lib = ctypes.CDLL(libpath)
    lib.rnnls_strerror.restype = ctypes.c_char_p
    assert lib.rnnls_strerror(0) == b"ok"
    assert b"argument" in lib.rnnls_strerror(1)
