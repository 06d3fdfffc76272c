"""Host-side checks that need no GPU: the library builds, loads and exports every
entry point that include/mra.h declares; the binding covers the same names;
the C structs have the layout the header describes."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_names():
    hdr = open(os.path.join(ROOT, "include", "mra.h")).read()
    return re.findall(r"MRA_API\s+[\w\s\*]+?\b(mra_\w+)\s*\(", hdr)


def test_header_declares_the_entry_points():
    names = set(header_names())
    for n in ("mra_sync", "mra_fit_prior", "mra_em_step", "mra_em_run", "mra_loglik_grad"):
        assert n in names


def test_library_exports_every_declared_symbol():
    shutil_nvcc = any(os.path.exists(p) for p in ("/usr/local/cuda/bin/nvcc",))
    from paper_2105_07372_gb300 import build, mra

    if not os.path.exists(build.LIB):
        if not shutil_nvcc:
            pytest.skip("no nvcc to build libmra")
        build.build_library()
    lib = ctypes.CDLL(build.LIB)
    for n in header_names():
        assert hasattr(lib, n), n
    assert set(header_names()) == set(mra.exported_symbols())
    lib.mra_status_string.restype = ctypes.c_char_p
    assert lib.mra_status_string(-6) == b"workspace too small"


def test_struct_layout():
    from paper_2105_07372_gb300 import mra

    assert ctypes.sizeof(mra.mra_dims) == 24
    assert mra.mra_em_params.tol.offset == 40 and mra.mra_em_params.sweep_ms.offset == 56
    assert ctypes.sizeof(mra.mra_em_params) == 72


def test_struct_layout_matches_the_c_compiler(tmp_path):
    """Offsets of every binding struct field equal offsetof() in the header, compiled by gcc."""
    import shutil
    import subprocess

    from paper_2105_07372_gb300 import mra

    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    structs = [mra.mra_dims, mra.mra_em_params, mra.mra_instance]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "mra.h"', "int main(void) {"]
    for st in structs:
        lines.append(f'  printf("{st.__name__} %zu\\n", sizeof({st.__name__}));')
        for f, _ in st._fields_:
            lines.append(f'  printf("{st.__name__}.{f} %zu\\n", offsetof({st.__name__}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n") if l)
    for st in structs:
        assert int(got[st.__name__]) == ctypes.sizeof(st), st.__name__
        for f, _ in st._fields_:
            assert int(got[f"{st.__name__}.{f}"]) == getattr(st, f).offset, (st.__name__, f)


def test_oracle_not_imported_by_product():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2105_07372_gb300")
    pat = re.compile(r"^\s*(import\s+oracle|from\s+oracle|from\s+\.\.\s*import\s+oracle)", re.M)
    for dp, _, fs in os.walk(pkg):
        for f in fs:
            if f.endswith(".py"):
                assert not pat.search(open(os.path.join(dp, f)).read()), f


def test_every_entry_point_names_its_passage():
    """Each declaration's comment cites the paper's passage it implements (Sec., Eq., App., Algorithm), or
    states that it has no counterpart in the paper."""
    src = open(os.path.join(ROOT, "include", "mra.h")).read()
    missing = []
    for m in re.finditer(r"MRA_API[^;]*?\b(mra_\w+)\s*\(", src):
        cstart, cend = src.rfind("/*", 0, m.start()), src.rfind("*/", 0, m.start())
        comment = " ".join(src[cstart:cend].replace("*", " ").split()) if 0 <= cstart < cend else ""
        if not re.search(r"Sec\.|Eq\.|App\.|Algorithm|counterpart in the paper|not in the paper", comment):
            missing.append(m.group(1))
    assert not missing, missing

