"""The C-ABI library builds, loads and exports every entry point include/rsv.h declares.

Runs without a GPU: nothing here launches device work.  The ctypes structs of
the binding are checked field by field against the C compiler's layout of the
header's structs.
"""
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rsv.h")


def declared_functions():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^(?:rsv_status|void|const char\*)\s+(rsv_\w+)\s*\(", txt, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2008_10904_gb300 import build, rsv
    build.build()
    return rsv.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("rsv_create_operator", "rsv_set_frequencies", "rsv_march_direct", "rsv_march_adjoint",
              "rsv_gains_modes", "rsv_destroy_operator", "rsv_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_2008_10904_gb300", "librsv.so")],
                         capture_output=True, text=True).stdout
    for name in declared_functions():
        assert re.search(rf"\bT {name}$", out, re.M), name


def test_binding_covers_every_symbol(lib):
    from paper_2008_10904_gb300 import rsv
    assert sorted(rsv.exported_symbols()) == declared_functions()
    for name in declared_functions():
        assert callable(getattr(rsv, name))


def test_struct_layout_matches_header(tmp_path):
    from paper_2008_10904_gb300 import rsv
    import ctypes
    fields = {"rsv_operator_desc": rsv.rsv_operator_desc, "rsv_march_opts": rsv.rsv_march_opts,
              "rsv_series_opts": rsv.rsv_series_opts, "rsv_trm_opts": rsv.rsv_trm_opts}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void){"]
    for sname, cls in fields.items():
        lines.append(f'printf("{sname} size %zu\\n", sizeof({sname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{sname} {f} %zu\\n", offsetof({sname}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for ln in out:
        parts = ln.split()
        if len(parts) == 3:
            got[(parts[0], parts[1])] = int(parts[2])
    for sname, cls in fields.items():
        assert got[(sname, "size")] == ctypes.sizeof(cls)
        for f, _ in cls._fields_:
            assert got[(sname, f)] == getattr(cls, f).offset, (sname, f)


def test_version_and_error_without_gpu(lib):
    from paper_2008_10904_gb300 import rsv
    assert "sm_103a" in rsv.rsv_version()
    assert isinstance(rsv.rsv_last_error(), str)


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2008_10904_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", txt, re.M), f
                assert "oracle/" not in txt, f
