"""The ctypes structures of the Python binding have the layout of the C
header's structs: same size, same field names, same offsets.  A C program
generated from the binding's field lists is compiled against
include/recsplit.h with the host compiler and prints sizeof and offsetof of
every field; a renamed or moved field fails to compile or to match."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_1910_06416_gb300 import recsplit as rs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "recsplit_stats_t": rs.Stats,
    "recsplit_profile_t": rs.Profile,
    "recsplit_keyset_t": rs.KeySet,
    "recsplit_server_config_t": rs.ServerConfig,
    "recsplit_completion_t": rs.Completion,
    "recsplit_server_stats_t": rs.ServerStats,
    "recsplit_tuning_t": rs.Tuning,
}


def c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("needs a host C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "recsplit.h"', "int main(void) {"]
    for cname, cls in STRUCTS.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    exe = tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        name, key, value = line.split()
        layout[(name, key)] = int(value)
    return layout


def test_binding_structs_match_the_header(tmp_path):
    layout = c_layout(tmp_path)
    for cname, cls in STRUCTS.items():
        assert layout[(cname, "size")] == C.sizeof(cls), cname
        for field, _ in cls._fields_:
            assert layout[(cname, field)] == getattr(cls, field).offset, (cname, field)


def header_prototypes():
    """name -> list of parameter type strings, from include/recsplit.h."""
    import re
    text = open(os.path.join(ROOT, "include", "recsplit.h")).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    protos = {}
    for m in re.finditer(r"\b(?:int|void|uint64_t|const char\s*\*)\s+(recsplit_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", text):
        args = " ".join(m.group(2).split())
        params = [] if args in ("", "void") else [a.strip() for a in args.split(",")]
        types = []
        for a in params:
            a = re.sub(r"\b[a-z_][a-z0-9_]*$", "", a).strip()  # drop the parameter name
            types.append(a)
        protos[m.group(1)] = types
    return protos


def ctype_of(decl):
    if "*" in decl:
        return "pointer"
    return {"uint64_t": C.c_uint64, "uint32_t": C.c_uint32, "int": C.c_int, "size_t": C.c_size_t,
            "int64_t": C.c_int64}[decl.replace("const ", "").strip()]


def test_binding_argtypes_match_the_prototypes():
    from paper_1910_06416_gb300 import build
    build.build()
    L = rs.lib()
    protos = header_prototypes()
    assert set(protos) == set(rs.header_functions())
    for name, types in protos.items():
        argtypes = getattr(L, name).argtypes
        assert argtypes is not None, name
        assert len(argtypes) == len(types), (name, types)
        for t, a in zip(types, argtypes):
            want = ctype_of(t)
            if want == "pointer":
                assert a is C.c_void_p or issubclass(a, C._Pointer) or a is C.c_char_p, (name, t, a)
            else:
                assert C.sizeof(a) == C.sizeof(want) and a(-1).value == want(-1).value, (name, t, a)
