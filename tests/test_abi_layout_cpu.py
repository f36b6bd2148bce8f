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
