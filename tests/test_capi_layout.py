"""Every struct the ctypes binding mirrors has the same size and field offsets as in
include/eat.h: a C program generated from the binding's field lists prints sizeof and
offsetof for each, compiled with gcc (no GPU needed)."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_1912_00966_gb300 import eat

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = ["eat_connections", "eat_build_opts", "eat_csr_input", "eat_stats", "eat_net_view",
           "eat_counters", "eat_query_opts", "eat_server_opts", "eat_server_result",
           "eat_server_stats", "eat_ladder_stats", "eat_ladder_view"]


def test_binding_structs_match_the_header(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "eat.h"', "int main(void) {"]
    want = []
    for name in STRUCTS:
        cls = getattr(eat, name)
        lines.append(f'    printf("{name} sizeof %zu\\n", sizeof({name}));')
        want.append(f"{name} sizeof {ctypes.sizeof(cls)}")
        for field, _ in cls._fields_:
            lines.append(f'    printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
            want.append(f"{name} {field} {getattr(cls, field).offset}")
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe)], check=True)
    got = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    assert [g for g in got if g] == want
