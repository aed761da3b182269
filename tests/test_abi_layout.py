"""The ctypes mirrors of the public structs in include/newton3p.h have the C
layout: every field's offset and every struct's size, read from a small C
program compiled against the header (no GPU, no library call)."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2307_16051_gb300 import nl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MIRRORS = {"nl_config": nl.Config, "nl_stats_t": nl.Stats, "nl_batch_info_t": nl.BatchInfo,
           "nl_server_config": nl.ServerConfig, "nl_request_info_t": nl.RequestInfo,
           "nl_server_info_t": nl.ServerInfo}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    d = tmp_path_factory.mktemp("abi")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "newton3p.h"', "int main(void) {"]
    for cname, py in MIRRORS.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in py._fields_:
            lines.append(f'  printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines += ["  return 0;", "}"]
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    table = {}
    for line in out.splitlines():
        s, f, v = line.split()
        table[(s, f)] = int(v)
    return table


@pytest.mark.parametrize("cname", list(MIRRORS))
def test_struct_layout_matches_header(c_layout, cname):
    py = MIRRORS[cname]
    assert c_layout[(cname, "size")] == ctypes.sizeof(py), cname
    for f in py._fields_:
        assert c_layout[(cname, f[0])] == getattr(py, f[0]).offset, (cname, f[0])

