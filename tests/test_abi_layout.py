"""The ctypes mirrors of the ABI's structs match include/kadabra.h: the size
of kadabra_config and kadabra_result and the offset of every field, as the C
compiler lays them out (CPU only; gcc compiles a small probe against the
header)."""

import ctypes
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _c_layout(struct, fields):
    lines = [
        "#include <stddef.h>",
        "#include <stdio.h>",
        '#include "kadabra.h"',
        "int main(void) {",
        f'  printf("size %zu\\n", sizeof({struct}));',
    ]
    for f in fields:
        lines.append(f'  printf("{f} %zu\\n", offsetof({struct}, {f}));')
    lines += ["  return 0;", "}"]
    d = tempfile.mkdtemp(prefix="kadabra_layout_")
    try:
        src = os.path.join(d, "probe.c")
        exe = os.path.join(d, "probe")
        with open(src, "w") as fh:
            fh.write("\n".join(lines) + "\n")
        subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    finally:
        shutil.rmtree(d, ignore_errors=True)
    return {k: int(v) for k, v in (line.split() for line in out.strip().splitlines())}


@pytest.mark.parametrize("name", ["kadabra_config", "kadabra_result"])
def test_struct_layout_matches_header(name):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_1604_08553_gb300 import kadabra as kd
    cls = getattr(kd, name)
    fields = [f for f, _ in cls._fields_]
    c = _c_layout(name, fields)
    assert c["size"] == ctypes.sizeof(cls), (name, c["size"], ctypes.sizeof(cls))
    for f in fields:
        assert c[f] == getattr(cls, f).offset, (name, f, c[f], getattr(cls, f).offset)
