"""The Python binding's ctypes structures against the C header, without a GPU:
a small C program compiled with gcc against include/vsz.h prints every
struct's size and every field's offset, and the ctypes definitions must
agree field by field."""
import ctypes
import os
import shutil
import subprocess

import pytest

import paper_2201_04614_gb300 as vsz
from paper_2201_04614_gb300 import shard

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = {
    "vsz_params": vsz._CParams,
    "vsz_header": vsz._CHeader,
    "vsz_compressed": vsz._CCompressed,
    "vsz_field_job": vsz._CFieldJob,
    "vsz_batch_class": vsz._CBatchClass,
    "vsz_trace_record": vsz._CTrace,
    "vsz_host_field": vsz._CHostField,
    "vsz_slab_stats": shard._SlabStats,
}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    d = tmp_path_factory.mktemp("abi")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "vsz.h"', "int main(void) {"]
    for cname, ct in STRUCTS.items():
        lines.append(f'    printf("{cname} . %zu\\n", sizeof({cname}));')
        for fname, _ in ct._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "layout"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    res = {}
    for line in out.splitlines():
        s, f, v = line.split()
        res[(s, f)] = int(v)
    return res


@pytest.mark.parametrize("cname", list(STRUCTS))
def test_ctypes_struct_matches_header(c_layout, cname):
    ct = STRUCTS[cname]
    assert ctypes.sizeof(ct) == c_layout[(cname, ".")], cname
    for fname, _ in ct._fields_:
        assert getattr(ct, fname).offset == c_layout[(cname, fname)], (cname, fname)

