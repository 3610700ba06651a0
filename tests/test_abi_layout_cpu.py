"""The Python binding's mirrors of the C structs have the header's layout.

A small C program is compiled against include/kmer_analysis.h with the host
compiler and prints sizeof and the offset of every field of every struct the
binding mirrors (ctypes structures, and the numpy dtype of kmer_record); the
binding must agree field by field.  A struct grown on one side only (a field
appended to the stats, say) would otherwise let the library write past the
Python object."""
import ctypes
import os
import shutil
import subprocess

import pytest

import paper_1809_07014_gb300 as pkg

HERE = os.path.dirname(os.path.abspath(__file__))
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

STRUCTS = ["kmer_analysis_params", "kmer_result_view", "kmer_analysis_stats", "kmer_contigs_view",
           "kmer_batch_job", "kmer_batch_stats", "kmer_request_info", "kmer_server_stats"]


def c_layouts(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no host C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "kmer_analysis.h"', "int main(void) {"]
    for s in STRUCTS:
        lines.append(f'  printf("{s} sizeof %zu\\n", sizeof({s}));')
        for f, _ in getattr(pkg, s)._fields_:
            lines.append(f'  printf("{s} {f} %zu\\n", offsetof({s}, {f}));')
    lines.append('  printf("kmer_record sizeof %zu\\n", sizeof(kmer_record));')
    for f in pkg.KMER_RECORD_DTYPE.names:
        lines.append(f'  printf("kmer_record {f} %zu\\n", offsetof(kmer_record, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", INCLUDE, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        name, field, value = line.split()
        layout[(name, field)] = int(value)
    return layout


def test_ctypes_mirrors_match_the_header(tmp_path):
    layout = c_layouts(tmp_path)
    for s in STRUCTS:
        cls = getattr(pkg, s)
        assert ctypes.sizeof(cls) == layout[(s, "sizeof")], s
        for f, _ in cls._fields_:
            assert getattr(cls, f).offset == layout[(s, f)], (s, f)
    dt = pkg.KMER_RECORD_DTYPE
    assert dt.itemsize == layout[("kmer_record", "sizeof")]
    for f in dt.names:
        assert dt.fields[f][1] == layout[("kmer_record", f)], f
