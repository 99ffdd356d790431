"""The ctypes mirrors of the C-ABI structs in paper_1510_03298_gb300/__init__.py have the layout
the C compiler gives the structs of include/glam.h: the same size, and every field at the same
offset.  A mismatch would make the binding read or write the wrong bytes of glam_opts,
glam_stats or glam_batch_item without any error.  A small C program prints sizeof and offsetof
as the host compiler lays the structs out (no GPU and no library call)."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _mirrors():
    import paper_1510_03298_gb300 as g
    return [("glam_dims", g.GlamDims), ("glam_quad", g.GlamQuadC), ("glam_opts", g.GlamOpts),
            ("glam_stats", g.GlamStats), ("glam_batch_item", g.GlamBatchItem)]


def _c_name(field):
    # the binding appends "_" where the C name is a Python keyword
    return field[:-1] if field.endswith("_") else field


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "glam.h"', 'int main(void) {']
    for cname, S in _mirrors():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f in S._fields_:
            lines.append(f'  printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {_c_name(f[0])}));')
    lines += ['  return 0;', '}']
    d = tmp_path_factory.mktemp("abi_layout")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-O0", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    table = {}
    for line in out.splitlines():
        struct, key, val = line.split()
        table[(struct, key)] = int(val)
    return table


@pytest.mark.parametrize("i", range(5))
def test_ctypes_mirror_matches_the_c_struct(c_layout, i):
    cname, S = _mirrors()[i]
    assert C.sizeof(S) == c_layout[(cname, "sizeof")], cname
    for f in S._fields_:
        assert getattr(S, f[0]).offset == c_layout[(cname, f[0])], (cname, f[0])
