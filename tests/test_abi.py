"""CPU checks of the C ABI: the library builds, loads, and exports every entry
point the header declares (no device calls)."""

import ctypes
import os
import re

from paper_1604_07893_gb300 import build as B
from paper_1604_07893_gb300 import _lib

HEADER = os.path.join(B.ROOT, "include", "pinv.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pinv_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pinv_init", "pinv_solve", "pinv_solve_batched", "pinv_submit", "pinv_poll"):
        assert required in names
    assert set(names) == set(_lib.EXPORTS)


def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_struct_sizes_match_the_header():
    """Compile a tiny C program against the header and compare sizeof with ctypes."""
    import subprocess
    import tempfile
    src = r'''
#include <stdio.h>
#include "pinv.h"
int main(void) { printf("%zu %zu %zu %zu\n", sizeof(pinv_config), sizeof(pinv_desc), sizeof(pinv_info),
                        sizeof(pinv_precond_desc)); return 0; }
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        exe = os.path.join(d, "s")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    assert [int(x) for x in out] == [ctypes.sizeof(_lib.Config), ctypes.sizeof(_lib.Desc),
                                     ctypes.sizeof(_lib.Info), ctypes.sizeof(_lib.PrecondDesc)]
