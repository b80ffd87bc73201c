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
int main(void) { printf("%zu %zu %zu %zu %zu\n", sizeof(pinv_config), sizeof(pinv_desc), sizeof(pinv_info),
                        sizeof(pinv_precond_desc), sizeof(pinv_serving_counters)); return 0; }
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        exe = os.path.join(d, "s")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    assert [int(x) for x in out] == [ctypes.sizeof(_lib.Config), ctypes.sizeof(_lib.Desc),
                                     ctypes.sizeof(_lib.Info), ctypes.sizeof(_lib.PrecondDesc),
                                     ctypes.sizeof(_lib.ServingStats)]


def test_every_field_offset_matches_the_header():
    """offsetof of each field of the public structs, compiled against the header,
    equals the binding's ctypes layout (a reordered or retyped field that keeps
    the struct size would otherwise pass the size check)."""
    import subprocess
    import tempfile
    structs = {"pinv_config": _lib.Config, "pinv_desc": _lib.Desc, "pinv_info": _lib.Info,
               "pinv_precond_desc": _lib.PrecondDesc, "pinv_serving_counters": _lib.ServingStats}
    lines = []
    for cname, cls in structs.items():
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    src = "#include <stdio.h>\n#include <stddef.h>\n#include \"pinv.h\"\nint main(void) {\n" + \
          "\n".join(lines) + "\nreturn 0; }\n"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "o.c")
        exe = os.path.join(d, "o")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(l.split() for l in out if l.strip())
    for cname, cls in structs.items():
        for fname, _ in cls._fields_:
            assert int(got[f"{cname}.{fname}"]) == getattr(cls, fname).offset, (cname, fname)


def test_header_is_strict_c99_and_cxx():
    """pinv.h is a plain C header: it compiles warning-free as pedantic C99 and
    as C++ (the extern "C" block), with a call of every entry point type-checked."""
    import subprocess
    import tempfile
    body = """
#include "pinv.h"
int use(void) {
    pinv_handle *h = 0; pinv_desc d; pinv_info info; pinv_precond_desc p; uint64_t id = 0;
    int ix = 0, ranks[4], co = 0; double a = 0.0;
    int r = pinv_init(&h, 0);
    r |= pinv_solve(h, &d, 0, &info) | pinv_solve_complex(h, &d, 0, &info);
    r |= pinv_preconditioner(h, &p, 0, &info) | pinv_solve_batched(h, 1, &d, 0, &info);
    r |= pinv_submit(h, &d, &id) | pinv_poll(h, id, &info) | pinv_alpha_estimate(h, &d, 0, &a);
    r |= pinv_step(h, 1, 1, 0, 1, 0, 0, 1, PINV_PREC_FP64, 0, 0, &a);
    r |= pinv_gemm(h, 1, 1, 1, 0, 1, 0, 0, 1, 0, 0, 1, PINV_PREC_FP64, 0);
    r |= pinv_drazin_index(h, 1, 0, 1, 2, 0, &ix, ranks) | pinv_autotune(h, 0, &co);
    r |= pinv_step_noalloc(1, 1, 0, 1, 0, 0, 1, 0, 0, &a);
    { pinv_serving_counters st; r |= pinv_serving_stats(h, &st) | pinv_set_wait_limit(h, 0u); }
    pinv_destroy(h);
    return r;
}
"""
    with tempfile.TemporaryDirectory() as d:
        for lang, compiler, flags, ext in (("c", "gcc", ["-std=c99"], "c"), ("c++", "g++", ["-std=c++11"], "cpp")):
            src = os.path.join(d, f"u.{ext}")
            open(src, "w").write(body)
            subprocess.run([compiler] + flags + ["-Wall", "-Wextra", "-Werror", "-pedantic",
                                                 "-Wno-unused-parameter", "-Wno-maybe-uninitialized",
                                                 "-Wno-uninitialized", "-I", os.path.dirname(HEADER),
                                                 "-c", src, "-o", os.path.join(d, f"u_{ext}.o")], check=True)


def test_binding_enum_codes_match_the_header():
    """The binding's name -> code tables equal the header's enum constants,
    compiled against the header (a renumbered or added constant would
    otherwise reach the library as another choice)."""
    import subprocess
    import tempfile
    names = {
        "KIND": {"moore_penrose": "PINV_MOORE_PENROSE", "drazin": "PINV_DRAZIN", "outer_g": "PINV_OUTER_G",
                 "drazin_normal": "PINV_DRAZIN_NORMAL"},
        "STOP": {"rel_fro": "PINV_STOP_REL_FRO", "paper": "PINV_STOP_PAPER", "order18": "PINV_STOP_ORDER18"},
        "PREC": {"fp64": "PINV_PREC_FP64", "mixed_bf16": "PINV_PREC_MIXED_BF16", "mixed_fp8": "PINV_PREC_MIXED_FP8",
                 "fp32": "PINV_PREC_FP32", "fp64_tc": "PINV_PREC_FP64_TC", "bf16_fp32": "PINV_PREC_BF16_FP32",
                 "fp32_refine": "PINV_PREC_FP32_REFINE"},
        "VARIANT": {"plain": "PINV_VARIANT_PLAIN", "stabilized": "PINV_VARIANT_STABILIZED"},
        "FINISH": {"none": "PINV_FINISH_NONE", "clean": "PINV_FINISH_CLEAN"},
    }
    consts = [c for table in names.values() for c in table.values()]
    src = "#include <stdio.h>\n#include \"pinv.h\"\nint main(void) {\n"
    src += "".join(f'    printf("%d\\n", (int){c});\n' for c in consts) + "    return 0;\n}\n"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "e.c")
        exe = os.path.join(d, "e")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        vals = [int(x) for x in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    header = dict(zip(consts, vals))
    for table, m in names.items():
        binding = getattr(_lib, table)
        for key, const in m.items():
            assert binding[key] == header[const], (table, key)
    # every code the binding offers is one the header names
    assert set(_lib.PREC) == set(names["PREC"])
