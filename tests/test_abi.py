"""The C-ABI library builds, loads, and exports every symbol include/imrt.h declares (no GPU calls)."""
import ctypes
import os
import re

from paper_0908_4421_gb300 import _lib
from paper_0908_4421_gb300 import build as cuda_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b([a-z_][a-z0-9_]*)\s*\(", text)) - {"if", "sizeof"}
    return names


def test_library_exports_every_declared_symbol():
    path = cuda_build.build()
    lib = ctypes.CDLL(path)
    declared = declared_functions()
    assert {"plan_create", "plan_solve", "plan_dose", "plan_destroy"} <= declared
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(_lib.EXPORTS) == declared


def test_version_and_defaults_without_gpu():
    lib = _lib.load(cuda_build.build())
    assert lib.imrt_version().decode().startswith("imrt-gb300")
    o = _lib.imrt_options()
    lib.imrt_default_options(ctypes.byref(o))
    assert (o.eps, o.alpha, o.delta, o.max_iter, o.max_backtracks, o.k_trials) == (1e-4, 2.0, 1e-6, 200, 50, 1)


def test_struct_layouts_match_header(tmp_path):
    """Every ctypes field offset equals the C compiler's offsetof for the header's structs."""
    import subprocess
    structs = [_lib.imrt_csr, _lib.imrt_options, _lib.imrt_result, _lib.imrt_plan_info]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "imrt.h"', "int main(void) {"]
    for st in structs:
        name = st.__name__
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in st._fields_:
            lines.append(f'printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    expect = []
    for st in structs:
        expect.append(f"{st.__name__} size {ctypes.sizeof(st)}")
        for f, _ in st._fields_:
            expect.append(f"{st.__name__} {f} {getattr(st, f).offset}")
    assert [l for l in out if l] == expect


def test_every_declaration_is_documented():
    """Each function the header declares is preceded by its comment (arguments, layout,
    ownership and errors are stated there)."""
    text = open(os.path.join(ROOT, "include", "imrt.h")).read()
    decls = list(re.finditer(r"^(?:imrt_status|void|const char\*|int32_t)\s+(\w+)\s*\(", text, re.M))
    assert {m.group(1) for m in decls} == declared_functions()
    undocumented = [m.group(1) for m in decls if not text[:m.start()].rstrip().endswith("*/")]
    assert not undocumented, undocumented


def test_python_options_mirror_the_c_defaults_and_fields():
    """Options (Python) and imrt_options (C) have the same fields and the same defaults, and
    Result covers every field of imrt_result."""
    import dataclasses

    from paper_0908_4421_gb300.api import Options, Result
    lib = _lib.load(cuda_build.build())
    c = _lib.imrt_options()
    lib.imrt_default_options(ctypes.byref(c))
    c_fields = {name for name, _ in _lib.imrt_options._fields_}
    py = Options()
    assert {f.name for f in dataclasses.fields(Options)} == c_fields
    for f in dataclasses.fields(Options):  # a NULL pointer (the stream) reads back as None
        assert getattr(py, f.name) == (getattr(c, f.name) or 0), f.name
    custom = Options(eps=0.25, alpha=3.0, lambda0=0.5, delta=1e-3, max_iter=7, max_backtracks=9, x_init=2,
                     precision=_lib.FP16, k_trials=4, mode=_lib.MODE_HOST, profile=1, trace=2, polish_iter=5,
                     kernel_variant=2, timeout_ms=12.5, stream=1234)
    back = custom.to_c()
    for f in dataclasses.fields(Options):
        assert getattr(back, f.name) == getattr(custom, f.name), f.name
    assert {f.name for f in dataclasses.fields(Result)} == {name for name, _ in _lib.imrt_result._fields_}
