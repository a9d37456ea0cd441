"""CPU-side checks of the C ABI boundary: the library builds for sm_103a, loads, and
exports every entry point include/sgeo.h declares; the product package never touches the
oracle."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sgeo.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sg_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    import paper_2603_15780_gb300 as sg
    L = sg.lib()
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(L, n), f"libsgeo.so does not export {n}"
    assert set(names) == set(sg.EXPORTED)


def test_defaults_and_status_strings():
    import paper_2603_15780_gb300 as sg
    o = sg.default_opts()
    assert o.max_steps == 1 << 20 and o.block == 256 and o.fp64_escalate == 1
    assert abs(o.tau_near - 1e-4) < 1e-9 and o.tau_snap == 0.0 and o.precision == 0  # snap: 1e-6 (FP32, mixed) / 1e-12 (FP64); precision: automatic
    assert sg.lib().sg_status_string(2) == b"non-manifold mesh"
    assert sg.lib().sg_version().startswith(b"sgeo")


def test_null_arguments_rejected_without_gpu_work():
    import paper_2603_15780_gb300 as sg
    L = sg.lib()
    out = C.c_void_p()
    assert L.sg_mesh_create(None, 3, None, 1, C.byref(out)) == 1
    o = sg.default_opts()
    assert L.sg_exp_map(None, 1, None, None, None, None, None, 0, *([None] * 9), C.byref(o), None) == 1
    assert L.sg_exp_map_backward(None, 0, 1e-4, 1e-4, 1, *([None] * 11), 0, *([None] * 7), C.byref(o), None) == 1
    assert L.sg_exp_map_trace(None, 1, None, None, None, None, None, 8, *([None] * 10), C.byref(o), None) == 1
    assert L.sg_mesh_update_vertices(None, None, None) == 1
    assert L.sg_transport_back(None, 1, *([None] * 7), 1, None, None, C.byref(o), None) == 1
    n = C.c_size_t()
    assert L.sg_exp_map_workspace_size(None, 1, None, C.byref(n)) == 1


def test_product_code_does_not_reference_the_oracle():
    pkg = os.path.join(ROOT, "paper_2603_15780_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "om_" not in txt, f


def test_header_is_plain_c_and_cxx():
    """include/sgeo.h is a C-ABI header: it compiles alone as C99 and as C++11, with no torch or
    CUDA headers."""
    import shutil
    import subprocess
    hdr = os.path.join(ROOT, "include", "sgeo.h")
    for cc, lang, std in (("gcc", "c", "-std=c99"), ("g++", "c++", "-std=c++11")):
        if shutil.which(cc) is None:
            pytest.skip(f"{cc} not available")
        subprocess.check_call([cc, "-fsyntax-only", std, "-Wall", "-Werror", "-x", lang, hdr])


def test_opts_mirror_matches_the_header():
    """The binding's ctypes mirror of sg_opts has the header's size and field offsets."""
    import shutil
    import subprocess
    import tempfile
    import paper_2603_15780_gb300 as sg
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    fields = [f for f, _ in sg.Opts._fields_]
    src = '#include <stdio.h>\n#include <stddef.h>\n#include "sgeo.h"\nint main(void) {\n'
    src += '    printf("%zu\\n", sizeof(sg_opts));\n'
    src += "".join(f'    printf("%zu\\n", offsetof(sg_opts, {f}));\n' for f in fields) + "    return 0;\n}\n"
    with tempfile.TemporaryDirectory() as d:
        c, exe = os.path.join(d, "o.c"), os.path.join(d, "o")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        got = [int(x) for x in subprocess.check_output([exe]).split()]
    assert got[0] == C.sizeof(sg.Opts)
    assert got[1:] == [getattr(sg.Opts, f).offset for f in fields]
    assert not sg.default_opts().order   # no order buffer unless the caller gives one
