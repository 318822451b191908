"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every entry point include/*.h declares (no compute calls here)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        names |= set(re.findall(r"\b(jpsi_\w+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    import paper_1810_11966_gb300 as jp
    lib = jp.load(build_if_missing=True)
    names = declared_symbols()
    assert {"jpsi_create", "jpsi_run_plain", "jpsi_run", "jpsi_destroy"} <= names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(jp.EXPORTS) == names


def test_checked_build_exports_the_same_symbols():
    # the bounds-checked build that the GPU tests run the parity suites on
    import paper_1810_11966_gb300.build as b
    b.build()
    lib = ctypes.CDLL(b.LIB_CHECKED)
    missing = [n for n in sorted(declared_symbols()) if not hasattr(lib, n)]
    assert not missing, missing
    log = open(os.path.join(b.BUILD, "jpsi_kernels_checked.log")).read()
    assert "-DJPSI_CHECKED=1" in log.splitlines()[0]


def test_strerror_without_gpu():
    import paper_1810_11966_gb300 as jp
    lib = jp.load(build_if_missing=True)
    assert lib.jpsi_strerror(0) == b"ok"
    assert lib.jpsi_strerror(3) == b"triplet buffer too small"


def test_struct_layouts_match_header(tmp_path):
    # the binding's ctypes structs against the C header, field by field: a C
    # program built with gcc from include/jpsi.h prints sizes and offsets
    import subprocess
    import paper_1810_11966_gb300 as jp
    structs = {"jpsi_params": jp.jpsi_params, "jpsi_batch": jp.jpsi_batch, "jpsi_outputs": jp.jpsi_outputs,
               "jpsi_timing": jp.jpsi_timing, "jpsi_tuning": jp.jpsi_tuning, "jpsi_timeslice": jp.jpsi_timeslice}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "jpsi.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.check_call(["gcc", "-I", inc, str(src), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)]).decode().splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, (name, f)


def test_built_for_sm103a():
    import paper_1810_11966_gb300.build as b
    b.build()
    log = open(os.path.join(b.BUILD, "jpsi_kernels.log")).read()
    assert "compute_103a" in log and "sm_103a" in log
