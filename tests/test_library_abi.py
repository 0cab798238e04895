"""CPU checks of the C ABI library: it builds, loads without a GPU and exports
every function include/bigmeans.h declares; the binding declares the same set."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "bigmeans.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:bm_status|void|int32_t|const char\*)\s+(\w+)\s*\(", src, flags=re.M)
    return set(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2403_18766_gb300 import build
    build.build()
    import ctypes
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("bigmeans_fit", "bigmeans_fit_host", "bm_sample", "bm_gather", "bm_kmeanspp",
              "bm_lloyd", "bm_assign", "bm_last_error", "bm_fit_create", "bm_fit_rounds",
              "bm_fit_finish", "bm_fit_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_the_header(lib):
    from paper_2403_18766_gb300 import native
    assert set(native.SIGNATURES) == _declared()
    assert native.version().startswith("bigmeans-gb300")


def test_struct_layouts_match_c(tmp_path):
    """Every field offset and struct size of the binding equals what the C
    compiler makes of include/bigmeans.h."""
    import ctypes
    import shutil
    import subprocess
    from paper_2403_18766_gb300 import native
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"bm_sample_policy": native.SamplePolicy, "bm_budget": native.Budget, "bm_report": native.Report,
               "bm_job": native.Job, "bm_result": native.JobResult, "bm_ctx_info": native.CtxInfo}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "bigmeans.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_errors_without_gpu_are_status_codes(lib):
    from paper_2403_18766_gb300 import native
    # argument checks happen before any CUDA call
    st = native.lib.bm_sample(1, 3, 0, 0, 0, 10, 11, None, None)
    assert st == native.BM_EINVAL
    assert b"out of range" in native.lib.bm_last_error()
