"""The C-ABI library builds, loads and exports every function include/cswgs.h
declares, and the binding's ctypes layouts match the C structs.  No GPU: only
calls that touch no device are made."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cswgs.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(cswgs_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2003_05293_gb300 import capi
    return capi.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("cswgs_plan_create", "cswgs_plan_destroy", "cswgs_solve", "cswgs_solve_ex",
                 "cswgs_subset", "cswgs_batch_create", "cswgs_batch_run", "cswgs_submit",
                 "cswgs_poll", "cswgs_cancel", "cswgs_status_string"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2003_05293_gb300 import capi
    assert sorted(capi.SIGNATURES) == declared_functions()


def test_exports_are_c_symbols():
    from paper_2003_05293_gb300 import capi
    out = subprocess.run(["nm", "-D", "--defined-only", capi.library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (cswgs_[a-z0-9_]+)$", out, flags=re.M))
    assert set(declared_functions()) <= exported


def test_host_only_calls(lib):
    assert lib.cswgs_abi_version() == 2
    assert lib.cswgs_status_string(0) == b"ok"
    assert lib.cswgs_status_string(1) == b"invalid argument"
    from paper_2003_05293_gb300 import capi
    d = capi.cswgs_plan_desc()
    lib.cswgs_plan_desc_default(ctypes.byref(d))
    assert (d.device, d.max_P, d.max_N, d.max_batch, d.precision) == (0, 2048, 1024, 64, 1)
    o = capi.cswgs_solve_opts()
    lib.cswgs_solve_opts_default(ctypes.byref(o))
    assert (o.full_iterations, o.first_iteration, o.final_pass) == (2, 1, 1)
    assert (o.pupil.aperture, o.pupil.subset_mode, o.pupil.beam_waist) == (0, 0, 0.0) and not o.slm
    # NULL arguments are refused before any device work
    assert lib.cswgs_plan_create(None, None) == capi.CSWGS_EINVAL
    assert lib.cswgs_solve(None, None, None, 1, 8, 0.5, 1, 0, None, 0, None, None) == capi.CSWGS_EINVAL
    assert b"NULL" in lib.cswgs_last_error()


def test_struct_layouts_match_header(tmp_path):
    from paper_2003_05293_gb300 import capi
    src = tmp_path / "sz.c"
    src.write_text('#include "cswgs.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                   "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n\","
                   "sizeof(cswgs_plan_desc), sizeof(cswgs_solve_opts), sizeof(cswgs_request),"
                   "sizeof(cswgs_result), sizeof(cswgs_serve_stats),"
                   "offsetof(cswgs_request, phase_out), offsetof(cswgs_plan_desc, tune_cache),"
                   "sizeof(cswgs_pupil), sizeof(cswgs_slm_frame), offsetof(cswgs_request, slm),"
                   "offsetof(cswgs_slm_frame, levels));return 0;}\n")
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(capi.cswgs_plan_desc), ctypes.sizeof(capi.cswgs_solve_opts),
            ctypes.sizeof(capi.cswgs_request), ctypes.sizeof(capi.cswgs_result),
            ctypes.sizeof(capi.cswgs_serve_stats), capi.cswgs_request.phase_out.offset,
            capi.cswgs_plan_desc.tune_cache.offset, ctypes.sizeof(capi.cswgs_pupil),
            ctypes.sizeof(capi.cswgs_slm_frame), capi.cswgs_request.slm.offset,
            capi.cswgs_slm_frame.levels.offset]
    assert got == want
