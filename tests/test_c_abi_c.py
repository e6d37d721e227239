"""The C ABI from plain C, without a GPU: include/mgard.h compiles as strict
C99 and as C++17, and a C program linked against the library gets status
codes and messages from the calls that fail before touching a device."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")

C_PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "mgard.h"

int main(void)
{
    int64_t bad[2] = {10, 10};          /* 9 is not divisible by 2 */
    mgard_plan *plan = (mgard_plan *)1;
    mgard_status st = mgard_plan_create(2, bad, 1, NULL, MGARD_F32, &plan);
    if (st != MGARD_ERR_UNSUPPORTED_SHAPE || plan != NULL) return 1;
    if (strstr(mgard_last_error(), "divisible") == NULL) return 2;
    if (mgard_plan_create(2, bad, 1, NULL, MGARD_F32, NULL) != MGARD_ERR_INVALID_ARG) return 8;
    if (strcmp(mgard_status_string(MGARD_ERR_WORKSPACE), "MGARD_ERR_WORKSPACE") != 0) return 3;
    if (mgard_decompose(NULL, NULL, NULL, 0, NULL) != MGARD_ERR_INVALID_ARG) return 4;
    if (mgard_recompose_classes(NULL, 1, NULL, NULL, 0, NULL) != MGARD_ERR_INVALID_ARG) return 5;
    if (mgard_workspace_bytes(NULL) != 0 || mgard_plan_levels(NULL) != -1) return 6;
    if (mgard_plan_destroy(NULL) != MGARD_OK) return 7;
    /* every entry point rejects a NULL plan or batch before touching a device */
    if (mgard_recompose(NULL, NULL, NULL, 0, NULL) != MGARD_ERR_INVALID_ARG) return 9;
    if (mgard_decompose_adjoint(NULL, NULL, NULL, 0, NULL) != MGARD_ERR_INVALID_ARG) return 10;
    if (mgard_recompose_adjoint(NULL, NULL, NULL, 0, NULL) != MGARD_ERR_INVALID_ARG) return 11;
    if (mgard_decompose_host(NULL, NULL, NULL, NULL, NULL, 0, NULL) != MGARD_ERR_INVALID_ARG) return 12;
    if (mgard_plan_tune(NULL, 0, 0, 0) != MGARD_ERR_INVALID_ARG) return 13;
    if (mgard_plan_get_tune(NULL, 0, 0) != -1 || mgard_plan_launches(NULL, 0) != -1) return 14;
    if (mgard_plan_check(NULL, NULL, NULL) != MGARD_ERR_INVALID_ARG) return 15;
    if (mgard_profile_enable(NULL, 1) != MGARD_ERR_INVALID_ARG) return 16;
    if (mgard_profile_read(NULL, 0, NULL, NULL, NULL, NULL) != -1) return 17;
    {
        mgard_batch *b = (mgard_batch *)1;
        if (mgard_batch_create(0, NULL, 1, &b) != MGARD_ERR_INVALID_ARG || b != NULL) return 18;
        if (mgard_batch_decompose(NULL, NULL, NULL, 0, NULL) != MGARD_ERR_INVALID_ARG) return 19;
        if (mgard_batch_workspace_bytes(NULL) != 0 || mgard_batch_destroy(NULL) != MGARD_OK) return 20;
    }
    if (mgard_decompose_noalloc(2, bad, 1, MGARD_F32, NULL, NULL) != MGARD_ERR_INVALID_ARG) return 21;
    printf("ok %d\n", (int)MGARD_NOALLOC_SCRATCH_BYTES);
    return 0;
}
"""


def _cc():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    return cc


def test_header_compiles_as_c99_and_cxx17(tmp_path):
    cc = _cc()
    src = tmp_path / "h.c"
    src.write_text('#include "mgard.h"\nint f(void) { return (int)MGARD_OK; }\n')
    subprocess.run([cc, "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror", "-I", INCLUDE,
                    "-c", str(src), "-o", str(tmp_path / "h.o")], check=True)
    cxx = shutil.which("g++")
    if cxx:
        srcpp = tmp_path / "h.cpp"
        srcpp.write_text('#include "mgard.h"\nint f() { return (int)MGARD_OK; }\n')
        subprocess.run([cxx, "-std=c++17", "-Wall", "-Wextra", "-Werror", "-I", INCLUDE,
                        "-c", str(srcpp), "-o", str(tmp_path / "hpp.o")], check=True)


def test_c_program_links_and_gets_status_codes(tmp_path):
    from paper_2007_04457_gb300 import build as gbuild

    cc = _cc()
    lib = gbuild.build()
    libdir, libfile = os.path.split(lib)
    src = tmp_path / "prog.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "prog"
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", INCLUDE, str(src), "-o", str(exe),
                    os.path.join(libdir, libfile), f"-Wl,-rpath,{libdir}"], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.startswith("ok ")
