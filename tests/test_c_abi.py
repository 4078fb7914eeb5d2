"""The boundary is a C ABI: a plain C11 program compiles against the public
headers, links the library and gets the documented statuses (no GPU here:
process creation reports a CUDA error, argument errors come first)."""
import os
import shutil
import subprocess

import pytest

from paper_2510_05392_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SRC = r"""
#include <stdio.h>
#include <string.h>
#include "mgpu.h"
#include "mgpu_bench.h"
#include "mgpu_surrogate.h"

int main(void) {
    mg_process *p = NULL;
    /* argument errors are reported before any CUDA call */
    if (mg_process_create("g g > t t~ q", NULL, &p) != MG_ERR_BAD_PROCESS) return 1;
    mg_params par = {0.0, 1.4915, 0.118, MG_HEL_FILTERED, MG_FP64};
    if (mg_process_create("g g > t t~ g g", &par, &p) != MG_ERR_BAD_ARG) return 2;
    if (mg_sigmakin(NULL, NULL, 1, NULL, NULL) != MG_ERR_BAD_ARG) return 3;
    if (strcmp(mg_status_string(MG_ERR_NOT_FILTERED), "helicities not filtered") != 0) return 4;
    unsigned long long n = 0;
    if (mg_launch_count(&n) != MG_OK) return 5;
    /* a valid request: MG_OK with a GPU, MG_ERR_CUDA without one */
    int st = mg_process_create("g g > t t~ g g", NULL, &p);
    if (st == MG_OK) mg_process_destroy(p);
    printf("%d\n", st);
    return (st == MG_OK || st == MG_ERR_CUDA) ? 0 : 6;
}
"""


def test_plain_c_program_against_the_headers(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib = build.build()
    src = tmp_path / "abi.c"
    src.write_text(SRC)
    exe = tmp_path / "abi"
    libdir = os.path.dirname(lib)
    r = subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-o", str(exe), "-L", libdir, "-l:" + os.path.basename(lib),
                        "-Wl,-rpath," + libdir], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)


def test_library_exports_every_declared_function():
    """Every function the public headers declare is exported by the built
    library."""
    import ctypes
    import re
    lib = ctypes.CDLL(build.build())
    names = set()
    for h in ("mgpu.h", "mgpu_bench.h", "mgpu_surrogate.h"):
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(mg_\w+)\s*\(", text))
    assert len(names) > 30
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
