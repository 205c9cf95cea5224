"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/ms.h declares (no compute calls here)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ms.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"MS_API\s+[\w\s\*]+?\b(ms_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no nvcc")
    from paper_2007_14283_gb300 import build
    return build.build()


def test_header_declares_the_boundary_calls():
    names = _declared()
    for required in ("ms_create", "ms_seed_batch", "ms_iterate", "ms_merge_modes", "ms_label",
                     "ms_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_the_header(libpath):
    import paper_2007_14283_gb300 as ms
    ms.load(libpath)
    for n in _declared():
        assert hasattr(ms, n), n


def test_config_defaults_are_the_papers(libpath):
    import paper_2007_14283_gb300 as ms
    ms.load(libpath)
    c = ms.ms_config_default()
    assert (c.bandwidth_cos, c.gamma, c.n_initial, c.L, c.H, c.P_target) == (0.9, 0.9, 128, 2.0, 8.0, 0.99)
    assert c.tol == 1e-6 and c.merge_cos == 0.9 and c.precision == ms.MS_FP32


def test_invalid_config_rejected_without_gpu(libpath):
    import paper_2007_14283_gb300 as ms
    ms.load(libpath)
    c = ms.ms_config_default(dim=0)
    with pytest.raises(ms.MsError) as e:
        ms.ms_workspace_bytes(c, 100)
    assert e.value.status == ms.MS_ERR_INVALID_ARG


def test_kernels_compiled_for_sm103a(libpath):
    # the build passes exactly one -gencode for sm_103a
    from paper_2007_14283_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


C_PROGRAM = r"""
#include <stdio.h>
#include "ms.h"
int main(void) {
    ms_config c;
    int64_t bytes = 0;
    ms_status s;
    ms_config_default(&c);
    if (c.dim != 16 || c.n_initial != 128) return 2;
    c.dim = 0;
    s = ms_workspace_bytes(&c, 100, &bytes);
    printf("%s\n", ms_last_error());
    return s == MS_ERR_INVALID_ARG ? 0 : 1;
}
"""


def test_header_is_plain_c_and_links_from_c(libpath, tmp_path):
    # the boundary is a C ABI: the header compiles as strict C99 and a C
    # program links against the library and calls its host-side entry points
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    src = tmp_path / "main.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "main"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                    "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe), libpath,
                    "-Wl,-rpath," + os.path.dirname(libpath)], check=True, capture_output=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert "dim" in r.stdout
