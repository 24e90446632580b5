"""The C-ABI library builds, loads without a GPU, exports every function that
include/pdlp.h declares, and the ctypes structures match the C layouts."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2312_14832_b300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pdlp.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return C.CDLL(build.LIB)


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pdlp_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("pdlp_setup", "pdlp_solve", "pdlp_free", "pdlp_default_params", "pdlp_last_error"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert names
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(_lib.SIGNATURES), "ctypes signatures and header differ"


def test_struct_layouts_match_header(tmp_path):
    prog = tmp_path / "sizes.c"
    prog.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "pdlp.h"
int main(void) {
  printf("%zu %zu %zu %zu\\n", sizeof(pdlp_params), sizeof(pdlp_result), sizeof(pdlp_check_record),
         sizeof(pdlp_info));
  printf("%zu %zu %zu %zu\\n", offsetof(pdlp_params, stream), offsetof(pdlp_params, log_capacity),
         offsetof(pdlp_result, launches), offsetof(pdlp_info, norm_K));
  return 0;
}
""")
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(prog)])
    out = subprocess.check_output([str(exe)]).decode().split()
    want = [C.sizeof(_lib.Params), C.sizeof(_lib.Result), C.sizeof(_lib.CheckRecord), C.sizeof(_lib.Info),
            _lib.Params.stream.offset, _lib.Params.log_capacity.offset, _lib.Result.launches.offset,
            _lib.Info.norm_K.offset]
    assert list(map(int, out)) == want


def test_default_params_without_gpu(lib):
    import paper_2312_14832_b300 as pk
    p = pk.default_params()
    assert p.tol == 1e-4 and p.check_every == 64 and p.beta_suff == 0.2 and p.beta_nec == 0.8
    assert p.beta_art == 0.36 and p.step_scale == 0.9 and p.ruiz_iters == 10


def test_last_error_null_handle(lib):
    """With a null handle pdlp_last_error gives the calling thread's last setup error: here
    that of a setup rejected before any device work (null output handle)."""
    f = lib.pdlp_last_error
    f.restype = C.c_char_p
    f.argtypes = [C.c_void_p]
    setup = lib.pdlp_setup
    setup.restype = C.c_int
    setup.argtypes = [C.c_void_p] + [C.c_int64] * 3 + [C.c_void_p] * 8
    assert setup(None, 1, 1, 0, None, None, None, None, None, None, None, None) == -1
    assert f(None) == b"null output handle"
