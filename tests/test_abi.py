"""CPU-side checks of the C ABI: the library builds/loads, exports every symbol
include/ripple.h declares, and the ctypes structs match the C layout."""
import os
import re
import subprocess

import pytest

import paper_2104_08571_gb300 as R
from paper_2104_08571_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


def declared_symbols():
    names = set()
    for h in os.listdir(HEADER_DIR):
        if h.endswith(".h"):
            text = open(os.path.join(HEADER_DIR, h)).read()
            names |= set(re.findall(r"RIPPLE_API\s+[\w\s\*]+?\b(ripple_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return R.load()


def test_library_exports_every_declared_symbol(lib):
    decl = declared_symbols()
    assert len(decl) >= 15
    missing = [n for n in decl if not hasattr(lib, n)]
    assert not missing, missing
    assert set(R.exported_symbols()) <= decl


def test_binding_covers_every_declared_symbol():
    assert declared_symbols() == set(R.exported_symbols())


def test_struct_layouts_match_c(tmp_path):
    src = tmp_path / "sizes.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "ripple.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\\n", sizeof(ripple_fv_params), sizeof(ripple_fv_stats),
         sizeof(ripple_eik_params), sizeof(ripple_eik_stats), sizeof(ripple_field_desc));
  printf("%zu %zu %zu\\n", offsetof(ripple_fv_params, scheme), offsetof(ripple_field_desc, dims),
         offsetof(ripple_field_desc, current));
  printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(ripple_request), offsetof(ripple_request, fv),
         offsetof(ripple_request, nsrc), sizeof(ripple_ticket_info), sizeof(ripple_batch_config),
         sizeof(ripple_batch_stats), offsetof(ripple_batch_config, active_cells));
  return 0;
}
""")
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-I", HEADER_DIR, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    import ctypes
    want = [ctypes.sizeof(R.ripple_fv_params), ctypes.sizeof(R.ripple_fv_stats),
            ctypes.sizeof(R.ripple_eik_params), ctypes.sizeof(R.ripple_eik_stats),
            ctypes.sizeof(R.ripple_field_desc), R.ripple_fv_params.scheme.offset,
            R.ripple_field_desc.dims.offset, R.ripple_field_desc.current.offset,
            ctypes.sizeof(R.ripple_request), R.ripple_request.fv.offset, R.ripple_request.nsrc.offset,
            ctypes.sizeof(R.ripple_ticket_info), ctypes.sizeof(R.ripple_batch_config),
            ctypes.sizeof(R.ripple_batch_stats), R.ripple_batch_config.active_cells.offset]
    assert [int(x) for x in out] == want


def test_errors_are_reported_without_a_gpu(lib):
    # on a machine without a usable GPU the ABI returns a status, it never crashes
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(R.RippleError) as ei:
        R.ripple_ctx_create(0)
    assert ei.value.status in (R.RIPPLE_ERR_CUDA, R.RIPPLE_ERR_INVALID)
    assert R.ripple_last_error()


def test_null_handles_are_ok(lib):
    assert lib.ripple_field_destroy(None) == 0
    assert lib.ripple_ctx_destroy(None) == 0
    assert lib.ripple_fv_step(None, None, 1, None) == R.RIPPLE_ERR_INVALID
