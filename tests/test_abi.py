"""Host-side checks of the C ABI that need no GPU: the library builds, loads and exports
every entry point that include/pms.h declares, and the binding's structs match it."""

from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1307_0571_gb300 import build
    build.build()
    from paper_1307_0571_gb300 import pms
    return pms.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "pms.h")).read()
    return sorted(set(re.findall(r"\b(pms_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for want in ["pms_solve", "pms_solve_batch", "pms_submit", "pms_poll", "pms_create",
                 "pms_destroy", "pms_result_free", "pms_strerror", "pms_solve_device"]:
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_lists_every_export():
    from paper_1307_0571_gb300 import pms
    assert sorted(pms.EXPORTS) == _declared()


def test_strerror(lib):
    from paper_1307_0571_gb300 import pms
    assert pms.strerror(pms.PMS_OK) == "ok"
    assert "alphabet" in pms.strerror(pms.PMS_E_ALPHABET)
    assert pms.strerror(12345) == "unknown error"


def test_no_device_fails_loudly(lib):
    # without a usable sm_103a GPU the library refuses to run (no CPU fallback)
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1307_0571_gb300 import pms
    with pytest.raises(pms.PMSError) as e:
        pms.Context(0)
    assert e.value.code == pms.PMS_E_CUDA


def test_struct_sizes_match_header(lib):
    # a C compile of the header gives the struct sizes the binding must match
    import subprocess
    import tempfile
    from paper_1307_0571_gb300 import pms
    prog = r'''
#include <stdio.h>
#include "pms.h"
int main(void){printf("%zu %zu %zu %zu\n", sizeof(pms_opts), sizeof(pms_instance),
 sizeof(pms_stats), sizeof(pms_result)); return 0;}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "s")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        sizes = [int(v) for v in subprocess.check_output([exe]).split()]
    assert sizes == [ctypes.sizeof(pms.pms_opts), ctypes.sizeof(pms.pms_instance),
                     ctypes.sizeof(pms.pms_stats), ctypes.sizeof(pms.pms_result)]
