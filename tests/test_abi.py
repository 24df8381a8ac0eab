"""CPU checks of the C-ABI library: it builds, loads and exports every symbol
that include/dotpe.h declares (no compute call needs a GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "dotpe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dotpe_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2507_16022_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_symbols()
    for required in ("dotpe_bank_load", "dotpe_event_submit", "dotpe_event_poll", "dotpe_evidence",
                     "dotpe_lnl_blocks"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_symbol():
    import paper_2507_16022_gb300 as dp
    assert sorted(dp.SYMBOLS) == _declared_symbols()


def test_strerror_and_version(lib):
    import paper_2507_16022_gb300 as dp
    L = dp.load()
    assert L.dotpe_version() == 7
    assert L.dotpe_strerror(dp.DOTPE_E_ADMISSION).decode() == "event can never fit the HBM budget"
    assert L.dotpe_strerror(12345).decode() == "unknown status"


def test_null_arguments_are_rejected_without_a_device(lib):
    import paper_2507_16022_gb300 as dp
    L = dp.load()
    assert L.dotpe_create(None, None) == dp.DOTPE_E_INVALID
    assert L.dotpe_destroy(None) == dp.DOTPE_E_INVALID
    assert L.dotpe_bank_load(None, None, None) == dp.DOTPE_E_INVALID
    assert L.dotpe_event_submit(None, None, None) == dp.DOTPE_E_INVALID
    assert L.dotpe_evidence(None, 1, None) == dp.DOTPE_E_INVALID
    assert L.dotpe_preselect(None, None, None, None, None, None, None) == dp.DOTPE_E_INVALID
    assert L.dotpe_rb_weights(None, None, None, None) == dp.DOTPE_E_INVALID
    assert L.dotpe_bank_subset(None, 1, None, 1, None) == dp.DOTPE_E_INVALID
    assert L.dotpe_bank_save(None, 1, None) == dp.DOTPE_E_INVALID
    assert L.dotpe_bank_open(None, None, None) == dp.DOTPE_E_INVALID
    assert L.dotpe_evidence_merge(0, None, 1, 32, None, None) == dp.DOTPE_E_INVALID
    assert "null" in L.dotpe_last_error_message().decode()


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2507_16022_gb300 as dp
    with pytest.raises(dp.DotpeError) as ei:
        dp.dotpe_create(0)
    assert ei.value.status in (dp.DOTPE_E_DEVICE, dp.DOTPE_E_INVALID)


def test_ctypes_struct_sizes_match_header(lib):
    # compile-time sizes of the ABI structs, checked with the host compiler
    import subprocess
    import tempfile
    import paper_2507_16022_gb300 as dp
    code = r'''
#include <stdio.h>
#include "dotpe.h"
int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(dotpe_config), sizeof(dotpe_bank_desc),
 sizeof(dotpe_event_desc), sizeof(dotpe_event_stats), sizeof(dotpe_evidence_out),
 sizeof(dotpe_presel_desc), sizeof(dotpe_presel_out), sizeof(dotpe_rb_desc), sizeof(dotpe_shard));return 0;}
'''
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "s.c")
        exe = os.path.join(d, "s")
        open(src, "w").write(code)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe])
        sizes = [int(x) for x in subprocess.check_output([exe]).split()]
    assert sizes == [ctypes.sizeof(c) for c in (dp.dotpe_config, dp.dotpe_bank_desc,
                                               dp.dotpe_event_desc, dp.dotpe_event_stats,
                                               dp.dotpe_evidence_out, dp.dotpe_presel_desc,
                                               dp.dotpe_presel_out, dp.dotpe_rb_desc, dp.dotpe_shard)]
