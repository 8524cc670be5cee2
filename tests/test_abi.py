"""The C-ABI library loads and exports every symbol include/*.h declares (CPU only)."""
import glob
import os
import re

import pytest

import paper_2407_06107_b300 as stf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(stf_\w+)\s*\(", src, flags=re.M))
    return names


def test_header_declares_entry_points():
    d = _declared()
    for need in ("stf_create", "stf_filter_shade", "stf_create_texture", "stf_create_volume",
                 "stf_march_volume", "stf_get_device_status", "stf_status_string"):
        assert need in d


def test_library_exports_every_declared_symbol():
    L = stf.lib()
    missing = [n for n in sorted(_declared()) if not hasattr(L, n)]
    assert not missing, missing


def test_binding_signatures_cover_header():
    # the Python binding marshals every entry point the header declares
    assert _declared() <= set(stf.SIGNATURES)


def test_status_strings_without_device():
    L = stf.lib()
    assert L.stf_status_string(0) == b"STF_OK"
    assert L.stf_status_string(6) == b"STF_ERR_DEVICE_STATUS"


def test_null_arguments_rejected_without_device():
    import ctypes as C
    L = stf.lib()
    assert L.stf_create(0, None, None) == 1            # STF_ERR_INVALID_ARG
    assert L.stf_destroy(None) == 1
    assert L.stf_filter_shade(None, 1, None, None, 0, 2, 0, 1, 1, 0, None) == 1
    assert L.stf_march_volume(None, 1, None, 1, 1, 1, 0, 2, 1, 1, 0, 0, 1, None, None) == 1
