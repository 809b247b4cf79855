"""Host-side checks of the C ABI: the library builds, loads and exports every declared entry point;
the Python binding carries the same names.  No compute call is made (no GPU needed)."""
import os
import re
import ctypes

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, 'include', 'egb.h')


def declared_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r'^\s*(?:egb_status|const char \*)\s*(egb_\w+)\s*\(', src, re.M)))


@pytest.fixture(scope='module')
def lib_path():
    from paper_2006_11945_gb300 import build
    return build.build()


def test_header_declares_the_method_calls():
    names = declared_functions()
    for n in ('egb_create', 'egb_medium', 'egb_source', 'egb_evolve', 'egb_superpose', 'egb_sync',
              'egb_release', 'egb_destroy', 'egb_last_error'):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_binding_has_the_same_names(lib_path):
    import paper_2006_11945_gb300 as egb
    for n in declared_functions():
        assert hasattr(egb, n) or n == 'egb_last_error', n
    egb.load()


def test_null_context_is_rejected_without_a_device(lib_path):
    import paper_2006_11945_gb300 as egb
    lib = egb.load()
    assert lib.egb_evolve(None, 1, 1, 0.5) == egb.EGB_E_INVALID
    assert lib.egb_sync(None) == egb.EGB_E_INVALID
