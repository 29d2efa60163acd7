"""The C-ABI library builds here (cross-compiled for sm_103a), loads, and exports every symbol
that include/abcore.h declares. No compute call is made (no GPU on this machine)."""

import ctypes
import os
import re
import subprocess

import pytest

from tests.conftest import ROOT


@pytest.fixture(scope="module")
def lib_path():
    from paper_2606_07148_gb300.buildlib import build
    return build()


def _declared():
    with open(os.path.join(ROOT, "include", "abcore.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*\*?\s*(abcore_\w+)\s*\(", text, re.M)))


def test_header_declares_the_api():
    names = _declared()
    for want in ["abcore_create", "abcore_destroy", "abcore_load_csr", "abcore_load_edges",
                 "abcore_compute", "abcore_compute_batch", "abcore_query_edge", "abcore_serve_start",
                 "abcore_serve_submit", "abcore_serve_poll", "abcore_serve_stop"]:
        assert want in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in _declared():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (abcore_\w+)", out))
    assert set(_declared()) <= exported


def test_binding_names_match_header(lib_path):
    from paper_2606_07148_gb300 import abi
    assert sorted(abi.EXPORTED) == _declared()
    for name in _declared():
        assert callable(getattr(abi, name))


def test_product_path_does_not_touch_the_oracle():
    pkg = os.path.join(ROOT, "paper_2606_07148_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                with open(os.path.join(dirpath, fn)) as f:
                    text = f.read()
                assert "import oracle" not in text and "from oracle" not in text, fn
                assert "abcore_oracle" not in text and "liboracle" not in text, fn


def test_errors_without_a_context(lib_path):
    from paper_2606_07148_gb300 import abi
    assert abi.abcore_destroy(None) == 0
    assert abi.abcore_last_error(None) == b""
    assert abi.abcore_compute(None, 1, 1, None, None, 0) == abi.ABCORE_EINVAL


def test_header_documents_every_parameter():
    # abcore_set_param's comment in the header lists every name the library accepts
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with open(os.path.join(root, "include", "abcore.h")) as f:
        header = f.read()
    block = header[header.index("/* Set a parameter by name"):header.index("int abcore_set_param(")]
    documented = set(re.findall(r'"([a-z0-9_]+)"', block))
    with open(os.path.join(root, "paper_2606_07148_gb300", "csrc", "api.cu")) as f:
        api = f.read()
    accepted = set(re.findall(r'k == "([a-z0-9_]+)"', api))
    assert accepted, "no parameter names found in the implementation"
    assert accepted == documented, (sorted(accepted - documented), sorted(documented - accepted))
