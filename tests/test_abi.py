"""The C ABI library loads and exports every entry point include/quapi.h declares (CPU only)."""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "quapi.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = set(re.findall(r"\b(quapi_[a-z_0-9]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib_path():
    from paper_1205_6872_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("quapi_setup", "quapi_setup_eta", "quapi_propagate", "quapi_query_memory",
              "quapi_propagate_batch", "quapi_last_error", "quapi_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for n in sorted(_declared()):
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (quapi_[a-z_0-9]+)\b", out))
    assert _declared() <= exported


def test_binding_names_match_header(lib_path):
    from paper_1205_6872_gb300 import quapi
    assert set(quapi.EXPORTED) == _declared()
    for n in quapi.EXPORTED:
        assert callable(getattr(quapi, n))


def test_query_memory_host_only(lib_path):
    from paper_1205_6872_gb300 import quapi
    t, tot = quapi.quapi_query_memory(2, 14, quapi.QUAPI_FP32)
    assert t == 2 * 4 ** 14 * 8
    assert tot > t
    t64, _ = quapi.quapi_query_memory(2, 14, quapi.QUAPI_FP64)
    assert t64 == 2 * 4 ** 14 * 16
    t3, _ = quapi.quapi_query_memory(3, 8, quapi.QUAPI_FP64)
    assert t3 == 2 * 9 ** 8 * 16
    with pytest.raises(quapi.QuapiError):
        quapi.quapi_query_memory(4, 3, quapi.QUAPI_FP64)
    with pytest.raises(quapi.QuapiError):
        quapi.quapi_query_memory(2, 0, quapi.QUAPI_FP64)
    with pytest.raises(quapi.QuapiError):
        quapi.quapi_query_memory(2, 17, quapi.QUAPI_FP64)
    with pytest.raises(quapi.QuapiError):
        quapi.quapi_query_memory(2, 3, 16)


def test_opts_defaults(lib_path):
    from paper_1205_6872_gb300 import quapi
    o = quapi.quapi_opts_init()
    assert o.precision == quapi.QUAPI_FP64 and o.endpoint_mode == quapi.QUAPI_ENDPOINT_STRANG
    assert not o.workspace and o.workspace_bytes == 0
